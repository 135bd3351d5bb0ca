"""Pins of the effective-dimension estimator (CPU only).

* A diagonal: every Rademacher probe gives g^T (A + lam I)^{-1} g =
  sum_i 1/(sigma_i + lam) exactly, so the estimate equals the closed form
  sum_i sigma_i/(sigma_i + lam) to rounding, with zero spread;
* A = Q diag(sigma) Q^T: the estimate lies within 5 standard errors of the
  closed form, and the spread of the probes matches the Rademacher variance
  2(|B|_F^2 - sum B_ii^2), B = lam (A + lam I)^{-1};
* the identity d_lambda = n - lam tr((A + lam I)^{-1}) against the dense
  inverse.
"""

import numpy as np
import pytest

from oracle import effdim, hutchinson, reference
from workloads import outlier_spectrum, spectrum_matrix


def test_diagonal_matrix_is_exact():
    sig = outlier_spectrum(200, 8)
    lam = 1e-2
    G = hutchinson.probes(200, 16, 5)
    est, se = effdim.estimate(np.diag(sig), lam, G)
    assert est == pytest.approx(reference.effective_dimension(sig, lam), rel=1e-13)
    assert se < 1e-10


def test_identity_with_the_dense_inverse():
    sig = outlier_spectrum(120, 6)
    A = spectrum_matrix(sig, 3)
    lam = 5e-3
    d = 120 - lam * np.trace(np.linalg.inv(A + lam * np.eye(120)))
    assert d == pytest.approx(reference.effective_dimension(sig, lam), rel=1e-9)


@pytest.mark.parametrize("seed", [1, 2])
def test_general_matrix_within_standard_errors(seed):
    n, m, lam = 256, 128, 1e-2
    sig = outlier_spectrum(n, 8)
    A = spectrum_matrix(sig, seed)
    G = hutchinson.probes(n, m, seed)
    est, se = effdim.estimate(A, lam, G)
    exact = reference.effective_dimension(sig, lam)
    assert abs(est - exact) <= 5 * se
    sd = np.sqrt(effdim.variance_one_probe(A, lam))
    assert se * np.sqrt(m) == pytest.approx(sd, rel=0.35)


@pytest.mark.parametrize("n,k,lam", [(1024, 32, 1e-3), (4096, 8, 1e-2), (2048, 64, 1e-1), (512, 4, 3e-2)])
def test_params_follow_lemma_2_1(n, k, lam):
    """With the exact d_lambda of a generated spectrum: lambda_l <= lambda
    (Lemma 2.1(1)), and when s >= d the shift bounds the paper's
    (2/s) sum_{i>s} lambda_i from above and is at most lambda (Lemma 2.1(2))."""
    sig = outlier_spectrum(n, k)
    d = reference.effective_dimension(sig, lam)
    p = effdim.params_from_effdim(d, n, lam)
    assert p["l"] >= 2 * d and p["l"] < 2 * d + 1
    if p["l"] <= n:
        assert sig[p["l"] - 1] <= lam          # lambda_l, 1-based
    assert p["s"] % 16 == 0 and 16 <= p["s"] <= min(n, 1024)
    assert p["capped"] == int(p["s"] < p["l"])
    if p["s"] >= d:
        tail = float(np.sum(sig[p["s"]:]))
        assert 2.0 * tail / p["s"] <= p["lambda0"] * (1 + 1e-12)
        assert p["lambda0"] <= lam * (1 + 1e-12)
    else:
        assert p["lambda0"] == 0.0
    assert p["direct"] == int(d >= n / 4)


def test_params_edge_cases():
    # tiny d: the smallest sketch, shift 2 lam d / 16
    p = effdim.params_from_effdim(0.3, 64, 1e-2)
    assert (p["l"], p["s"], p["capped"]) == (1, 16, 0)
    assert p["lambda0"] == pytest.approx(2 * 1e-2 * 0.3 / 16)
    # huge d: capped, no shift, direct regime
    p = effdim.params_from_effdim(3000.0, 16384, 1e-2)
    assert (p["s"], p["capped"], p["lambda0"], p["direct"]) == (1024, 1, 0.0, 0)
    p = effdim.params_from_effdim(300.0, 1000, 1e-2)
    assert (p["l"], p["s"], p["capped"], p["direct"]) == (600, 608, 0, 1)
    # capped at n rounded down to 16, still s >= d: the Lemma 2.1(2) shift
    p = effdim.params_from_effdim(600.0, 1000, 1e-2)
    assert (p["s"], p["capped"]) == (992, 1)
    assert p["lambda0"] == pytest.approx(2 * 1e-2 * 600 / 992)
    with pytest.raises(ValueError):
        effdim.params_from_effdim(-1.0, 64, 1e-2)
