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
