"""Pins of the Schatten-p oracle (integral representation over ridge solves;
CPU only).

* the quadrature with closed-form d_t reproduces sum sigma^p to 1e-8 for
  p in {0.5, 1, 1.5} with 80 nodes (pins the constant sin(pi q)/pi, the
  exponent q - 1 of t, the weights and both geometric tails), and its error
  falls geometrically as the step shrinks;
* p = 1 on a PSD matrix gives tr(A) (the Schatten-1 identity);
* a diagonal A: Rademacher probes give d_t exactly (zero spread), so the
  estimator equals the quadrature of the exact d_t;
* a general rectangular A: the Hutchinson estimate lies within 5 standard
  errors of the exact value;
* the shift z I moves the estimate to |A + z I|_p^p.
"""

import numpy as np
import pytest

from oracle import hutchinson, schatten
from workloads import householder_spectrum, outlier_spectrum, spectrum_matrix, svd_matrix


def _bounds(sig):
    e = np.asarray(sig) ** 2
    return 1e-6 * e.min(), 1e6 * e.max()


@pytest.mark.parametrize("p", [0.5, 1.0, 1.5])
def test_quadrature_with_exact_effdims(p):
    sig = householder_spectrum(300, 10, 2, hi=1e2, lo=1e1)
    t0, t1 = _bounds(sig)
    ex = float(np.sum(sig ** p))
    errs = []
    for count in (20, 40, 80):
        t, h = schatten.nodes(t0, t1, count)
        d = schatten.exact_effdims(sig, t)
        errs.append(abs(schatten.combine(p, t, h, d, sig.shape[0], float(np.sum(sig ** 2))) / ex - 1))
    assert errs[2] <= 1e-8
    assert errs[1] <= 1e-2 * errs[0] or errs[1] <= 1e-10


def test_p1_on_psd_is_the_trace():
    sig = outlier_spectrum(200, 6)
    A = spectrum_matrix(sig, 4)
    t0, t1 = _bounds(sig)
    t, h = schatten.nodes(t0, t1, 80)
    # the singular values of a PSD matrix are its eigenvalues
    d = schatten.exact_effdims(np.linalg.eigvalsh(A).clip(min=0), t)
    est = schatten.combine(1.0, t, h, d, 200, float(np.sum(A * A)))
    assert est == pytest.approx(float(np.trace(A)), rel=1e-6)


def test_diagonal_matrix_is_exact_per_probe():
    sig = householder_spectrum(120, 5, 7, hi=30.0, lo=3.0)
    A = np.diag(sig)
    G = hutchinson.probes(120, 6, 3)
    t0, t1 = _bounds(sig)
    est, se, X = schatten.estimate(A, 1.0, t0, t1, 120, G)
    t, h = schatten.nodes(t0, t1, 120)
    ref = schatten.combine(1.0, t, h, schatten.exact_effdims(sig, t), 120, float(np.sum(sig ** 2)))
    assert np.allclose(X, ref, rtol=1e-10)
    assert est == pytest.approx(float(np.sum(sig)), rel=1e-5)


@pytest.mark.parametrize("p", [0.7, 1.0, 1.3])
def test_general_matrix_within_standard_errors(p):
    sig = householder_spectrum(96, 6, 5, hi=1e2, lo=1e1)
    A = svd_matrix(400, 96, sig, 6)
    G = hutchinson.probes(96, 64, 9)
    t0, t1 = _bounds(sig)
    est, se, _ = schatten.estimate(A, p, t0, t1, 80, G)
    ex = schatten.exact(A, p)
    assert abs(est - ex) <= 5 * se + 1e-5 * ex
    assert se < 0.25 * ex          # Rademacher spread; the outliers dominate for larger p


def test_shift_moves_to_the_shifted_matrix():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((80, 80))
    z = 0.37
    G = hutchinson.probes(80, 48, 1)
    sv = np.linalg.svd(A + z * np.eye(80), compute_uv=False)
    t0, t1 = 1e-6 * sv.min() ** 2, 1e6 * sv.max() ** 2
    est, se, _ = schatten.estimate(A, 1.0, t0, t1, 120, G, z=z)
    ex = float(np.sum(sv))
    assert abs(est - ex) <= 5 * se + 1e-5 * ex
    with pytest.raises(ValueError):
        schatten.estimate(A[:, :40], 1.0, t0, t1, 10, G[:40], z=z)
