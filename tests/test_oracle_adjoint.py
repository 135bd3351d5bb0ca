"""Pins for the oracle's adjoint formulas: central finite differences of the
FP64 dense solve (independent of the adjoint algebra) and symmetry facts."""

import numpy as np
import pytest

from oracle import adjoint, reference


def _problem(n=120, seed=0):
    rng = np.random.default_rng(seed)
    P = rng.random((n, 3))
    b = rng.standard_normal(n)
    g = rng.standard_normal(n)
    return P, b, g


def test_rbf_matches_workload_generator():
    from workloads import rbf_kernel
    P, _, _ = _problem(90)
    assert np.allclose(adjoint.rbf(P, 0.2), rbf_kernel(P, 0.2), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("use_b_as_g", [False, True])
def test_gradients_match_central_differences(use_b_as_g):
    P, b, g = _problem()
    if use_b_as_g:
        g = b.copy()          # L = b^T x: the adjoint solve equals the forward solve
    ell, lam = 0.2, 1e-2
    K = adjoint.rbf(P, ell)
    gr = adjoint.grads(K, b, lam, g, adjoint.rbf_dK_dell(P, ell))
    h = 1e-5
    fd_ell = (adjoint.loss(P, ell + h, lam, b, g) - adjoint.loss(P, ell - h, lam, b, g)) / (2 * h)
    assert gr["dtheta"] == pytest.approx(fd_ell, rel=1e-6)
    fd_lam = (adjoint.loss(P, ell, lam + h * 1e-2, b, g) - adjoint.loss(P, ell, lam - h * 1e-2, b, g)) / (2 * h * 1e-2)
    assert gr["dlam"] == pytest.approx(fd_lam, rel=1e-6)
    e = np.zeros_like(b)
    e[7] = 1.0
    fd_b7 = (g @ reference.solve_dense(K, b + h * e, lam) - g @ reference.solve_dense(K, b - h * e, lam)) / (2 * h)
    assert gr["db"][7] == pytest.approx(fd_b7, rel=1e-7)
    if use_b_as_g:
        assert np.allclose(gr["a"], gr["x"], rtol=1e-12)


def test_dK_dell_closed_form_one_pair():
    # two points at distance d: K = exp(-d^2/(2 l^2)), dK/dl = K d^2 / l^3
    P = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    d2, ell = 0.25, 0.15
    val = adjoint.rbf_dK_dell(P, ell)[0, 1]
    assert val == pytest.approx(np.exp(-d2 / (2 * ell ** 2)) * d2 / ell ** 3, rel=1e-14)
