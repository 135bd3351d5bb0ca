"""Pins of the least-squares oracle (sketch-and-precondition with MSP inner
solves; CPU only).

* A~ = Phi A is a constant-factor subspace embedding: the eigenvalues of
  (A~^T A~)^{-1} A^T A lie in [1/4, 4] for s_ls = 4 d;
* with the exact preconditioner (A~^T A~)^{-1} the outer flexible PCG reaches
  the least-squares solution of numpy.linalg.lstsq in O(log 1/eps) steps;
* with inexact MSP inner solves (Theorem 3.1 on A~, lambda = 0) it still
  converges, and |A x - b|^2 <= min |A x - b|^2 + eps |b|^2 (the corollary);
* b in the range of A: the residual vanishes.
"""

import numpy as np
import pytest

from oracle import general, lsq
from workloads import householder_spectrum, svd_matrix

N, D, K = 2000, 96, 6


@pytest.fixture(scope="module")
def problem():
    sig = householder_spectrum(D, K, 3, hi=1e2, lo=1e1)
    A = svd_matrix(N, D, sig, 4)
    b = np.random.default_rng(5).standard_normal(N)
    return A, sig, b


def _inner(sig, s=48):
    l = 2 * K
    lam0 = 2.0 / l * float(np.sum(sig[l:] ** 2))
    return general.GenParams(s=s, lam0=lam0, t2=8, t3=8)


def test_sketch_is_a_subspace_embedding(problem):
    A, sig, b = problem
    p = lsq.LsqParams(s_ls=4 * D)
    At = lsq.sketch_rows(A, p)
    G = At.T @ At
    ev = np.linalg.eigvals(np.linalg.solve(G, A.T @ A)).real
    assert ev.min() >= 0.25 and ev.max() <= 4.0, (ev.min(), ev.max())


def test_exact_preconditioner_reaches_lstsq(problem):
    A, sig, b = problem
    p = lsq.LsqParams(s_ls=4 * D, exact_inner=True, tol=1e-12)
    x, res, At = lsq.solve(A, b, p)
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    # the preconditioned CG bound: |r_k| <= 2 sqrt(kappa) ((sqrt k - 1)/(sqrt k + 1))^k |r_0|
    ev = np.linalg.eigvals(np.linalg.solve(At.T @ At, A.T @ A)).real
    kap = ev.max() / ev.min()
    rate = (np.sqrt(kap) - 1) / (np.sqrt(kap) + 1)
    bound = int(np.ceil(np.log(1e-12 / (2 * np.sqrt(kap))) / np.log(rate)))
    assert res.converged and res.iters <= bound, (res.iters, bound)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_msp_inner_solves_meet_the_corollary(problem):
    A, sig, b = problem
    p = lsq.LsqParams(s_ls=4 * D, inner=_inner(sig), inner_tol=1e-2, tol=1e-10)
    x, res, _ = lsq.solve(A, b, p)
    assert res.converged
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    best = np.linalg.norm(A @ xs - b) ** 2
    eps = 1e-12
    assert np.linalg.norm(A @ x - b) ** 2 <= best + eps * np.linalg.norm(b) ** 2
    # |x - x*| <= |A^T (b - A x)| / sigma_min^2
    g = A.T @ (b - A @ x)
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(g) / np.min(sig) ** 2 + 1e-13 * np.linalg.norm(xs)


def test_consistent_system_has_zero_residual(problem):
    A, sig, _ = problem
    xt = np.random.default_rng(6).standard_normal(D)
    b = A @ xt
    p = lsq.LsqParams(s_ls=4 * D, inner=_inner(sig), inner_tol=1e-2, tol=1e-12)
    x, res, _ = lsq.solve(A, b, p)
    assert np.linalg.norm(x - xt) <= 1e-9 * np.linalg.norm(xt)
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
