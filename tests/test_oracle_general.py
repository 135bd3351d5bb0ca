"""Pins of the three-level oracle for (A^T A + lambda I) x = c (CPU only).

Each level is checked against a dense statement that does not share its
arithmetic:
* Algorithm 5 (SolveM2) with exact level-3 solves equals (W^2 + lambda~ W)^{-1} r
  for W = A~^T A~ formed densely (the identity of Section 5);
* the level-3 systems, preconditioned by the sketched M3a, M3b, have O(1)
  condition numbers (the embedding property the paper relies on);
* Algorithm 4 (SolveM1) with an exact level-2 solve equals M^{-1} r for the
  dense M = C W^{-1} C^T + lambda~ I, C = A^T A~ (the Woodbury identity);
* the level-2 matrix C^T C + lambda~ W and M2 = W^2 + lambda~ W are within a
  factor 2 of each other for the paper's lambda0 (the spectral approximation
  behind M2, Section 5), so kappa <= 4;
* the full solve (iterated levels) reaches the dense solution;
* with S = I and lambda0 = 0 the preconditioner is the system itself and
  level 1 takes one iteration;
* the generator's singular values are the prescribed ones.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import general
from workloads import householder_spectrum, svd_matrix

M, N, K, LAM = 1200, 192, 8, 1e-3
S = 128      # s = 8 l with l = 2 K: the spectral approximation holds with margin


@pytest.fixture(scope="module")
def problem():
    sig = householder_spectrum(N, K, 4, hi=1e2, lo=1e1)
    A = svd_matrix(M, N, sig, 5)
    l = 2 * K
    lam0 = 2.0 / l * float(np.sum(sig[l:] ** 2))
    return A, sig, lam0


def _setup(problem, s=S, **kw):
    A, sig, lam0 = problem
    p = general.GenParams(s=s, lam0=lam0, **kw)
    return general.setup(A, LAM, p), p


def test_generator_singular_values(problem):
    A, sig, _ = problem
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(np.sort(sv)[::-1], np.sort(sig)[::-1], rtol=1e-12, atol=0)


def test_solve_m2_is_inverse_of_w2_plus_lam_w(problem):
    st, p = _setup(problem, level3="exact")
    W = st.At.T @ st.At
    M2 = W @ W + st.lam_tilde * W
    r = np.random.default_rng(1).standard_normal(p.s)
    z = general.solve_m2(st, r, p)
    ref = np.linalg.solve(M2, r)
    # (u - v) / lambda~ cancels: rounding of the two solves, about
    # u kappa(W) |v|, is amplified by |W| / lambda~
    ew = np.linalg.eigvalsh(W)
    bound = 16 * 2.0 ** -52 * (ew[-1] / ew[0]) * (1 + ew[-1] / st.lam_tilde)
    assert np.linalg.norm(z - ref) <= bound * np.linalg.norm(ref)
    assert bound < 1e-5


def test_level3_preconditioners_are_fine(problem):
    st, p = _setup(problem)
    W = st.At.T @ st.At
    # phi = 4 s rows: an embedding distortion near 1/2, so kappa about 8 for
    # M3a; the shift lambda~ I common to both sides pulls M3b closer
    for L, shift, cap in ((st.L3a, 0.0, 12.0), (st.L3b, st.lam_tilde, 4.0)):
        Li = np.linalg.inv(L)
        ev = np.linalg.eigvalsh(Li @ (W + shift * np.eye(p.s)) @ Li.T)
        assert ev[-1] / ev[0] <= cap, ev[-1] / ev[0]


def test_solve_m2_iterated_reaches_exact(problem):
    st, p = _setup(problem, t3=40)
    st_e, p_e = _setup(problem, level3="exact")
    r = np.random.default_rng(2).standard_normal(p.s)
    z = general.solve_m2(st, r, p)
    ref = general.solve_m2(st_e, r, p_e)
    assert np.linalg.norm(z - ref) <= 1e-8 * np.linalg.norm(ref)


def test_level2_matvec_is_ct_c_plus_lam_w(problem):
    st, p = _setup(problem)
    Cm = st.A.T @ st.At
    W = st.At.T @ st.At
    y = np.random.default_rng(3).standard_normal(p.s)
    ref = Cm.T @ (Cm @ y) + st.lam_tilde * (W @ y)
    got = general.level2_matvec(st, y)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_solve_m1_exact_is_woodbury(problem):
    st, p = _setup(problem, level2="exact")
    Mfull = general.dense_preconditioner(st)
    r = np.random.default_rng(4).standard_normal(N)
    w = general.solve_m1(st, r, p)
    ref = np.linalg.solve(Mfull, r)
    assert np.linalg.norm(w - ref) <= 1e-8 * np.linalg.norm(ref)


def test_level2_preconditioner_within_factor_two(problem):
    st, p = _setup(problem)
    Cm = st.A.T @ st.At
    W = st.At.T @ st.At
    B = Cm.T @ Cm + st.lam_tilde * W
    M2 = W @ W + st.lam_tilde * W
    # generalized eigenvalues of (B, M2) via the Cholesky of M2
    L = np.linalg.cholesky(M2)
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ B @ Li.T)
    assert ev[0] >= 0.5 and ev[-1] <= 2.0, (ev[0], ev[-1])


def test_full_solve_reaches_dense_solution(problem):
    A, _, _ = problem
    st, p = _setup(problem, tol=1e-10)
    c = np.random.default_rng(5).standard_normal(N)
    x, res = general.solve(A, c, LAM, p, st)
    assert res.converged
    xs = np.linalg.solve(A.T @ A + LAM * np.eye(N), c)
    r = c - general.matvec(A, LAM, x)
    lmin = np.linalg.eigvalsh(A.T @ A)[0] + LAM
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c) * 1.0001
    assert np.linalg.norm(x - xs) <= np.linalg.norm(r) / lmin * 1.01 + 1e-14 * np.linalg.norm(xs)
    # the preconditioner does its job: far fewer iterations than the
    # square root of kappa(A^T A + lam I) that plain CG needs
    kappa = (np.linalg.eigvalsh(A.T @ A)[-1] + LAM) / lmin
    assert res.iters < 0.25 * np.sqrt(kappa) * np.log(2e10)


def test_identity_sketch_gives_one_iteration(problem):
    A, _, _ = problem
    S = sp.identity(N, format="csr")
    # one exact application of M^{-1} = (A^T A + lam I)^{-1}; the Woodbury
    # form cancels by |A|^2 / lam, so lam = 1 keeps that factor at 1e4 and
    # the residual after the step near 1e-11
    p = general.GenParams(s=N, lam0=0.0, level2="exact", level3="exact", tol=1e-8)
    st = general.setup(A, 1.0, p, S=S)
    c = np.random.default_rng(6).standard_normal(N)
    x, res = general.solve(A, c, 1.0, p, st)
    assert res.iters == 1 and res.converged


def test_lambda_tilde_must_be_positive(problem):
    A, _, _ = problem
    with pytest.raises(ValueError):
        general.setup(A, 0.0, general.GenParams(s=16, lam0=0.0))
