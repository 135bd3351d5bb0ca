"""Pins for the oracle's Nystrom preconditioner, Krylov solvers and the MSP
driver (Algorithms 1, 2, 6, 7; Lemma 4.3/4.4; Section 6). Ground truths are
dense Cholesky/eigendecompositions, scipy's CG, exact algebraic identities and
special cases that reduce to a textbook computation."""

import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import krylov, msp, nystrom, reference, sketch
from workloads import make_workload, outlier_spectrum, spectrum_matrix


def _psd(n, seed, decay=1.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(2, -3, n) ** decay
    return (Q * ev) @ Q.T, ev


# ---------------------------------------------------------------- Nystrom / M --

def test_woodbury_identity_dense():
    # Eq. M_inverse: M (1/lam~)(I - C (C^T C + lam~ W)^{-1} C^T) = I
    A, _ = _psd(200, 0)
    S = sketch.sparse_embedding(200, 30, 4, seed=3)
    C = sketch.sketch_C(A, S)
    W = sketch.core_W(S, C)
    lt = 0.37
    M = nystrom.nystrom_preconditioner_dense(C, W, lt)
    R = np.random.default_rng(1).standard_normal((200, 3))
    Minv_R = np.stack([nystrom.woodbury_inverse_apply(C, W, lt, R[:, k]) for k in range(3)], 1)
    assert np.allclose(M @ Minv_R, R, rtol=0, atol=1e-9 * np.abs(R).max())


def test_nystrom_below_A_and_lemma43_sandwich():
    # A^ = C W^{-1} C^T satisfies A^ <= A (proof of Lemma 4.4). With
    # lam0 := |A - A^|_2, A + lam I <= M <= A + (lam + lam0) I (Lemma 4.3), so
    # kappa(M^{-1/2}(A + lam I)M^{-1/2}) <= 1 + lam0 / (lam_n + lam).
    n = 160
    A, ev = _psd(n, 2)
    S = sketch.sparse_embedding(n, 40, 8, seed=5)
    C = sketch.sketch_C(A, S)
    W = sketch.core_W(S, C)
    Ahat = C @ np.linalg.solve(W, C.T)
    d = np.linalg.eigvalsh(A - 0.5 * (Ahat + Ahat.T))
    assert d.min() > -1e-9 * ev.max()
    lam = 1e-2
    lam0 = float(d.max())
    M = Ahat + (lam + lam0) * np.eye(n)
    M = 0.5 * (M + M.T)
    mu = sla.eigh(A + lam * np.eye(n), M, eigvals_only=True)
    kappa = mu.max() / mu.min()
    assert mu.max() <= 1 + 1e-8
    assert kappa <= 1 + lam0 / (ev.min() + lam) + 1e-6


def test_level2_with_orthogonal_phi_is_exact():
    # If Phi is orthogonal (a signed permutation, phi = n) then C~^T C~ = C^T C and
    # M2 equals the level-2 operator C^T C + lam~ W exactly (up to rounding).
    n, s = 120, 24
    A, _ = _psd(n, 4)
    S = sketch.sparse_embedding(n, s, 4, seed=6)
    C = sketch.sketch_C(A, S)
    W = sketch.core_W(S, C)
    perm = np.random.default_rng(0).permutation(n)
    sg = np.where(np.random.default_rng(1).random(n) < 0.5, -1.0, 1.0)
    Phi = sp.csr_matrix((sg, (perm, np.arange(n))), shape=(n, n))
    Ct = sketch.level2_sketch(Phi, C)
    M2 = nystrom.level2_matrix(Ct, W, 0.5)
    G = C.T @ C + 0.5 * W
    assert np.allclose(M2, G, rtol=1e-12, atol=1e-12 * np.abs(G).max())


def test_cholesky_shift_paths():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((30, 30))
    spd = B @ B.T + np.eye(30)
    f = nystrom.cholesky_with_shift(spd)
    assert f.shift == 0.0 and np.allclose(f.L @ f.L.T, spd)
    # exactly singular PSD: plain Cholesky may fail; with the shift it succeeds
    V = rng.standard_normal((30, 5))
    sing = V @ V.T
    f = nystrom.cholesky_with_shift(sing)
    assert np.allclose(f.L @ f.L.T, sing + f.shift * np.eye(30), atol=1e-10)
    v = rng.standard_normal(30)
    assert np.allclose((sing + f.shift * np.eye(30)) @ f.solve(v), v, atol=1e-6 * np.abs(v).max() * 1e6)
    # clearly indefinite: no admissible shift
    with pytest.raises(nystrom.NotPositiveDefinite):
        nystrom.cholesky_with_shift(-np.eye(30))


def test_lambda0_closed_form_outlier_spectrum():
    # n=1024 outlier spectrum, l = 32: sum_{i>32} i^{-1.5} (i = 33..1024), times 2/l.
    sig = outlier_spectrum(1024, 32)
    tail = sum(i ** -1.5 for i in range(33, 1025))
    assert nystrom.lambda0_from_spectrum(sig, 32) == pytest.approx(2 / 32 * tail, rel=1e-14)


# ------------------------------------------------------------------- Krylov --

def _small_system(n=60, seed=0):
    A, _ = _psd(n, seed, decay=0.6)
    b = np.random.default_rng(seed + 1).standard_normal(n)
    rng = np.random.default_rng(seed + 2)
    E = rng.standard_normal((n, n)) * 0.1
    M = A + np.eye(n) + E @ E.T           # an SPD preconditioner
    return A, b, M


def test_alg6_alg7_pcg_agree_exact_preconditioner():
    # Section 6: with SolveM applied exactly, Algorithm 6, Algorithm 7 and PCG
    # produce the same iterate x_t; the tridiagonals of Alg 6 and Alg 7 coincide.
    A, b, M = _small_system()
    mv = lambda v: A @ v
    sm = lambda r: np.linalg.solve(M, r)
    for t in (1, 3, 7, 12):
        r6 = krylov.lanczos_left(mv, b, sm, t)
        r7 = krylov.lanczos_sym(mv, b, M, t)
        rp = krylov.pcg(mv, b, sm, tol=0.0, maxit=t)
        scale = np.linalg.norm(r7.x)
        assert np.linalg.norm(r6.x - r7.x) <= 1e-9 * scale
        assert np.linalg.norm(rp.x - r7.x) <= 1e-9 * scale
        assert np.allclose(r6.alpha, r7.alpha, rtol=1e-8)
        assert np.allclose(r6.beta[: t - 1], r7.beta[: t - 1], rtol=1e-8)


def test_pcg_matches_scipy_cg():
    A, b, M = _small_system(80, 3)
    Minv = np.linalg.inv(M)
    xs = []
    spla.cg(A, b, M=Minv, rtol=1e-12, maxiter=15, callback=lambda xk: xs.append(xk.copy()))
    for flexible in (False, True):
        r = krylov.pcg(lambda v: A @ v, b, lambda v: Minv @ v, tol=0.0, maxit=len(xs),
                       flexible=flexible)
        assert np.linalg.norm(r.x - xs[-1]) <= 1e-8 * np.linalg.norm(xs[-1])


def test_pcg_energy_error_monotone_and_cg_bound():
    # Krylov optimality: |x_t - x*|_A decreases monotonically; the count to eps is
    # within the classical bound ceil(sqrt(kappa)/2 * ln(2/eps)).
    A, b, M = _small_system(90, 5)
    xs_star = np.linalg.solve(A, b)
    errs = []
    Minv = np.linalg.inv(M)
    def cb_mv(v):
        return A @ v
    res = krylov.pcg(cb_mv, b, lambda v: Minv @ v, tol=1e-10, maxit=500)
    # recompute energy errors by re-running with growing maxit
    for t in range(1, res.iters + 1):
        x = krylov.pcg(cb_mv, b, lambda v: Minv @ v, tol=0.0, maxit=t).x
        e = x - xs_star
        errs.append(math.sqrt(e @ A @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))
    mu = sla.eigh(A, M, eigvals_only=True)
    kappa = mu.max() / mu.min()
    e0 = math.sqrt(xs_star @ A @ xs_star)
    t_eps = next(t for t, e in enumerate(errs, 1) if e <= 1e-8 * e0)
    assert t_eps <= math.ceil(0.5 * math.sqrt(kappa) * math.log(2 / 1e-8)) + 1


def test_scalar_preconditioner_gives_plain_cg():
    # lam0 >> |A|: M ~ lam~ I, a scalar preconditioner, so MSP's outer PCG iterates
    # equal textbook unpreconditioned CG (scipy) to rounding.
    n = 100
    A, _ = _psd(n, 7, decay=0.5)
    b = np.random.default_rng(3).standard_normal(n)
    p = msp.MspParams(s=10, lam0=1e12, inner="exact", outer="pcg", tol=0.0, max_outer=8)
    x, info = msp.solve(A, b, 0.1, p)
    xs = []
    spla.cg(A + 0.1 * np.eye(n), b, rtol=1e-15, maxiter=8, callback=lambda xk: xs.append(xk.copy()))
    assert np.linalg.norm(x - xs[-1]) <= 1e-7 * np.linalg.norm(xs[-1])


# ---------------------------------------------------------------- MSP solve --

def test_signed_permutation_sketch_converges_in_one_step():
    # S a signed permutation (s = n): A^ = A, so with lam0 = 0 the preconditioner
    # is M = A + lam I exactly and PCG converges in one outer iteration.
    n = 64
    A, _ = _psd(n, 8, decay=0.7)
    b = np.random.default_rng(2).standard_normal(n)
    perm = np.random.default_rng(5).permutation(n)
    sg = np.where(np.random.default_rng(6).random(n) < 0.5, -1.0, 1.0)
    S = sp.csr_matrix((sg, (perm, np.arange(n))), shape=(n, n))
    p = msp.MspParams(s=n, lam0=0.0, inner="exact", tol=1e-9)
    st = msp.setup(A, 0.05, p, S=S)
    x, info = msp.solve(A, b, 0.05, p, st=st)
    assert info.outer_iters == 1
    assert np.allclose(x, reference.solve_dense(A, b, 0.05), rtol=1e-8)


def test_block_diagonal_special_case():
    # Lower-bound construction (Section 7): A = [[M, 0], [0, sigma I]]; the
    # solution of (A + lam I) x = b is ((M + lam I)^{-1} b1, b2 / (sigma + lam)).
    k, m = 20, 80
    Mk, _ = _psd(k, 9)
    A = np.zeros((k + m, k + m))
    A[:k, :k] = Mk
    A[k:, k:] = 0.3 * np.eye(m)
    b = np.random.default_rng(4).standard_normal(k + m)
    lam = 1e-2
    x, info = msp.solve(A, b, lam, msp.MspParams(s=32, tol=1e-12, inner_tol=1e-13))
    assert info.converged
    x1 = np.linalg.solve(Mk + lam * np.eye(k), b[:k])
    assert np.allclose(x[:k], x1, rtol=1e-8, atol=1e-10 * np.abs(x1).max())
    assert np.allclose(x[k:], b[k:] / (0.3 + lam), rtol=1e-9)


@pytest.mark.parametrize("outer", ["fcg", "pcg", "lanczos"])
def test_msp_outlier_workload_matches_cholesky(outer):
    # n=1024, 32 outliers 1e4->1e2, tail i^-1.5, lam=1e-3, s=64, gamma=8; the
    # paper's lam0 = (2/l) sum_{i>l} sigma_i with l = 32.
    w = make_workload("outlier", seed=0)
    lam0 = nystrom.lambda0_from_spectrum(w.sigma, 32)
    p = msp.MspParams(s=w.s, lam0=lam0, outer=outer, max_outer=300 if outer == "lanczos" else 2000)
    x, info = msp.solve(w.A, w.b, w.lam, p)
    xs = reference.solve_dense(w.A, w.b, w.lam)
    kappa = (w.sigma.max() + w.lam) / (w.sigma.min() + w.lam)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-9 * kappa ** 0.5
    eta = reference.backward_error(w.A, x, w.b, w.lam, norm_A=w.sigma.max())
    assert eta <= 1e-13
    if outer != "lanczos":
        assert info.converged and info.outer_iters < 80


def test_solve_m1_pcg_inner_converges_to_exact_level2():
    # Algorithm 2 with a tight level-2 tolerance equals SolveM1 with the level-2
    # system solved densely (well-conditioned A so both are accurate to ~1e-12).
    n = 256
    A, _ = _psd(n, 12, decay=0.4)
    pe = msp.MspParams(s=48, inner="exact")
    pi = msp.MspParams(s=48, inner="pcg", inner_tol=1e-15, max_inner=300)
    st = msp.setup(A, 1e-2, pe)
    r = np.random.default_rng(0).standard_normal(n)
    we = msp.solve_m1(st, r, pe)
    wi = msp.solve_m1(st, r, pi)
    assert np.linalg.norm(we - wi) <= 1e-10 * np.linalg.norm(we)
    # and both equal the dense Woodbury form of M^{-1} r
    wd = nystrom.woodbury_inverse_apply(st.C, st.W, st.lam_tilde, r)
    assert np.linalg.norm(we - wd) <= 1e-10 * np.linalg.norm(we)


def test_refinement_reaches_target():
    w = make_workload("outlier", seed=2, n=256)
    p = msp.MspParams(s=w.s, tol=1e-4, inner_tol=1e-6)
    st = msp.setup(w.A, w.lam, p)
    corr = lambda r: msp.solve(w.A, r, w.lam, p, st=st)[0]
    # each correction solve reduces |r| by ~1e-4; the FP64 floor of this system
    # (|A| |x| / |b| ~ 1e6) is ~2e-10, so ask for 1e-9
    x, hist = msp.refine(w.A, w.b, w.lam, corr, tol=1e-9)
    assert hist[-1] <= 1e-9
    assert all(hist[i + 1] < 1e-3 * hist[i] for i in range(len(hist) - 2))
    assert hist[-1] < hist[-2]
    assert 3 <= len(hist) <= 5
    xs = reference.solve_dense(w.A, w.b, w.lam)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


# ----------------------------------------------------------- definitions --

def test_dense_solve_and_backward_error():
    A, ev = _psd(120, 11)
    b = np.random.default_rng(0).standard_normal(120)
    x = reference.solve_dense(A, b, 0.2)
    assert np.allclose(x, np.linalg.solve(A + 0.2 * np.eye(120), b), rtol=1e-10)
    assert reference.backward_error(A, x, b, 0.2, norm_A=ev.max()) < 1e-15
    # eta is scale-invariant and at most the relative residual
    y = x * (1 + 1e-6)
    eta = reference.backward_error(A, y, b, 0.2, norm_A=ev.max())
    assert eta <= reference.rel_residual(A, y, b, 0.2)
    assert abs(reference.norm2_power(A, iters=300) - ev.max()) <= 1e-8 * ev.max()


def test_effective_dimension_and_schatten_closed_forms():
    sig = outlier_spectrum(400, 12)
    A = spectrum_matrix(sig, seed=3)
    lam = 1e-3
    dense = np.trace(np.linalg.solve(A + lam * np.eye(400), A))
    assert reference.effective_dimension(sig, lam) == pytest.approx(dense, rel=1e-9)
    assert reference.schatten(sig, 1.0) == pytest.approx(np.linalg.norm(A, "nuc"), rel=1e-10)
    assert reference.schatten(sig, 1.0) == pytest.approx(np.trace(A), rel=1e-12)
    ev = np.linalg.eigvalsh(A)
    assert reference.schatten(sig, 0.5) == pytest.approx(np.sum(np.abs(ev) ** 0.5) ** 2, rel=1e-8)


# ---- certified lower bound of |A|_2 and the backward-error bound

def test_norm_lower_bound_closed_forms():
    from oracle import reference as ref
    n = 37
    # A = 1 1^T: |A|_2 = n, the all-ones Rayleigh quotient attains it
    assert ref.norm_lower_bound(np.ones((n, n))) == pytest.approx(n, rel=1e-15)
    # A = I: every column has norm 1 = |A|_2
    assert ref.norm_lower_bound(np.eye(n)) == pytest.approx(1.0, rel=1e-15)
    # A = v v^T with one spike: the column norm |v_k| |v| attains |v|^2 when v = e_k
    v = np.zeros(n)
    v[5] = 3.0
    assert ref.norm_lower_bound(np.outer(v, v)) == pytest.approx(9.0, rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_norm_lower_bound_below_the_norm(seed):
    from oracle import reference as ref
    from workloads import make_workload
    for name in ("outlier", "rbf"):
        w = make_workload(name, seed=seed, n=256, rbf_dtype=np.float64)
        A = np.asarray(w.A, dtype=np.float64)
        L = ref.norm_lower_bound(A)
        top = float(np.linalg.eigvalsh(A)[-1])
        assert 0.0 < L <= top * (1 + 1e-12)
        if name == "rbf":
            # positive kernel: the ones quotient is within a small factor
            assert L >= 0.25 * top


def test_backward_error_bound_dominates():
    from oracle import reference as ref
    from workloads import make_workload
    w = make_workload("rbf", seed=3, n=200, rbf_dtype=np.float64)
    A = np.asarray(w.A, dtype=np.float64)
    xs = ref.solve_dense(A, w.b, w.lam)
    x = xs + 1e-6 * np.random.default_rng(0).standard_normal(xs.shape)
    exact = ref.backward_error(A, x, w.b, w.lam, norm_A=float(np.linalg.eigvalsh(A)[-1]))
    assert ref.backward_error_bound(A, x, w.b, w.lam) >= exact * (1 - 1e-12)


# ---- energy norm of the error (the norm of Theorem 3.2's guarantee)

def test_energy_error_pins():
    # Pinned by identities that do not use its formula:
    #  * x = 0 gives exactly 1;
    #  * x = x* + t q_i (q_i an eigenvector of A) gives |t| sqrt(s_i + lam) / |x*|_E
    #    with |x*|_E^2 = b^T x* (since (A + lam I) x* = b);
    #  * |x - x*|_E^2 = r^T (A + lam I)^{-1} r for the residual r = b - (A + lam I) x.
    n, lam = 150, 0.03
    A, ev = _psd(n, 21)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(n)
    xs = np.linalg.solve(A + lam * np.eye(n), b)
    assert reference.energy_error(A, np.zeros(n), xs, lam) == pytest.approx(1.0, rel=1e-12)
    w, V = np.linalg.eigh(A)
    i, t = 17, 0.37
    x = xs + t * V[:, i]
    want = abs(t) * math.sqrt(w[i] + lam) / math.sqrt(b @ xs)
    assert reference.energy_error(A, x, xs, lam) == pytest.approx(want, rel=1e-9)
    x = xs + 1e-3 * rng.standard_normal(n)
    r = b - (A @ x + lam * x)
    want = math.sqrt(r @ np.linalg.solve(A + lam * np.eye(n), r) / (b @ xs))
    assert reference.energy_error(A, x, xs, lam) == pytest.approx(want, rel=1e-8)


@pytest.mark.parametrize("outer", ["fcg", "pcg"])
def test_msp_outer_energy_error_monotone_exact_level2(outer):
    # Krylov optimality of the outer iteration (Algorithm 1 step 5 with an exact
    # SolveM1, so M is fixed): |x_t - x*|_{A + lam I} never increases, while
    # |r_t| may. Outlier workload, n = 1024, the paper's lam0 with l = 32.
    w = make_workload("outlier", seed=1)
    lam0 = nystrom.lambda0_from_spectrum(w.sigma, 32)
    base = msp.MspParams(s=w.s, lam0=lam0, inner="exact", outer=outer, tol=0.0)
    st = msp.setup(w.A, w.lam, base)
    xs = reference.solve_dense(w.A, w.b, w.lam)
    # 25 iterations stay above the FP64 floor of this system (kappa ~ 1e7: the
    # energy error settles near 4e-10 after ~28 iterations, where rounding,
    # not the Krylov recurrence, sets the increments)
    errs = []
    for t in range(1, 26):
        p = dataclasses.replace(base, max_outer=t)
        x, _ = msp.solve(w.A, w.b, w.lam, p, st=st)
        errs.append(reference.energy_error(w.A, x, xs, w.lam))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))
    assert errs[-1] <= 1e-8


def test_extended_residual_exact_on_integers():
    # integer A (< 2^28) and x (< 2^28), n = 16: every product and partial
    # sum is an integer below 2^60, exact in the extended type (64-bit or
    # 113-bit significand) but not in FP64. b is an FP64 number near A x, so
    # the exact residual r = b - (A + I) x is a small integer vector, computed
    # here with Python integers; FP64 evaluation misses it by ~2^7 per entry
    rng = np.random.default_rng(7)
    n = 16
    Ai = [[int(v) for v in row] for row in rng.integers(-2**28, 2**28, (n, n))]
    xi = [int(v) for v in rng.integers(-2**28, 2**28, n)]
    ax = [sum(Ai[i][j] * xi[j] for j in range(n)) + xi[i] for i in range(n)]
    b = np.array([float(v) for v in ax])                 # rounded to FP64
    r = [int(b[i]) - ax[i] for i in range(n)]            # exact
    want = math.sqrt(sum(v * v for v in r)) / math.sqrt(sum(int(v) ** 2 for v in b))
    A = np.array(Ai, dtype=np.float64)
    x = np.array(xi, dtype=np.float64)
    got = reference.rel_residual_extended(A, x, b, 1.0)
    assert want > 0 and got == pytest.approx(want, rel=1e-9, abs=0.0)
    assert reference.rel_residual(A, x, b, 1.0) != pytest.approx(want, rel=1e-3, abs=0.0)
