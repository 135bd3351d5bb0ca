"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
* sketch patterns (integers): bit-exact;
* C = A S^T: elementwise within the recursive-summation bound
  |dC_ij| <= (k+1) u sum_k |A_ik||S_jk| (Higham, Thm 3.1 form), u the unit
  roundoff of the storage precision, k the number of terms;
* W, C~-Gram: relative to |M2|, FP32 data (BF16/FP32 Gram) vs FP64;
* solves: the relative residual in FP64 against the tolerance asked for, and
  |x - x*| / |x*| <= kappa * tol against the dense Cholesky solution.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import msp as omsp
from oracle import nystrom as onys
from oracle import reference, sketch
from workloads import make_workload

pytestmark = pytest.mark.gpu

SEED = 0x4D5350


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("n,rows,gamma,seed,stream", [
    (1000, 64, 8, SEED, 0), (257, 16, 16, 7, 2), (300, 8, 8, 123, 0), (64, 1000, 3, 1, 4),
    (5000, 1024, 8, SEED, 0)])
def test_pattern_bit_exact(ctx, n, rows, gamma, seed, stream):
    idx, sgn = ctx.sketch_pattern(n, rows, gamma, seed, stream)
    oi, os_ = sketch.embedding_pattern(n, rows, gamma, seed, stream)
    assert np.array_equal(idx.cpu().numpy(), oi.astype(np.int32))
    assert np.array_equal(sgn.cpu().numpy(), os_)


def _sum_bound(A, S, u):
    # elementwise bound (k+1) u sum_k |A_ik| |S_ck|, k = nnz in column c of S^T
    absA = np.abs(A)
    absS = np.abs(S.toarray())
    k = (absS != 0).sum(axis=1)[None, :]
    return (k + 2) * u * (absA @ absS.T)


@pytest.mark.parametrize("n,s,gamma,dt", [(1000, 128, 8, torch.float64), (1000, 100, 8, torch.float32),
                                          (777, 300, 5, torch.float32), (4100, 1024, 8, torch.float32),
                                          (33, 16, 4, torch.float64)])
def test_sketch_C_matches_oracle(ctx, n, s, gamma, dt):
    rng = np.random.default_rng(n + s)
    B = rng.standard_normal((n, n))
    A = (B + B.T) / 2
    A_dev = _cuda(A, dt)
    A_used = A_dev.double().cpu().numpy()        # the values the GPU actually read
    sk = ctx.sketch(A_dev, s, gamma, SEED)
    C = sk.C().double().cpu().numpy()
    S = sketch.sparse_embedding(n, s, gamma, SEED)
    Co = sketch.sketch_C(A_used, S)
    u = 2.0 ** -53 if dt == torch.float64 else 2.0 ** -24
    bound = _sum_bound(A_used, S, u) + 4 * u * np.abs(Co)
    assert np.all(np.abs(C - Co) <= bound)


@pytest.mark.parametrize("dt,phi,work", [(torch.float64, 256, "outlier"), (torch.float64, 0, "outlier"),
                                         (torch.float32, 512, "rbf"), (torch.float32, 0, "rbf")])
def test_nystrom_W_M2_and_factor(ctx, dt, phi, work):
    # FP64 data: the n=512 outlier spectrum (kappa ~ 1e8); FP32 data: the RBF
    # kernel (an FP32-accumulated Gram of an outlier C would be indefinite).
    w = make_workload(work, seed=3, n=512)
    A = w.A
    A_dev = _cuda(A, dt)
    A_used = A_dev.double().cpu().numpy()
    s = 64
    sk = ctx.sketch(A_dev, s, 8, SEED)
    lam, lam0 = w.lam, 0.05
    f = ctx.nystrom(sk, lam, lam0, phi=phi, gamma_phi=8, seed=SEED)
    parts = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in f.parts().items()}
    S = sketch.sparse_embedding(512, s, 8, SEED)
    Co = sketch.sketch_C(A_used, S)
    Wo = sketch.core_W(S, Co)
    import scipy.sparse as sp
    Phi = sketch.level2_embedding(512, phi, 8, SEED) if phi else sp.identity(512, format="csr")
    Cto = sketch.level2_sketch(Phi, Co)
    M2o = onys.level2_matrix(Cto, Wo, lam + lam0)
    u = 2.0 ** -53 if dt == torch.float64 else 2.0 ** -24
    assert parts["lambda_tilde"] == pytest.approx(lam + lam0, rel=1e-15)
    assert np.abs(parts["W"] - Wo).max() <= 512 * u * np.abs(Wo).max()
    assert np.array_equal(parts["W"], parts["W"].T)
    K = Cto.shape[0]
    assert np.abs(parts["M2"] - M2o).max() <= 4 * (K + 64) * u * np.abs(M2o).max()
    # L^{-1} (M2 + shift I) L^{-T} = I  (backward-stable Cholesky + inverse, FP64)
    Li = parts["Linv"]
    Mw = parts["M2"] + parts["shift"] * np.eye(s)
    E = Li @ Mw @ Li.T - np.eye(s)
    assert np.abs(E).max() <= 1e-13 * np.linalg.cond(Mw) + 1e-10


def test_solve_m1_matches_oracle_fp64(ctx):
    # well-conditioned PSD matrix so that the dense level-2 solve of the oracle
    # and the GPU's level-2 PCG are both accurate to ~1e-12
    n = 600
    rng = np.random.default_rng(12)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.logspace(2, -3, n) ** 0.4) @ Q.T
    A = 0.5 * (A + A.T)
    A_dev = _cuda(A, torch.float64)
    s = 64
    sk = ctx.sketch(A_dev, s, 8, SEED)
    f = ctx.nystrom(sk, 1e-2, 0.0, phi=256, gamma_phi=8, seed=SEED)
    r = np.random.default_rng(0).standard_normal(n)
    wg, its = ctx.solve_m1(f, _cuda(r), inner_tol=1e-14, max_inner=300)
    p = omsp.MspParams(s=s, phi=256, lam0=0.0, inner="exact")
    st = omsp.setup(A, 1e-2, p)
    wo = omsp.solve_m1(st, r, p)
    wg = wg.cpu().numpy()
    assert 0 < its < 300
    assert np.linalg.norm(wg - wo) <= 1e-9 * np.linalg.norm(wo)


def test_solve_fp64_outlier_workload(ctx):
    # n=1024, 32 outliers 1e4->1e2, tail i^-1.5, lam=1e-3, s=64, gamma=8 (FP64)
    w = make_workload("outlier", seed=0)
    lam0 = onys.lambda0_from_spectrum(w.sigma, 32)
    A_dev = _cuda(w.A, torch.float64)
    sk = ctx.sketch(A_dev, w.s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, lam0, phi=4 * w.s)
    # the workload's stopping rule: relative residual 1e-10
    x, info = ctx.solve(f, A_dev, _cuda(w.b), w.lam, precision="fp64", tol=1e-10, inner_tol=1e-10)
    x = x.cpu().numpy()
    xs = reference.solve_dense(w.A, w.b, w.lam)
    assert info["rel_resid"] <= 1e-10
    # evaluated in extended precision: in FP64 the residual of this system
    # (kappa ~ 1e7, |x| ~ 850 |b|) is only resolved to ~2.4e-10
    assert reference.rel_residual_extended(w.A, x, w.b, w.lam) <= 1.2e-10
    kappa = (w.sigma.max() + w.lam) / (w.sigma.min() + w.lam)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-10
    # oracle with the same parameters takes a similar number of iterations
    p = omsp.MspParams(s=w.s, lam0=lam0, phi=4 * w.s, tol=1e-10, inner_tol=1e-10)
    _, oinfo = omsp.solve(w.A, w.b, w.lam, p)
    # (the GPU count includes the refinement steps that correct the drift of
    # the recurrence residual, a few iterations each)
    slack = max(3, 0.15 * oinfo.outer_iters)
    assert oinfo.outer_iters - slack <= info["outer_iters"] <= oinfo.outer_iters + slack + 8 * (info["refine_steps"] - 1)


@pytest.mark.parametrize("n", [2048, 3000])
def test_solve_mixed_rbf_to_1e10(ctx, n):
    w = make_workload("rbf", seed=1, n=n)
    A32 = w.A.astype(np.float32)
    A64 = A32.astype(np.float64)             # the problem the GPU is given
    A_dev = _cuda(A32)
    s = max(128, w.s)
    sk = ctx.sketch(A_dev, s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=4 * s)
    x, info = ctx.solve(f, A_dev, _cuda(w.b), w.lam, precision="mixed", tol=1e-10)
    x = x.cpu().numpy()
    rr = reference.rel_residual(A64, x, w.b, w.lam)
    assert info["rel_resid"] <= 1e-10 and rr <= 1.2e-10
    xs = reference.solve_dense(A64, w.b, w.lam)
    ev = np.linalg.eigvalsh(A64)
    kappa = (ev.max() + w.lam) / (max(ev.min(), 0) + w.lam)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-10
    assert info["refine_steps"] >= 2


@pytest.mark.parametrize("s", [300, 640])
def test_solve_ragged_sketch_sizes(ctx, s):
    # padded sketch sizes that are not powers of two (s_pad = 384, 640)
    w = make_workload("rbf", seed=8, n=2500)
    A_dev = _cuda(w.A.astype(np.float32))
    sk = ctx.sketch(A_dev, s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    x, info = ctx.solve(f, A_dev, _cuda(w.b), w.lam, precision="mixed", tol=1e-10, max_inner=0)
    rr = reference.rel_residual(w.A.astype(np.float32).astype(np.float64), x.cpu().numpy(), w.b, w.lam)
    assert info["rel_resid"] <= 1e-10 and rr <= 1.2e-10


@pytest.mark.parametrize("n", [1000, 2048 + 77])
def test_packed_and_dense_A_pass_agree(ctx, n):
    # The sketch keeps a packed copy of A's upper 128 x 128 tiles; msp_solve uses
    # it when given the sketched A and the dense row pass for any other pointer
    # (here a copy). Both must converge to the same solution; ragged n exercises
    # the zero-padded last tile row/column.
    w = make_workload("rbf", seed=7, n=n)
    A_dev = _cuda(w.A.astype(np.float32))
    A_copy = A_dev.clone()
    sk = ctx.sketch(A_dev, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    b = _cuda(w.b)
    xp, ip = ctx.solve(f, A_dev, b, w.lam, precision="mixed", tol=1e-10, max_inner=0,
                       profile=1)
    xd, idn = ctx.solve(f, A_copy, b, w.lam, precision="mixed", tol=1e-10, max_inner=0,
                        profile=1)
    assert ip["rel_resid"] <= 1e-10 and idn["rel_resid"] <= 1e-10
    xs = reference.solve_dense(w.A.astype(np.float32).astype(np.float64), w.b, w.lam)
    for x in (xp, xd):
        assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-7 * np.linalg.norm(xs)
    assert abs(ip["outer_iters"] - idn["outer_iters"]) <= 2 + 0.05 * idn["outer_iters"]


@pytest.mark.parametrize("n", [257, 4096, 4100])
def test_fp64_residual_operator(ctx, n):
    # y = (A + lam I) x with FP64 accumulation from FP32 A (the refinement's
    # residual operator): exact widening of each A entry (zeros, subnormals
    # flushed, wide magnitudes) and FP64 sums, vs a host FP64 product.
    rng = np.random.default_rng(n)
    A = (rng.standard_normal((n, n)) * np.exp(rng.uniform(-30, 30, (n, n)))).astype(np.float32)
    A[rng.random((n, n)) < 0.05] = 0.0
    A[0, :8] = np.float32(1e-42)          # subnormals
    A_dev = _cuda(A)
    x = rng.standard_normal(n)
    y = ctx.matvec_f64(A_dev, _cuda(x), lam=0.37).cpu().numpy()
    A64 = A.astype(np.float64)
    A64[np.abs(A64) < np.finfo(np.float32).tiny] = 0.0
    ref = A64 @ x + 0.37 * x
    scale = np.abs(A64) @ np.abs(x) + 0.37 * np.abs(x)
    assert np.all(np.abs(y - ref) <= 4 * n * 2.0 ** -53 * scale)


@pytest.mark.parametrize("n", [4096, 16384 + 4])
def test_fp64_residual_operator_float_float_bound(ctx, n):
    # FP32 A with n and lda multiples of 4: the FP32-pipe float-float kernel.
    # Against an extended-precision product its error stays within
    # (n / 128 + 2) 2^-47 sum_j |a_ij x_j| (plus the FP64 rounding of y).
    rng = np.random.default_rng(n + 1)
    m = 512                                   # rows checked (a row block of A)
    A = rng.standard_normal((m, n)).astype(np.float32)
    A[:, ::7] *= np.float32(1e3)              # mixed magnitudes within a row
    full = np.zeros((n, n), dtype=np.float32)
    full[:m] = A
    x = rng.standard_normal(n) * np.exp(rng.uniform(-5, 5, n))
    y = ctx.matvec_f64(_cuda(full), _cuda(x), lam=0.5).cpu().numpy()[:m]
    Al = A.astype(np.float64).astype(np.longdouble)
    xl = x.astype(np.longdouble)
    ref = Al @ xl + np.longdouble(0.5) * xl[:m]
    scale = np.abs(A.astype(np.float64)) @ np.abs(x) + 0.5 * np.abs(x[:m])
    err = np.abs(y.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= (n / 128 + 2) * 2.0 ** -47 * scale + 2.0 ** -52 * np.abs(y))
    # and typically near the FP64 rounding of the result
    assert np.median(err / scale) < 2.0 ** -46


def test_solve_plain_fp32_rbf(ctx):
    # plain FP32 (no refinement): the FP32 recurrence reaches 1e-5 but the true
    # residual stalls near u32 * |A| |x| / |b|; check the normwise backward error
    w = make_workload("rbf", seed=2, n=2048)
    A64 = w.A.astype(np.float32).astype(np.float64)
    A_dev = _cuda(w.A.astype(np.float32))
    sk = ctx.sketch(A_dev, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=512)
    x, info = ctx.solve(f, A_dev, _cuda(w.b), w.lam, precision="fp32", tol=1e-5)
    x = x.cpu().numpy()
    rr = reference.rel_residual(A64, x, w.b, w.lam)
    normA = float(np.linalg.eigvalsh(A64).max())
    eta = reference.backward_error(A64, x, w.b, w.lam, norm_A=normA)
    assert rr <= 1e-3 and eta <= 1e-6
    assert info["rel_resid"] == pytest.approx(rr, rel=1e-6)


def test_zero_rhs_and_errors(ctx):
    from paper_2405_05865_gb300 import MspError
    w = make_workload("rbf", seed=3, n=512)
    A_dev = _cuda(w.A.astype(np.float32))
    sk = ctx.sketch(A_dev, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam)
    x, info = ctx.solve(f, A_dev, torch.zeros(512, dtype=torch.float64, device="cuda"), w.lam)
    assert torch.count_nonzero(x) == 0 and info["rel_resid"] == 0.0
    bad = torch.full((512,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(MspError) as e:
        ctx.solve(f, A_dev, bad, w.lam)
    assert e.value.status == 6
    with pytest.raises(MspError) as e:
        ctx.solve(f, A_dev, _cuda(w.b), -1.0)
    assert e.value.status == 1
    with pytest.raises(MspError) as e:
        ctx.sketch(A_dev, 8, 8)              # s < 16
    assert e.value.status == 1
    # iteration cap: MSP_ENOCONV with the last iterate returned
    x, info = ctx.solve(f, A_dev, _cuda(w.b), w.lam, precision="fp32", tol=1e-12, max_outer=2,
                        raise_on_noconv=False)
    assert info["status"] == 5 and info["outer_iters"] == 2 and torch.isfinite(x).all()


def test_negative_definite_reports_not_pd(ctx):
    # A = -5 I: M2 = 25 Pi^T Phi^T Phi Pi - 5 lam~ Pi^T Pi is still positive
    # definite, but p^T (A + lam I) p < 0 in the first level-1 step.
    from paper_2405_05865_gb300 import MspError
    n = 256
    A = -np.eye(n) * 5.0
    A_dev = _cuda(A, torch.float64)
    sk = ctx.sketch(A_dev, 32, 4, SEED)
    f = ctx.nystrom(sk, 1e-2)
    b = _cuda(np.random.default_rng(1).standard_normal(n))
    with pytest.raises(MspError) as e:
        ctx.solve(f, A_dev, b, 1e-2, precision="fp64")
    assert e.value.status == 4


# ---- certified |A|_2 lower bound and the backward-error stopping rule

@pytest.mark.parametrize("name,n,seed", [("rbf", 1500, 2), ("outlier", 700, 1)])
def test_norm_lower_bound_matches_oracle(ctx, name, n, seed):
    w = make_workload(name, seed=seed, n=n)
    A = np.asarray(w.A)
    dt = torch.float32 if A.dtype == np.float32 else torch.float64
    L = ctx.norm_lower_bound(_cuda(A, dt))
    Lo = reference.norm_lower_bound(A.astype(np.float64))
    # certified: at most the exact expression, within the FP32 chunk bound
    assert Lo * (1 - 1e-5) <= L <= Lo * (1 + 1e-12)


def test_solve_backward_error_rule(ctx):
    w = make_workload("rbf", seed=4, n=2048)
    A = _cuda(w.A)
    sk = ctx.sketch(A, s=128)
    f = ctx.nystrom(sk, lam=w.lam, phi=0)
    x, info = ctx.solve(f, A, _cuda(w.b), lam=w.lam, max_inner=0, criterion="backward", tol=1e-10,
                        refine_tol=1e-4)
    x = x.cpu().numpy()
    A64 = np.asarray(w.A, dtype=np.float64)
    Lo = reference.norm_lower_bound(A64)
    assert Lo * (1 - 1e-5) <= info["norm_lb"] <= Lo * (1 + 1e-12)
    # the bound the sketch took of A in its one pass (reused by every solve
    # with it) is, to the rounding of the FP32 chunk sums, the one the
    # stand-alone row pass gives and the one a solve takes itself of a copy;
    # all of them certified (at most |A|_2)
    lb_rows = ctx.norm_lower_bound(A)
    assert info["norm_lb"] == pytest.approx(lb_rows, rel=1e-6)
    _, info_c = ctx.solve(f, A.clone(), _cuda(w.b), lam=w.lam, max_inner=0, criterion="backward", tol=1e-10,
                          refine_tol=1e-4)
    assert info_c["norm_lb"] == lb_rows
    assert max(lb_rows, info["norm_lb"]) <= Lo * (1 + 1e-12)
    assert info["backward_err"] <= 1e-10
    top = float(np.linalg.eigvalsh(A64)[-1])
    eta = reference.backward_error(A64, x, w.b, w.lam, norm_A=top)
    assert eta <= info["backward_err"] * (1 + 1e-6) + 1e-16
    assert eta <= 1e-10


@pytest.mark.parametrize("n,pad", [(3000, 0), (2176, 5)])
def test_solve_full_host_buffers_match_device(ctx, n, pad):
    """msp_solve_full with host A, b, x (A copied in row chunks overlapped with
    the sketch and the packing; ragged last chunk; a strided host A when
    pad > 0) gives bit for bit the result of the device-resident call, and
    meets the backward-error rule on the host's FP64 residual."""
    w = make_workload("rbf", seed=4, n=n)
    A32 = np.ascontiguousarray(w.A.astype(np.float32))
    big = np.zeros((n, n + pad), dtype=np.float32)
    big[:, :n] = A32
    Ah = torch.from_numpy(big).pin_memory()[:, :n]
    bh = torch.from_numpy(w.b).pin_memory()
    opts = dict(tol=1e-10, refine_tol=1e-3, max_inner=0, criterion="backward")
    s = 256
    xh, info_h = ctx.solve_full(Ah, bh, w.lam, s, 8, 0.0, 0, 8, 0x4D5350, **opts)
    xd, info_d = ctx.solve_full(torch.from_numpy(A32).cuda(), bh.cuda(), w.lam, s, 8, 0.0, 0, 8, 0x4D5350, **opts)
    assert not xh.is_cuda
    assert np.array_equal(xh.numpy(), xd.cpu().numpy())
    # only the upper triangle of a host FP32 A is read: garbage below the
    # diagonal changes nothing
    junk = big.copy()
    low = np.tril_indices(n, -1)
    junk[low] = 7.0
    Aj = torch.from_numpy(junk).pin_memory()[:, :n]
    xj, _ = ctx.solve_full(Aj, bh, w.lam, s, 8, 0.0, 0, 8, 0x4D5350, **opts)
    assert np.array_equal(xj.numpy(), xh.numpy())
    assert info_h["outer_iters"] == info_d["outer_iters"]
    K = A32.astype(np.float64)
    x = xh.numpy()
    r = w.b - (K @ x + w.lam * x)
    L = reference.norm_lower_bound(K)
    assert np.linalg.norm(r) <= 1e-10 * ((L + w.lam) * np.linalg.norm(x) + np.linalg.norm(w.b))


def test_solve_many_matches_single_solves(ctx):
    """msp_solve_many: every column equals the single-RHS msp_solve of it with
    the same factor, bit for bit (columns are independent runs)."""
    w = make_workload("rbf", seed=6, n=1500)
    A = torch.from_numpy(np.ascontiguousarray(w.A.astype(np.float32))).cuda()
    sk = ctx.sketch(A, s=128)
    f = ctx.nystrom(sk, lam=w.lam, phi=0)
    B = torch.from_numpy(np.random.default_rng(3).standard_normal((1500, 5))).cuda()
    opts = dict(tol=1e-10, refine_tol=1e-3, max_inner=0, criterion="backward")
    X, infos = ctx.solve_many(f, A, B, w.lam, **opts)
    for j in range(5):
        x, info = ctx.solve(f, A, B[:, j].contiguous(), w.lam, **opts)
        assert torch.equal(X[:, j], x)
        assert infos[j]["outer_iters"] == info["outer_iters"] and infos[j]["status"] == 0
    X0, infos0 = ctx.solve_many(f, A, B[:, :0], w.lam, **opts)
    assert X0.shape == (1500, 0) and infos0 == []
    f.close()
    sk.close()
