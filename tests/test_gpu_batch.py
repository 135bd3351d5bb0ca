"""Batched MSP (msp_batch_create / msp_batch_solve) against the FP64 oracle.

Tolerances:
* every column: |b - (A + lam I) x| / |b| <= tol recomputed here in FP64 from
  the stored FP32 matrix (the problem the library was given);
* the solution against the dense Cholesky oracle by the bound
  |x - x*| <= |r| / lam (A PSD);
* independence of the columns (no coupling): permuting the right-hand sides
  or repeating an instance permutes / repeats the solutions bit for bit;
* the batched result and a single-RHS msp_solve of the same column agree
  within the sum of their residual bounds.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import reference

pytestmark = pytest.mark.gpu

LAM = 1e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _instance(n, ell, m, seed, s):
    spec = workloads.BatchSpec(n, ell, LAM, s, m, seed)
    _, K, B = workloads.batch_instance(spec)
    return K, B


def _check_column(K, b, x, lam, tol):
    K64 = K.astype(np.float64)
    r = b - (K64 @ x + lam * x)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        assert not np.any(x)
        return 0.0
    rel = np.linalg.norm(r) / nb
    assert rel <= tol, rel
    xs = reference.solve_dense(K64, b, lam)
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(r) / lam + 1e-12 * np.linalg.norm(xs)
    return rel


# ragged sizes spanning several 128-row blocks and 64-column tiles
CASES = [(300, 0.1, 3, 1, 64), (517, 0.07, 16, 2, 128), (640, 0.18, 5, 3, 128),
         (1000, 0.05, 16, 4, 192), (1283, 0.12, 1, 5, 320), (16, 0.3, 2, 6, 16)]


@pytest.fixture(scope="module")
def small_batch(ctx):
    insts = [_instance(*c) for c in CASES]
    dev = [dict(A=torch.from_numpy(K).cuda(), B=torch.from_numpy(B).cuda(), lam=LAM, s=c[4])
           for (K, B), c in zip(insts, CASES)]
    bt = ctx.batch(dev)
    infos = bt.solve(tol=1e-10, refine_tol=1e-6, max_refine=10)
    X = [bt.X(k).cpu().numpy() for k in range(len(CASES))]
    yield insts, dev, bt, infos, X
    bt.close()


def test_batch_mixed_meets_tolerance(small_batch):
    insts, _, _, infos, X = small_batch
    for (K, B), info, Xk in zip(insts, infos, X):
        assert info["status"] == 0
        assert info["rel_resid"] <= 1e-10
        for j in range(B.shape[1]):
            _check_column(K, B[:, j], Xk[:, j], LAM, 1e-10)


def test_batch_info_is_consistent(small_batch):
    """The library's refinement residual against one in extended precision on
    the host. The batched residual is float-float: x = x_hi + x_lo (FP32
    pair, 48 bits), exact FP32 products (FMA) summed as an unevaluated FP32
    pair (TwoSum). Its error is bounded by a small multiple of
    2^-48 |(|A| |x| + lam |x|)| per column; the test allows 4 times that."""
    insts, _, _, infos, X = small_batch
    u2 = 2.0 ** -48
    for (K, B), info, Xk in zip(insts, infos, X):
        Kl = K.astype(np.longdouble)
        Xl = Xk.astype(np.longdouble)
        R = B.astype(np.longdouble) - (Kl @ Xl + np.longdouble(LAM) * Xl)
        T = np.abs(K.astype(np.float64)) @ np.abs(Xk) + LAM * np.abs(Xk)
        nb = np.linalg.norm(B, axis=0)
        rel = max(float(np.sqrt(np.sum(R[:, j] ** 2)) / nb[j]) for j in range(B.shape[1]))
        bound = 4 * u2 * max(np.linalg.norm(T[:, j]) / nb[j] for j in range(B.shape[1]))
        assert abs(info["rel_resid"] - rel) <= bound, (info["rel_resid"], rel, bound)
        assert info["outer_iters"] > 0 and info["refine_steps"] >= 1


def test_batch_is_deterministic(ctx, small_batch):
    _, _, bt, _, X = small_batch
    bt.solve(tol=1e-10, refine_tol=1e-6, max_refine=10)
    for k in range(len(CASES)):
        assert np.array_equal(bt.X(k).cpu().numpy(), X[k])


def test_batch_columns_independent(ctx):
    K, B = _instance(700, 0.09, 6, 21, 128)
    perm = [3, 0, 5, 1, 4, 2]
    A = torch.from_numpy(K).cuda()
    insts = [dict(A=A, B=torch.from_numpy(B).cuda(), lam=LAM, s=128),
             dict(A=A, B=torch.from_numpy(np.ascontiguousarray(B[:, perm])).cuda(), lam=LAM, s=128),
             dict(A=A, B=torch.from_numpy(B).cuda(), lam=LAM, s=128)]
    bt = ctx.batch(insts)
    bt.solve(tol=1e-10, refine_tol=1e-6)
    X0, X1, X2 = (bt.X(k).cpu().numpy() for k in range(3))
    bt.close()
    assert np.array_equal(X1, X0[:, perm])
    assert np.array_equal(X2, X0)


def test_batch_matches_single_rhs_solve(ctx):
    K, B = _instance(900, 0.1, 2, 31, 192)
    A = torch.from_numpy(K).cuda()
    bt = ctx.batch([dict(A=A, B=torch.from_numpy(B).cuda(), lam=LAM, s=192)])
    bt.solve(tol=1e-10, refine_tol=1e-6)
    Xb = bt.X(0).cpu().numpy()
    bt.close()
    sk = ctx.sketch(A, s=192)
    f = ctx.nystrom(sk, lam=LAM, phi=0)
    K64 = K.astype(np.float64)
    for j in range(2):
        xs, info = ctx.solve(f, A, torch.from_numpy(B[:, j].copy()).cuda(), lam=LAM, max_inner=0,
                             refine_tol=1e-6)
        xs = xs.cpu().numpy()
        r1 = np.linalg.norm(B[:, j] - (K64 @ Xb[:, j] + LAM * Xb[:, j]))
        r2 = np.linalg.norm(B[:, j] - (K64 @ xs + LAM * xs))
        assert np.linalg.norm(Xb[:, j] - xs) <= 1.01 * (r1 + r2) / LAM


def test_batch_zero_rhs_and_fp32(ctx):
    K, B = _instance(400, 0.1, 3, 41, 64)
    B[:, 1] = 0.0
    A = torch.from_numpy(K).cuda()
    bt = ctx.batch([dict(A=A, B=torch.from_numpy(B).cuda(), lam=LAM, s=64)])
    infos = bt.solve(tol=1e-10, refine_tol=1e-6)
    X = bt.X(0).cpu().numpy()
    assert infos[0]["status"] == 0
    assert not np.any(X[:, 1])
    # plain FP32: one correction solve, no refinement; residual near FP32 level
    infos = bt.solve(precision="fp32", tol=1e-5)
    X = bt.X(0).cpu().numpy()
    assert infos[0]["refine_steps"] == 1
    for j in (0, 2):
        _check_column(K, B[:, j], X[:, j], LAM, 1e-4)
    bt.close()


def test_batch_graph_capture(ctx):
    """The solve is one asynchronous launch: capture it in a CUDA graph and
    replay; the result equals the eager one bit for bit."""
    from paper_2405_05865_gb300 import Context
    K, B = _instance(600, 0.1, 4, 51, 128)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c2 = Context(0, stream=s)
        A = torch.from_numpy(K).cuda()
        bt = c2.batch([dict(A=A, B=torch.from_numpy(B).cuda(), lam=LAM, s=128)])
        bt.solve(tol=1e-10, refine_tol=1e-6)
        X_eager = bt.X(0).clone()
        bt.X(0).zero_()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        bt.solve(sync=False, tol=1e-10, refine_tol=1e-6)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bt.X(0), X_eager)
    infos = bt.info()
    assert infos[0]["status"] == 0 and infos[0]["rel_resid"] <= 1e-10
    bt.close()
    c2.close()


def test_batch_bad_arguments(ctx):
    from paper_2405_05865_gb300 import MspError
    K, B = _instance(100, 0.1, 1, 61, 32)
    A = torch.from_numpy(K).cuda()
    Bd = torch.from_numpy(B).cuda()
    with pytest.raises(MspError):
        ctx.batch([dict(A=A, B=Bd, lam=LAM, s=512)])            # s > n
    with pytest.raises(MspError):
        ctx.batch([dict(A=A, B=Bd, lam=-1.0, s=32)])            # lam <= 0
    with pytest.raises(MspError):
        B17 = torch.zeros((100, 17), dtype=torch.float64, device="cuda")
        ctx.batch([dict(A=A, B=B17, lam=LAM, s=32)])            # m > 16


def test_batch_backward_error_rule(ctx):
    """Smooth and rough kernels under the backward-error rule: every column's
    normwise backward error, recomputed here with the exact |A|_2, is at most
    tol, and the library's L matches the oracle's bound."""
    cases = [(1500, 0.2, 16, 71, 320), (800, 0.05, 7, 72, 192)]
    insts = [_instance(*c) for c in cases]
    dev = [dict(A=torch.from_numpy(K).cuda(), B=torch.from_numpy(B).cuda(), lam=LAM, s=c[4])
           for (K, B), c in zip(insts, cases)]
    bt = ctx.batch(dev)
    infos = bt.solve(tol=1e-10, refine_tol=1e-4, criterion="backward")
    for k, ((K, B), info) in enumerate(zip(insts, infos)):
        K64 = K.astype(np.float64)
        X = bt.X(k).cpu().numpy()
        assert info["status"] == 0 and info["backward_err"] <= 1e-10
        Lo = reference.norm_lower_bound(K64)
        assert Lo * (1 - 1e-5) <= info["norm_lb"] <= Lo * (1 + 1e-12)
        top = float(np.linalg.eigvalsh(K64)[-1])
        for j in range(B.shape[1]):
            eta = reference.backward_error(K64, X[:, j], B[:, j], LAM, norm_A=top)
            assert eta <= 1e-10
    bt.close()


def test_batch_multi_unit_rows(ctx):
    """Instances wide enough that each 128-row block of A is streamed as
    several units whose partial products are summed by the block that
    finishes last (at 32 tiles per unit, n = 2500: 2 units, n = 4200: 3
    units per row block), next to a one-unit instance; backward error checked
    with the exact |A|_2, and repeated solves identical bit for bit."""
    cases = [(2500, 0.1, 4, 81, 320), (4200, 0.15, 3, 82, 512), (700, 0.08, 2, 83, 128)]
    insts = [_instance(*c) for c in cases]
    dev = [dict(A=torch.from_numpy(K).cuda(), B=torch.from_numpy(B).cuda(), lam=LAM, s=c[4])
           for (K, B), c in zip(insts, cases)]
    bt = ctx.batch(dev)
    assert bt.autotune(32) == 32
    infos = bt.solve(tol=1e-10, refine_tol=1e-4, criterion="backward")
    X1 = [bt.X(k).cpu().numpy() for k in range(len(cases))]
    bt.solve(tol=1e-10, refine_tol=1e-4, criterion="backward")
    for k, ((K, B), info) in enumerate(zip(insts, infos)):
        assert np.array_equal(bt.X(k).cpu().numpy(), X1[k])      # fixed-order unit sums
        K64 = K.astype(np.float64)
        assert info["status"] == 0 and info["backward_err"] <= 1e-10
        top = float(np.linalg.eigvalsh(K64)[-1])
        for j in range(B.shape[1]):
            x = X1[k][:, j]
            assert reference.backward_error(K64, x, B[:, j], LAM, norm_A=top) <= 1e-10
            r = B[:, j] - (K64 @ x + LAM * x)
            xs = reference.solve_dense(K64, B[:, j], LAM)
            assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(r) / LAM + 1e-12 * np.linalg.norm(xs)
    bt.close()


def test_batch_unit_width(ctx):
    """Every unit width gives a certified solution; the search returns a
    width it tried; bad widths are refused."""
    from paper_2405_05865_gb300 import MspError
    cases = [(2600, 0.12, 3, 91, 320), (900, 0.07, 2, 92, 128)]
    insts = [_instance(*c) for c in cases]
    dev = [dict(A=torch.from_numpy(K).cuda(), B=torch.from_numpy(B).cuda(), lam=LAM, s=c[4])
           for (K, B), c in zip(insts, cases)]
    bt = ctx.batch(dev)
    for ut in (16, 32, 64):
        assert bt.autotune(ut) == ut
        infos = bt.solve(tol=1e-10, refine_tol=1e-4, criterion="backward")
        for k, ((K, B), info) in enumerate(zip(insts, infos)):
            assert info["status"] == 0 and info["backward_err"] <= 1e-10
            X = bt.X(k).cpu().numpy()
            K64 = K.astype(np.float64)
            for j in range(B.shape[1]):
                r = B[:, j] - (K64 @ X[:, j] + LAM * X[:, j])
                assert np.linalg.norm(r) <= 1.01e-10 * ((info["norm_lb"] + LAM) * np.linalg.norm(X[:, j])
                                                        + np.linalg.norm(B[:, j]))
    found = bt.autotune(0)
    assert found in (16, 32, 64)
    for bad in (8, 48):
        with pytest.raises(MspError):
            bt.autotune(bad)
    bt.close()


def test_batch_shared_setup_matches_separate_copies(ctx):
    """Instances naming one A (same sizes, lam, sketch parameters) share one
    set-up; the result equals that of a batch given separate copies of A."""
    K, B = _instance(777, 0.08, 16, 41, 128)
    K2, B2 = _instance(450, 0.2, 7, 42, 64)
    A = torch.from_numpy(K).cuda()
    cols = [B[:, :16], B[:, 3:13], B[:, :5][:, ::-1]]
    shared = [dict(A=A, B=torch.from_numpy(np.ascontiguousarray(c)).cuda(), lam=LAM, s=128) for c in cols]
    shared.insert(1, dict(A=torch.from_numpy(K2).cuda(), B=torch.from_numpy(B2).cuda(), lam=LAM, s=64))
    copies = [dict(d, A=d["A"].clone()) for d in shared]
    bt_s, bt_c = ctx.batch(shared), ctx.batch(copies)
    info_s = bt_s.solve(tol=1e-10, refine_tol=1e-6)
    info_c = bt_c.solve(tol=1e-10, refine_tol=1e-6)
    for k in range(len(shared)):
        assert info_s[k]["status"] == 0
        assert np.array_equal(bt_s.X(k).cpu().numpy(), bt_c.X(k).cpu().numpy())
        assert info_s[k]["shift"] == info_c[k]["shift"]
    for k in (0, 2, 3):
        X = bt_s.X(k).cpu().numpy()
        Bk = shared[k]["B"].cpu().numpy()
        for j in range(X.shape[1]):
            _check_column(K, Bk[:, j], X[:, j], LAM, 1e-10)
    bt_s.close()
    bt_c.close()
