"""The level-1 iterations of msp_solve replayed as a CUDA graph against the
same iterations launched one by one on the stream.

Both issue the same two kernels (the A pass, the level-2 kernel) in the same
order with the same arguments, and every reduction has a fixed order, so the
solution, the iteration counts and the residual agree bit for bit. The solve
itself is checked against the FP64 oracle (relative residual and the dense
solution). Profiling: each timed launch is one of an iteration that did work
(the launches queued after the device flagged convergence return at once and
are not counted), so the launch counts equal the level-1 iteration count on
both paths.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nystrom as onys
from oracle import reference
from workloads import make_workload

pytestmark = pytest.mark.gpu

SEED = 0x4D5350


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.set_level1_graphs(True)
    c.close()


def _cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _both(ctx, f, A, b, lam, **opts):
    out = {}
    for graphs in (True, False):
        ctx.set_level1_graphs(graphs)
        try:
            x, info = ctx.solve(f, A, b, lam, **opts)
        finally:
            ctx.set_level1_graphs(True)
        out[graphs] = (x.cpu().numpy(), info)
    return out


def _same(out):
    (xg, ig), (xs, is_) = out[True], out[False]
    assert np.array_equal(xg, xs)
    for k in ("outer_iters", "inner_iters", "refine_steps", "rel_resid", "status"):
        assert ig[k] == is_[k], k
    # replays include the ones queued after convergence (up to a check
    # interval per solve), which return at once
    assert ig["level1_graph_iters"] >= ig["outer_iters"]
    assert ig["level1_graph_iters"] > 0
    assert is_["level1_graph_iters"] == 0


@pytest.mark.parametrize("n,s,packed", [(1000, 128, True), (2048 + 77, 256, True), (3000, 384, False)])
def test_graph_and_stream_iterations_agree_fp32(ctx, n, s, packed):
    # packed: the sketched A (the packed-tile A pass); otherwise a copy of it
    # (the dense row pass); ragged n and several check intervals
    w = make_workload("rbf", seed=11, n=n)
    A_dev = _cuda(w.A, torch.float32)
    sk = ctx.sketch(A_dev, s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    A = A_dev if packed else A_dev.clone()
    out = _both(ctx, f, A, _cuda(w.b), w.lam, precision="mixed", tol=1e-10, check_every=3)
    _same(out)
    A64 = A_dev.double().cpu().numpy()
    x = out[True][0]
    assert reference.rel_residual(A64, x, w.b, w.lam) <= 1.2e-10
    xs = reference.solve_dense(A64, w.b, w.lam)
    ev = np.linalg.eigvalsh(A64)
    kappa = (ev.max() + w.lam) / (max(ev.min(), 0) + w.lam)
    assert np.linalg.norm(x - xs) <= kappa * 1e-9 * np.linalg.norm(xs)
    f.close()
    sk.close()


def test_graph_and_stream_iterations_agree_fp64(ctx):
    # FP64 A, sketch and vectors (the dense FP64 row pass), sketched level 2
    w = make_workload("outlier", seed=0)
    lam0 = onys.lambda0_from_spectrum(w.sigma, 32)
    A_dev = _cuda(w.A, torch.float64)
    sk = ctx.sketch(A_dev, w.s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, lam0, phi=4 * w.s)
    out = _both(ctx, f, A_dev, _cuda(w.b), w.lam, precision="fp64", tol=1e-10, inner_tol=1e-10)
    _same(out)
    assert out[True][1]["rel_resid"] <= 1e-10
    assert reference.rel_residual_extended(w.A, out[True][0], w.b, w.lam) <= 1.2e-10
    f.close()
    sk.close()


def test_graph_is_rebuilt_when_the_arguments_change(ctx):
    # a second lambda, a second factor and a second right-hand side in turn:
    # each solve meets the oracle's residual and matches the stream path
    w = make_workload("rbf", seed=12, n=1500)
    A_dev = _cuda(w.A, torch.float32)
    A64 = A_dev.double().cpu().numpy()
    sk = ctx.sketch(A_dev, 128, 8, SEED)
    rng = np.random.default_rng(3)
    for lam in (w.lam, 4 * w.lam):
        f = ctx.nystrom(sk, lam, 0.0, phi=0)
        for b in (w.b, rng.standard_normal(1500)):
            out = _both(ctx, f, A_dev, _cuda(b), lam, precision="mixed", tol=1e-10)
            _same(out)
            assert reference.rel_residual(A64, out[True][0], b, lam) <= 1.2e-10
        f.close()
    sk.close()


def test_iteration_cap_and_check_interval(ctx):
    # max_outer = 5 with check_every = 3: the cap falls inside a check
    # interval; both paths stop after 5 iterations with the same iterate
    w = make_workload("rbf", seed=13, n=1200)
    A_dev = _cuda(w.A, torch.float32)
    sk = ctx.sketch(A_dev, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    out = _both(ctx, f, A_dev, _cuda(w.b), w.lam, precision="fp32", tol=1e-12, max_outer=5,
                check_every=3, raise_on_noconv=False)
    _same(out)
    assert out[True][1]["status"] == 5 and out[True][1]["outer_iters"] == 5
    assert out[True][1]["level1_graph_iters"] == 5
    f.close()
    sk.close()


def test_profiled_launches_are_the_iterations_that_ran(ctx):
    # profile = 1 on both paths: one timed A pass and one timed level-2
    # launch per level-1 iteration that did work, durations of the same size
    w = make_workload("rbf", seed=14, n=4096)
    A_dev = _cuda(w.A, torch.float32)
    sk = ctx.sketch(A_dev, 256, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    out = _both(ctx, f, A_dev, _cuda(w.b), w.lam, precision="mixed", tol=1e-10, profile=1,
                criterion="backward")
    _same(out)
    per = {}
    for graphs, (_, info) in out.items():
        it = info["outer_iters"]
        assert info["gemv_launches"] == it and info["level2_launches"] == it
        assert info["gemv_ms"] > 0 and info["level2_ms"] > 0
        per[graphs] = (info["gemv_ms"] / it, info["level2_ms"] / it)
    for k in range(2):
        assert 0.5 < per[True][k] / per[False][k] < 2.0, per
    f.close()
    sk.close()
