"""The one-pass sketch of a symmetric FP32 A (Algorithm 1, steps 2-3, with
the packed tiles and the row statistics the solves keep) against the FP64
oracle and against the row-wise passes it replaces.

* C = A S^T: elementwise within the recursive-summation bound
  (k + 2) u sum |A_ik| |S_ck| of either summation order;
* the norm bound L of the backward-error rule the sketch keeps: the value
  of the row-wise statistics pass, and at most |A|_2;
* the packed tiles: a solve through them reaches the oracle's solution.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return ((B + B.T) / 2).astype(np.float32)


def _bound(A, S, u):
    absS = np.abs(S.toarray())
    k = (absS != 0).sum(axis=1)[None, :]
    return (k + 2) * u * (np.abs(A) @ absS.T)


@pytest.mark.parametrize("n,s,gamma", [(1028, 128, 8), (4096, 1024, 8), (4096, 2048, 8), (2080, 640, 4),
                                       (300, 64, 3)])
def test_one_pass_C_matches_oracle_and_row_pass(ctx, n, s, gamma):
    A = _sym(n, n + s)
    A_dev = torch.from_numpy(A).cuda()
    S = sketch.sparse_embedding(n, s, gamma, SEED)
    Co = sketch.sketch_C(A.astype(np.float64), S)
    bound = _bound(A.astype(np.float64), S, 2.0 ** -24) + 4 * 2.0 ** -24 * np.abs(Co)
    out = {}
    for one in (True, False):
        ctx.set_sketch_one_pass(one)
        try:
            sk = ctx.sketch(A_dev, s, gamma, SEED)
            out[one] = sk.C().double().cpu().numpy()
            sk.close()
        finally:
            ctx.set_sketch_one_pass(True)
    for C in out.values():
        assert np.all(np.abs(C - Co) <= bound)
    assert np.all(np.abs(out[True] - out[False]) <= 2 * bound)


@pytest.mark.parametrize("n", [1000, 4100])
def test_one_pass_norm_bound_matches_row_statistics(ctx, n):
    w = make_workload("rbf", seed=4, n=n)
    A32 = w.A.astype(np.float32)
    A_dev = torch.from_numpy(A32).cuda()
    lb_rows = ctx.norm_lower_bound(A_dev)           # row-wise statistics kernel
    s = max(128, w.s)
    sk = ctx.sketch(A_dev, s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    x, info = ctx.solve(f, A_dev, torch.from_numpy(w.b).cuda(), w.lam, precision="mixed", tol=1e-10,
                        criterion="backward")
    lb_pass = info["norm_lb"]
    assert lb_pass == lb_rows           # the same row-statistics pass
    A64 = A32.astype(np.float64)
    assert lb_pass <= np.linalg.norm(A64, 2) * (1 + 1e-12)
    # the solve read A through the pass's packed tiles
    xs = reference.solve_dense(A64, w.b, w.lam)
    ev = np.linalg.eigvalsh(A64)
    kappa = (ev.max() + w.lam) / (max(ev.min(), 0) + w.lam)
    assert np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs) <= kappa * 1e-9
    f.close()
    sk.close()


def test_one_pass_padding_tiles_are_zero(ctx):
    # n = 1000: the last tile column holds 24 padding columns and rows; a
    # solve whose x would pick up garbage there stays at the oracle solution,
    # and the same solve through the separate passes agrees to the tolerance
    n = 1000
    w = make_workload("rbf", seed=5, n=n)
    A32 = w.A.astype(np.float32)
    A_dev = torch.from_numpy(A32).cuda()
    xs = []
    for one in (True, False):
        ctx.set_sketch_one_pass(one)
        try:
            sk = ctx.sketch(A_dev, 128, 8, SEED)
            f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
            x, info = ctx.solve(f, A_dev, torch.from_numpy(w.b).cuda(), w.lam, precision="mixed", tol=1e-10)
            assert np.isfinite(x.cpu().numpy()).all()
            assert reference.rel_residual(A32.astype(np.float64), x.cpu().numpy(), w.b, w.lam) <= 1.2e-10
            xs.append(x.cpu().numpy())
            f.close()
            sk.close()
        finally:
            ctx.set_sketch_one_pass(True)
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-8 * np.linalg.norm(xs[1])
