"""Parity at the benchmarked sizes, in the configuration bench.py times.

* RBF n = 16384, s = 1024, Phi = I, direct level 2, mixed precision to
  backward error 1e-10 (the headline solve);
* the batched RBF workload: 64 instances, n ~ U{512..8192}, 16 right-hand
  sides each (1024 solves), backward error 1e-10 per column.

Inputs come from the seeded generators on the host (FP64 kernel values
rounded once to FP32), never from the CUDA path. Every solution is checked on
the host in FP64: the normwise backward error |r| / ((L + lam)|x| + |b|)
with L <= |A|_2 (the oracle's certified bound, so the value is an upper
bound on the true backward error), and |x - x*| <= |r| / lam (A PSD), which
bounds the distance to the exact solution without factoring A.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import reference

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _eta(K64, x, b, lam, L):
    r = b - (K64 @ x + lam * x)
    return float(np.linalg.norm(r) / ((L + lam) * np.linalg.norm(x) + np.linalg.norm(b))), r


def test_rbf16k_headline_solve(ctx):
    w = workloads.make_workload("rbf", seed=0, n=16384)
    A = torch.from_numpy(np.ascontiguousarray(w.A)).cuda()
    b = torch.from_numpy(w.b).cuda()
    sk = ctx.sketch(A, s=1024)
    f = ctx.nystrom(sk, lam=w.lam, phi=0)
    x, info = ctx.solve(f, A, b, lam=w.lam, max_inner=0, criterion="backward", tol=TOL, refine_tol=1e-3)
    x = x.cpu().numpy()
    f.close()
    sk.close()
    del A
    K64 = np.asarray(w.A, dtype=np.float64)
    L = reference.norm_lower_bound(K64)
    eta, r = _eta(K64, x, w.b, w.lam, L)
    assert info["status"] == 0 and info["backward_err"] <= TOL
    assert eta <= TOL, eta
    # the library's bound and the host's agree to well inside the tolerance
    assert abs(eta - info["backward_err"]) <= 0.05 * TOL
    # distance to the exact solution x* = (A + lam I)^{-1} b
    assert np.linalg.norm(r) / w.lam <= 1e-4 * np.linalg.norm(x)


def test_batch64_bench_configuration(ctx):
    specs = workloads.batch_specs(0, count=64)
    insts, dev = [], []
    for sp in specs:
        _, K, B = workloads.batch_instance(sp)
        insts.append((K, B, sp))
        dev.append(dict(A=torch.from_numpy(K).cuda(), B=torch.from_numpy(B).cuda(), lam=sp.lam, s=sp.s))
    bt = ctx.batch(dev)
    infos = bt.solve(tol=TOL, refine_tol=1e-4, criterion="backward")
    worst = 0.0
    for k, ((K, B, sp), info) in enumerate(zip(insts, infos)):
        assert info["status"] == 0 and info["backward_err"] <= TOL, (k, info)
        X = bt.X(k).cpu().numpy()
        K64 = K.astype(np.float64)
        L = reference.norm_lower_bound(K64)
        R = B - (K64 @ X + sp.lam * X)
        for j in range(sp.m):
            eta = float(np.linalg.norm(R[:, j]) / ((L + sp.lam) * np.linalg.norm(X[:, j]) + np.linalg.norm(B[:, j])))
            assert eta <= TOL, (k, j, eta)
            worst = max(worst, eta)
            assert np.linalg.norm(R[:, j]) / sp.lam <= 1e-3 * np.linalg.norm(X[:, j])
    bt.close()
    assert worst > 0.0
