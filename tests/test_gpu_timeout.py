"""Device-side waits give up instead of hanging: with the grid-barrier limit
of the level-1 / level-2 kernels lowered to a nanosecond, a solve's first
barrier times out, the call returns MSP_ETIMEOUT, and once the limit is
restored the same context solves the system correctly (bit for bit as
before). Nothing faults or hangs: the blocks that give up return, and every
solve resets its control block."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reference
from workloads import make_workload

pytestmark = pytest.mark.gpu
SEED = 0x4D5350


def test_grid_barrier_timeout_and_recovery():
    from paper_2405_05865_gb300 import Context, MspError
    ctx = Context(0)
    w = make_workload("rbf", seed=15, n=2048)
    A32 = w.A.astype(np.float32)
    A = torch.from_numpy(A32).cuda()
    b = torch.from_numpy(w.b).cuda()
    sk = ctx.sketch(A, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    opts = dict(precision="mixed", tol=1e-10, max_inner=0)
    x0, _ = ctx.solve(f, A, b, w.lam, **opts)
    ctx.set_grid_wait_limit(1e-9)
    try:
        with pytest.raises(MspError) as e:
            ctx.solve(f, A, b, w.lam, **opts)
        assert e.value.status == 7          # MSP_ETIMEOUT
    finally:
        ctx.set_grid_wait_limit(0.0)
    x1, info = ctx.solve(f, A, b, w.lam, **opts)
    assert info["status"] == 0
    assert torch.equal(x0, x1)
    assert reference.rel_residual(A32.astype(np.float64), x1.cpu().numpy(), w.b, w.lam) <= 1.2e-10
    with pytest.raises(MspError):
        ctx.set_grid_wait_limit(-1.0)
    f.close()
    sk.close()
    ctx.close()
