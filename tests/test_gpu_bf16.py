"""BF16 where the method tolerates it (reduced-precision storage is a choice
of this implementation; the paper works in exact arithmetic, Section 2):

* the level-2 preconditioner data C and W stored in BF16 (msp_nystrom_ex):
  C is rounded first and W, M2 are formed from the rounded C, so M stays an
  SPD preconditioner; the refined solve must still reach 1e-10 against the
  FP64 residual of the FP32 problem;
* the sketch pass C = A Pi reading a BF16-stored A, against the oracle's C of
  the same (rounded) matrix within the FP32 summation bound;
* the FP64-accumulated product with a BF16 A, against the host product.

BF16 values are taken on the host with torch's CPU conversion (round to
nearest even) and widened exactly to FP64."""

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


def _bf16_values(A):
    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("n,s,crit", [(2048 + 77, 256, "residual"), (4096, 384, "backward")])
def test_bf16_preconditioner_data_solve(ctx, n, s, crit):
    w = make_workload("rbf", seed=11, n=n)
    A32 = w.A.astype(np.float32)
    A64 = A32.astype(np.float64)
    A = torch.from_numpy(A32).cuda()
    b = torch.from_numpy(w.b).cuda()
    sk = ctx.sketch(A, s, 8, SEED)
    fb = ctx.nystrom(sk, w.lam, 0.0, phi=0, data="bf16")
    x, info = ctx.solve(fb, A, b, w.lam, precision="mixed", tol=1e-10, max_inner=0, criterion=crit)
    x = x.cpu().numpy()
    if crit == "residual":
        assert reference.rel_residual(A64, x, w.b, w.lam) <= 1.2e-10
    else:
        L = reference.norm_lower_bound(A64)
        r = reference.residual(A64, x, w.b, w.lam)
        eta = np.linalg.norm(r) / ((L + w.lam) * np.linalg.norm(x) + np.linalg.norm(w.b))
        assert eta <= 1e-10
    # the same system with FP32 data: BF16 data changes the preconditioner,
    # not the answer, and the iteration count only moderately
    ff = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    x2, info2 = ctx.solve(ff, A, b, w.lam, precision="mixed", tol=1e-10, max_inner=0, criterion=crit)
    xs = reference.solve_dense(A64, w.b, w.lam)
    for xx in (x, x2.cpu().numpy()):
        assert np.linalg.norm(xx - xs) <= np.linalg.norm(reference.residual(A64, xx, w.b, w.lam)) / w.lam * 1.01 + \
            1e-12 * np.linalg.norm(xs)
    assert info["outer_iters"] <= 2 * info2["outer_iters"] + 10
    fb.close()
    ff.close()
    sk.close()


def test_bf16_data_iterative_level2(ctx):
    # the paper's sketched level 2 (phi = 2 s, level-2 PCG) on BF16 C and W
    w = make_workload("rbf", seed=12, n=2500)
    A32 = w.A.astype(np.float32)
    A = torch.from_numpy(A32).cuda()
    sk = ctx.sketch(A, 256, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=512, data="bf16")
    x, info = ctx.solve(f, A, torch.from_numpy(w.b).cuda(), w.lam, precision="mixed", tol=1e-10, max_inner=50,
                        inner_tol=1e-4)
    assert reference.rel_residual(A32.astype(np.float64), x.cpu().numpy(), w.b, w.lam) <= 1.2e-10
    assert info["inner_iters"] > 0
    f.close()
    sk.close()


@pytest.mark.parametrize("n,s", [(1000 + 3, 128), (4096, 1024)])
def test_bf16_sketch_pass_matches_oracle(ctx, n, s):
    w = make_workload("rbf", seed=13, n=n)
    Ab = _bf16_values(w.A)
    At = torch.from_numpy(w.A.astype(np.float32)).to(torch.bfloat16).cuda()
    sk = ctx.sketch(At, s, 8, SEED)
    C = sk.C().cpu().numpy().astype(np.float64)
    S = sketch.sparse_embedding(n, s, 8, SEED)
    Co = sketch.sketch_C(Ab, S)
    # |dC_ij| <= (k + 1) u32 sum_k |A_ik| |Pi_kj| (k <= n gamma / s terms per
    # entry on average; bounded here by the row's full sum)
    absC = sketch.sketch_C(np.abs(Ab), abs(S))
    assert np.all(np.abs(C - Co) <= (n + 1) * 2.0 ** -24 * absC + 1e-30)
    sk.close()


def test_bf16_matvec_f64(ctx):
    n = 1537
    w = make_workload("rbf", seed=14, n=n)
    Ab = _bf16_values(w.A)
    At = torch.from_numpy(w.A.astype(np.float32)).to(torch.bfloat16).cuda()
    x = np.random.default_rng(3).standard_normal(n)
    y = ctx.matvec_f64(At, torch.from_numpy(x).cuda(), 0.25).cpu().numpy()
    ref = Ab @ x + 0.25 * x
    assert np.all(np.abs(y - ref) <= 4 * n * 2.0 ** -53 * (np.abs(Ab) @ np.abs(x) + 0.25 * np.abs(x)))
