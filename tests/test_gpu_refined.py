"""The mixed-precision workload: A = Q diag(sigma) Q^T with Q a product of 64
Householder reflectors, 1024 outliers 1e6 -> 1e2 over a flat tail
0.5 + 0.5u (n = 32768, lambda = 1e-4, s = 2048 at full size; the same ratios
at reduced n here). The problem is the FP64 matrix: the level-1 iteration of
Algorithm 1 applies its FP32 rounding, and every FP64 refinement step forms
the residual with the FP64 matrix (msp_solve_refined), to a normwise backward
error of 1e-10 checked on the host in FP64.

x is also checked against the dense Cholesky solution through the exact
bound |x - x*| <= |r| / lambda_min(A + lambda I), lambda_min known from the
generated spectrum."""

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
    c.close()


@pytest.mark.parametrize("n", [2048, 4096 + 129])
def test_refined_solve_householder_workload(ctx, n):
    w = make_workload("householder", seed=0, n=n)
    A64 = np.asarray(w.A, dtype=np.float64)
    lam0 = onys.lambda0_from_spectrum(w.sigma, w.s // 2)     # l = number of outliers
    A32_dev = torch.from_numpy(A64.astype(np.float32)).cuda()
    A64_dev = torch.from_numpy(A64).cuda()
    b = torch.from_numpy(w.b).cuda()
    sk = ctx.sketch(A32_dev, w.s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, lam0, phi=0)
    x, info = ctx.solve_refined(f, A32_dev, A64_dev, b, w.lam, precision="mixed", tol=1e-10,
                                criterion="backward", max_inner=0)
    x = x.cpu().numpy()
    r = reference.residual(A64, x, w.b, w.lam)
    norm_A = float(w.sigma.max())
    eta = np.linalg.norm(r) / ((norm_A + w.lam) * np.linalg.norm(x) + np.linalg.norm(w.b))
    assert eta <= 1e-10
    assert info["backward_err"] <= 1e-10 and info["refine_steps"] >= 2
    # |x - x*| <= |r| / lambda_min(A + lam I) exactly; x* itself carries the
    # rounding of a backward-stable Cholesky solve, kappa u |x*|
    xs = reference.solve_dense(A64, w.b, w.lam)
    lmin = float(w.sigma.min()) + w.lam
    kappa = (norm_A + w.lam) / lmin
    err = np.linalg.norm(x - xs)
    assert err <= np.linalg.norm(r) / lmin + 8 * kappa * 2.0 ** -53 * np.linalg.norm(xs)
    sk.close()
    f.close()


def test_refined_solve_reaches_relative_residual(ctx):
    # the stricter rule |r| <= 1e-10 |b| against the FP64 matrix
    w = make_workload("householder", seed=1, n=2048)
    A64 = np.asarray(w.A, dtype=np.float64)
    lam0 = onys.lambda0_from_spectrum(w.sigma, w.s // 2)
    A32_dev = torch.from_numpy(A64.astype(np.float32)).cuda()
    A64_dev = torch.from_numpy(A64).cuda()
    sk = ctx.sketch(A32_dev, w.s, 8, SEED)
    f = ctx.nystrom(sk, w.lam, lam0, phi=0)
    x, info = ctx.solve_refined(f, A32_dev, A64_dev, torch.from_numpy(w.b).cuda(), w.lam,
                                precision="mixed", tol=1e-10, max_inner=0)
    assert reference.rel_residual(A64, x.cpu().numpy(), w.b, w.lam) <= 1.2e-10
    assert info["rel_resid"] <= 1e-10
    sk.close()
    f.close()


def test_refined_with_the_same_matrix_is_msp_solve(ctx):
    # A_res = A: the same arithmetic as msp_solve, bit for bit
    w = make_workload("rbf", seed=4, n=1500)
    A = torch.from_numpy(w.A.astype(np.float32)).cuda()
    b = torch.from_numpy(w.b).cuda()
    sk = ctx.sketch(A, 128, 8, SEED)
    f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
    x1, i1 = ctx.solve(f, A, b, w.lam, precision="mixed", tol=1e-10, max_inner=0)
    x2, i2 = ctx.solve_refined(f, A, A, b, w.lam, precision="mixed", tol=1e-10, max_inner=0)
    assert torch.equal(x1, x2)
    assert i1["outer_iters"] == i2["outer_iters"]
    sk.close()
    f.close()
