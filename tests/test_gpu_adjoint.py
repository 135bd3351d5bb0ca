"""Adjoint of the solve: x = (K_ell + lam I)^{-1} b with the RBF
kernel; the backward pass is a second MSP solve reusing the factor, plus the
fused dL/dell pair kernel. Checked against the oracle's FP64 dense-Cholesky
gradients and central finite differences of the FP64 dense solve."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint, reference
from workloads import rbf_points, rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,ell", [(300, 0.2), (2048 + 33, 0.1)])
def test_rbf_kernel_matches_host(ctx, n, ell):
    P = rbf_points(n, seed=3)
    K = ctx.rbf_kernel(torch.from_numpy(P).cuda(), ell).cpu().numpy().astype(np.float64)
    Kh = adjoint.rbf(P, ell)
    # FP32 arithmetic on exact (hi, lo) coordinate pairs: d^2 to ~1e-7 relative,
    # |dK| <= K |d arg| + expf error, |d arg| = |d(d^2)| / (2 ell^2)
    D2 = adjoint.rbf_sqdist(P)
    assert np.all(np.abs(K - Kh) <= (4e-7 * (1.0 + D2 / (2 * ell * ell))) * Kh + 1e-30)
    assert np.all(np.diag(K) == 1.0)


@pytest.mark.parametrize("loss", ["bx", "cx"])
def test_autograd_gradients(ctx, loss):
    from paper_2405_05865_gb300.autograd import rbf_solve
    n, ell0, lam0 = 2048, 0.1, 1e-2
    P = rbf_points(n, seed=11)
    b = rhs(n, seed=11)
    c = np.random.default_rng(5).standard_normal(n)
    g = b if loss == "bx" else c
    Pd = torch.from_numpy(P).cuda()
    ell = torch.tensor(ell0, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(lam0, dtype=torch.float64, requires_grad=True)
    bd = torch.from_numpy(b).cuda().requires_grad_(True)
    x = rbf_solve(Pd, ell, lam, bd, ctx, s=128, tol=1e-11)
    L = (x * torch.from_numpy(g).cuda()).sum()
    L.backward()
    # oracle: the FP32 K the GPU built (the system it solved) in FP64 dense
    # Cholesky; dK/dell of the FP64 host kernel
    K = ctx.rbf_kernel(Pd, ell0).cpu().numpy().astype(np.float64)
    dK = adjoint.rbf_dK_dell(P, ell0)
    gr = adjoint.grads(K, b, lam0, g, dK)
    assert np.linalg.norm(x.detach().cpu().numpy() - gr["x"]) <= 1e-8 * np.linalg.norm(gr["x"])
    assert np.linalg.norm(bd.grad.cpu().numpy() - gr["db"]) <= 1e-8 * np.linalg.norm(gr["db"])
    assert float(lam.grad) == pytest.approx(gr["dlam"], rel=1e-7)
    # dL/dell sums n^2 mixed-sign pair terms, each formed in FP32 (relative
    # error ~1e-6 through exp of the FP32 argument): bound the difference by
    # the summation error u32-scale times sum |a_i| |dK_ij| |x_j|
    a_abs = np.abs(gr["a"])
    bound = 64 * 2.0 ** -24 * float(a_abs @ (np.abs(dK) @ np.abs(gr["x"])))
    assert abs(float(ell.grad) - gr["dtheta"]) <= bound
    # central differences of the FP64 host function (h = 1e-4 relative)
    h = 1e-4 * ell0
    fd = (adjoint.loss(P, ell0 + h, lam0, b, g) - adjoint.loss(P, ell0 - h, lam0, b, g)) / (2 * h)
    assert float(ell.grad) == pytest.approx(fd, rel=1e-4)
    if loss == "bx":
        # g = b (a constant here): the adjoint solve equals the forward solve, a = x
        assert np.allclose(bd.grad.cpu().numpy(), gr["x"], rtol=1e-7, atol=1e-9 * np.abs(gr["x"]).max())
