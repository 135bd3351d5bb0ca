"""Least squares by sketch-and-precondition with three-level inner solves
(msp_lsq_create / msp_lsq_solve) against the definition (numpy lstsq in FP64
on the same FP32 matrix) and the FP64 oracle.

Inputs: A = U diag(sigma) V^T (n x d, 6 outliers 1e2 -> 1e1 over a flat tail
in [0.5, 1]) rounded once to FP32; b ~ N(0, I); A~ = Phi A with s_ls = 4 d
rows, gamma_ls = 4; inner solver on A~ with s = d/2, phi = 4 s and
lambda0 = (2/l) sum_{i>l} sigma_i^2, l = 2 k.

Tolerances: the solve stops at |A^T (b - A x)| <= 1e-10 |A^T b| (recomputed
here in FP64); then |x - x*| <= |A^T (b - A x)| / sigma_min^2 (A^T A
positive definite), and the reported |A x - b| matches the host's to 1e-12.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import general, lsq
from workloads import householder_spectrum, svd_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _problem(n, d, k, seed):
    sig = householder_spectrum(d, k, seed, hi=1e2, lo=1e1)
    A32 = svd_matrix(n, d, sig, seed + 1).astype(np.float32)
    lam0 = 2.0 / (2 * k) * float(np.sum(sig[2 * k:] ** 2))
    return A32, sig, lam0


CASES = [(2000, 96, 6, 3), (1501, 83, 5, 8)]   # aligned; odd d (padded copy)


@pytest.mark.parametrize("n,d,k,seed", CASES)
@pytest.mark.parametrize("t2,t3", [(8, 8), (0, 0)])
def test_lsq_matches_lstsq(ctx, n, d, k, seed, t2, t3):
    A32, sig, lam0 = _problem(n, d, k, seed)
    A64 = A32.astype(np.float64)
    s = max(16, d // 2)
    h = ctx.lsq(torch.from_numpy(A32).cuda(), 4 * d, lam0, s)
    b = np.random.default_rng(seed + 10).standard_normal(n)
    x, info = h.solve(torch.from_numpy(b).cuda(), tol=1e-10, level2_iters=t2, level3_iters=t3)
    h.close()
    x = x.cpu().numpy()
    g = A64.T @ (b - A64 @ x)
    c = A64.T @ b
    assert info["status"] == 0
    assert np.linalg.norm(g) <= 1e-10 * np.linalg.norm(c) * 1.0001
    xs = np.linalg.lstsq(A64, b, rcond=None)[0]
    smin = np.linalg.svd(A64, compute_uv=False)[-1]
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(g) / smin ** 2 + 1e-12 * np.linalg.norm(xs)
    r = np.linalg.norm(A64 @ x - b)
    assert abs(info["resid_norm"] - r) <= 1e-12 * np.linalg.norm(b)
    # the corollary's form: |A x - b|^2 <= min + eps |b|^2
    assert r ** 2 <= np.linalg.norm(A64 @ xs - b) ** 2 + 1e-12 * np.linalg.norm(b) ** 2


def test_lsq_outer_iterations_match_oracle_scale(ctx):
    """With the same sketch the device's outer iteration count is close to
    the oracle's (both flexible PCG with inner solves to 1e-2)."""
    n, d, k, seed = CASES[0]
    A32, sig, lam0 = _problem(n, d, k, seed)
    s = d // 2
    h = ctx.lsq(torch.from_numpy(A32).cuda(), 4 * d, lam0, s)
    b = np.random.default_rng(seed + 10).standard_normal(n)
    _, info = h.solve(torch.from_numpy(b).cuda(), tol=1e-10, precision="fp32", raise_on_noconv=False,
                      level2_iters=0, level3_iters=0)
    h.close()
    ip = general.GenParams(s=s, lam0=lam0, level2="exact")
    p = lsq.LsqParams(s_ls=4 * d, inner=ip, inner_tol=1e-2, tol=1e-6)
    _, res, _ = lsq.solve(A32.astype(np.float64), b, p)
    # the FP32 device run to 1e-6 of its own residual takes about as many steps
    assert info["outer_iters"] <= 3 * res.iters + 5


def test_lsq_consistent_system(ctx):
    n, d, k, seed = CASES[0]
    A32, sig, lam0 = _problem(n, d, k, seed)
    A64 = A32.astype(np.float64)
    xt = np.random.default_rng(21).standard_normal(d)
    b = A64 @ xt
    h = ctx.lsq(torch.from_numpy(A32).cuda(), 4 * d, lam0, d // 2)
    x, info = h.solve(torch.from_numpy(b).cuda(), tol=1e-11, level2_iters=0, level3_iters=0)
    h.close()
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xt) <= 1e-8 * np.linalg.norm(xt)
    assert info["resid_norm"] <= 1e-8 * np.linalg.norm(b)


def test_lsq_bad_arguments(ctx):
    from paper_2405_05865_gb300 import MspError
    A = torch.randn((300, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(MspError):
        ctx.lsq(A, 30, 1.0, 16)          # s_ls < d
    with pytest.raises(MspError):
        ctx.lsq(A, 160, 0.0, 16)         # lambda0 = 0
    h = ctx.lsq(A, 160, 1.0, 16)
    with pytest.raises(MspError):
        h.solve(torch.ones(300, dtype=torch.float64, device="cuda"), inner_tol=0.0)
    h.close()
