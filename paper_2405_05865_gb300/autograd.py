"""torch.autograd.Function for x = (K_ell + lam I)^{-1} b with the RBF kernel.

forward: K on the device (msp_rbf_kernel), sketch, Nystrom factor and the
         refined MSP solve (Algorithm 1 + FP64 refinement).
backward: the adjoint of the solve is a second MSP solve with the same
         symmetric operator, reusing the cached sketch and factor:
         a = (K + lam I)^{-1} g,  dL/db = a,  dL/dlam = -a^T x,
         dL/dell = -a^T (dK/dell) x from the fused pair kernel (dK is never
         formed). No gradient flows to the points.
"""

from __future__ import annotations

import torch

from .api import Context, DEFAULT_SEED


class RbfSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, points: torch.Tensor, ell: torch.Tensor, lam: torch.Tensor, b: torch.Tensor,
                ctx: Context, s: int, phi: int, opts: dict):
        ell_v, lam_v = float(ell), float(lam)
        K = ctx.rbf_kernel(points, ell_v)
        sk = ctx.sketch(K, s, 8, DEFAULT_SEED)
        f = ctx.nystrom(sk, lam_v, 0.0, phi=phi)
        x, info = ctx.solve(f, K, b.contiguous(), lam_v, **opts)
        fctx.state = (ctx, K, sk, f, points, ell_v, lam_v, opts)
        fctx.save_for_backward(x)
        fctx.info = info
        return x

    @staticmethod
    def backward(fctx, gx: torch.Tensor):
        (x,) = fctx.saved_tensors
        ctx, K, sk, f, points, ell_v, lam_v, opts = fctx.state
        a, _ = ctx.solve(f, K, gx.contiguous().to(torch.float64), lam_v, **opts)
        g_lam = ctx.dot(a, x, -1.0)
        g_ell = ctx.rbf_grad_ell(points, ell_v, a, x)
        fctx.state = None
        return None, g_ell, g_lam, a, None, None, None, None


def rbf_solve(points: torch.Tensor, ell: torch.Tensor, lam: torch.Tensor, b: torch.Tensor,
              ctx: Context, s: int, phi: int = 0, **opts) -> torch.Tensor:
    """x = (K_ell + lam I)^{-1} b, differentiable in ell, lam and b.
    ell and lam are 0-d float64 tensors; points (n, dim) and b (n,) are CUDA
    float64 tensors."""
    if "max_inner" not in opts and phi == 0:
        opts["max_inner"] = 0
    return RbfSolve.apply(points, ell, lam, b, ctx, s, phi, opts)
