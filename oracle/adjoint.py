"""Gradients of a loss through x = (K_theta + lam I)^{-1} b (oracle side, FP64).

For L = g^T x the adjoint of the solve is a second solve with the same
symmetric operator: a = (K + lam I)^{-1} g, and
    dL/db   = a,
    dL/dlam = -a^T x,
    dL/dK   = -a x^T,  so  dL/dtheta = -a^T (dK/dtheta) x.
For the RBF kernel K_ij = exp(-d_ij^2 / (2 ell^2)),
    dK_ij/dell = K_ij d_ij^2 / ell^3.
The forward uses lam as the full diagonal shift (K + lam I) x = b, the
reading of the kernel-ridge-regression system of Section 3 used throughout.
"""

from __future__ import annotations

import numpy as np

from . import reference


def rbf_sqdist(P: np.ndarray) -> np.ndarray:
    d = P[:, None, :] - P[None, :, :]
    return np.einsum("ijk,ijk->ij", d, d)


def rbf(P: np.ndarray, ell: float) -> np.ndarray:
    return np.exp(-rbf_sqdist(P) / (2.0 * ell * ell))


def rbf_dK_dell(P: np.ndarray, ell: float) -> np.ndarray:
    D2 = rbf_sqdist(P)
    return np.exp(-D2 / (2.0 * ell * ell)) * D2 / ell ** 3


def grads(K: np.ndarray, b: np.ndarray, lam: float, g: np.ndarray,
          dK_dtheta: np.ndarray | None = None) -> dict:
    """Analytic gradients of L = g^T x by two dense Cholesky solves."""
    x = reference.solve_dense(K, b, lam)
    a = reference.solve_dense(K, g, lam)
    out = {"x": x, "a": a, "db": a, "dlam": -float(a @ x)}
    if dK_dtheta is not None:
        out["dtheta"] = -float(a @ (dK_dtheta @ x))
    return out


def loss(P: np.ndarray, ell: float, lam: float, b: np.ndarray, g: np.ndarray) -> float:
    return float(g @ reference.solve_dense(rbf(P, ell), b, lam))
