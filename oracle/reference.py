"""Definition oracles: what MSP approximates, written out directly (FP64).

* x* = (A + lam I)^{-1} b by dense Cholesky (Theorem 3.2 / Theorem 4.2 define the
  target of the solve).
* Backward error (normwise, Rigal-Gaches): eta = |b - (A+lam I) x| /
  (|A + lam I|_2 |x| + |b|); the paper states its guarantee in the energy norm
  and, informally (Theorem 1.2), as |(A + lam I) x - b| <= eps |b|.
* Effective dimension d_lam = tr(A (A + lam I)^{-1}) = sum_i s_i / (s_i + lam)
  (Section 2), and the Schatten-p norm (sum_i s_i^p)^{1/p} (Section 3.2).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def solve_dense(A: np.ndarray, b: np.ndarray, lam: float) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    c = sla.cho_factor(A + lam * np.eye(n), lower=True)
    return sla.cho_solve(c, b)


def residual(A: np.ndarray, x: np.ndarray, b: np.ndarray, lam: float) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    return b - (A @ x + lam * x)


def rel_residual(A, x, b, lam) -> float:
    return float(np.linalg.norm(residual(A, x, b, lam)) / np.linalg.norm(b))


def rel_residual_extended(A, x, b, lam) -> float:
    """|b - (A + lam I) x| / |b| with the products and sums in numpy's
    extended type (80-bit on x86, IEEE quad on AArch64): resolves residuals
    of ill-conditioned systems below the FP64 evaluation floor
    u sum_j |A_ij x_j|."""
    Al = np.asarray(A, dtype=np.float64).astype(np.longdouble)
    xl = np.asarray(x, dtype=np.float64).astype(np.longdouble)
    bl = np.asarray(b, dtype=np.float64).astype(np.longdouble)
    r = bl - (Al @ xl + np.longdouble(lam) * xl)
    return float(np.sqrt(np.sum(r * r)) / np.sqrt(np.sum(bl * bl)))


def norm2_power(A: np.ndarray, iters: int = 30, seed: int = 1) -> float:
    """|A|_2 for symmetric PSD A by power iteration (lower bound that converges
    from below; 30 steps)."""
    A = np.asarray(A, dtype=np.float64)
    v = np.random.default_rng(seed).standard_normal(A.shape[0])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = A @ v
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


def backward_error(A, x, b, lam, norm_A: float | None = None) -> float:
    if norm_A is None:
        norm_A = norm2_power(A)
    r = residual(A, x, b, lam)
    return float(np.linalg.norm(r) / ((norm_A + lam) * np.linalg.norm(x) + np.linalg.norm(b)))


def norm_lower_bound(A) -> float:
    """A certified lower bound L <= |A|_2 for symmetric PSD A: the larger of the
    largest column 2-norm (|A e_i| <= |A|_2) and the Rayleigh quotient of the
    all-ones vector (1^T A 1 / n <= lambda_max(A) = |A|_2)."""
    A = np.asarray(A, dtype=np.float64)
    col = float(np.sqrt((A * A).sum(axis=0)).max())
    return max(col, float(A.sum()) / A.shape[0])


def backward_error_bound(A, x, b, lam) -> float:
    """|r| / ((L + lam) |x| + |b|) with L = norm_lower_bound(A). Since
    L + lam <= |A + lam I|_2, this is an upper bound on the normwise backward
    error |r| / (|A + lam I|_2 |x| + |b|) (Rigal and Gaches) of x."""
    r = residual(A, x, b, lam)
    L = norm_lower_bound(A)
    return float(np.linalg.norm(r) / ((L + lam) * np.linalg.norm(x) + np.linalg.norm(b)))


def energy_error(A, x, xs, lam) -> float:
    """|x - x*|_{A + lam I} / |x*|_{A + lam I}."""
    A = np.asarray(A, dtype=np.float64)
    e = x - xs
    num = float(e @ (A @ e) + lam * (e @ e))
    den = float(xs @ (A @ xs) + lam * (xs @ xs))
    return float(np.sqrt(max(num, 0.0) / den))


def effective_dimension(eigs: np.ndarray, lam: float) -> float:
    e = np.asarray(eigs, dtype=np.float64)
    return float(np.sum(e / (e + lam)))


def schatten(eigs: np.ndarray, p: float) -> float:
    """(sum_i |s_i|^p)^{1/p}."""
    e = np.abs(np.asarray(eigs, dtype=np.float64))
    return float(np.sum(e ** p) ** (1.0 / p))
