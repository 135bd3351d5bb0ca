"""Krylov solvers used at every level of MSP (oracle side, FP64).

* ``lanczos_left``: preconditioned Lanczos, Algorithm 6 (Section 6.1), written
  with the paper's two vector families: under-barred q (Krylov basis in the
  A-space) and over-barred q (its image under SolveM). Reading of a garble:
  the first over-barred vector is SolveM(b) / z' (the listing's "w'/z").
* ``lanczos_sym``: symmetric preconditioned Lanczos, Algorithm 7, which needs
  M^{-1/2}; analysis device only, used here on tiny n as a pin.
* ``pcg``: preconditioned conjugate gradient, which Section 6 notes gives the
  same output as Lanczos in exact arithmetic; ``flexible=True`` uses the
  Polak-Ribiere beta = r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k), safe when the
  preconditioner is applied inexactly and so varies between calls.
"""

from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np

Vec = np.ndarray
Op = Callable[[Vec], Vec]


@dataclasses.dataclass
class LanczosResult:
    x: Vec
    alpha: np.ndarray
    beta: np.ndarray      # beta'_2 .. beta'_{t+1}
    iters: int


def lanczos_left(matvec: Op, b: Vec, solve_m: Op, t: int) -> LanczosResult:
    """Algorithm 6: x_t = z' Qbar T'^{-1} e_1 after t iterations (or fewer on a
    zero beta')."""
    w0 = solve_m(b)
    z = np.sqrt(float(b @ w0))
    q_lo_prev = np.zeros_like(b)
    q_hi = w0 / z                # over-barred q_1
    q_lo = b / z                 # under-barred q_1
    beta = 0.0
    alphas, betas, Qhi = [], [], []
    for _ in range(t):
        Qhi.append(q_hi)
        u = matvec(q_hi) - beta * q_lo_prev
        alpha = float(u @ q_hi)
        w_lo = u - alpha * q_lo
        w_hi = solve_m(w_lo)
        alphas.append(alpha)
        bsq = float(w_lo @ w_hi)
        beta = np.sqrt(bsq) if bsq > 0 else 0.0
        betas.append(beta)
        if beta == 0.0:
            break
        q_lo_prev = q_lo
        q_lo = w_lo / beta
        q_hi = w_hi / beta
    k = len(alphas)
    T = np.diag(alphas)
    for i in range(k - 1):
        T[i, i + 1] = T[i + 1, i] = betas[i]
    e1 = np.zeros(k)
    e1[0] = 1.0
    x = z * (np.stack(Qhi, axis=1) @ np.linalg.solve(T, e1))
    return LanczosResult(x, np.array(alphas), np.array(betas), k)


def lanczos_sym(matvec: Op, b: Vec, M: np.ndarray, t: int) -> LanczosResult:
    """Algorithm 7 with an explicit SPD preconditioner M (dense; tiny n only)."""
    ev, V = np.linalg.eigh(M)
    Mmh = (V / np.sqrt(ev)) @ V.T          # M^{-1/2}
    w0 = Mmh @ b
    z = np.linalg.norm(w0)
    q_prev = np.zeros_like(b)
    q = w0 / z
    beta = 0.0
    alphas, betas, Q = [], [], []
    for _ in range(t):
        Q.append(q)
        u = Mmh @ matvec(Mmh @ q) - beta * q_prev
        alpha = float(u @ q)
        w = u - alpha * q
        alphas.append(alpha)
        beta = float(np.linalg.norm(w))
        betas.append(beta)
        if beta == 0.0:
            break
        q_prev, q = q, w / beta
    k = len(alphas)
    T = np.diag(alphas)
    for i in range(k - 1):
        T[i, i + 1] = T[i + 1, i] = betas[i]
    e1 = np.zeros(k)
    e1[0] = 1.0
    y = z * (np.stack(Q, axis=1) @ np.linalg.solve(T, e1))
    return LanczosResult(Mmh @ y, np.array(alphas), np.array(betas), k)


@dataclasses.dataclass
class PcgResult:
    x: Vec
    iters: int
    rel_residuals: list        # |r_k| / |b| of the recurrence residual, k = 0..iters
    converged: bool
    alphas: list = dataclasses.field(default_factory=list)
    betas: list = dataclasses.field(default_factory=list)


def pcg(matvec: Op, b: Vec, solve_m: Op, tol: float, maxit: int,
        flexible: bool = False, x0: Vec | None = None,
        stop_norm: Callable[[Vec], float] | None = None) -> PcgResult:
    """(Flexible) PCG from x0 (default 0); stops when stop_norm(r) <= tol * stop_norm(b)
    (default Euclidean norm) or after maxit iterations."""
    norm = stop_norm or (lambda v: float(np.linalg.norm(v)))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - matvec(x) if x0 is not None else b.copy()
    nb = norm(b)
    hist = [norm(r) / nb if nb > 0 else 0.0]
    if nb == 0.0:
        return PcgResult(x, 0, hist, True)
    z = solve_m(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for k in range(1, maxit + 1):
        q = matvec(p)
        pq = float(p @ q)
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        alphas.append(alpha)
        hist.append(norm(r) / nb)
        if hist[-1] <= tol:
            return PcgResult(x, k, hist, True, alphas, betas)
        z_new = solve_m(r)
        rz_new = float(r @ z_new)
        beta = (rz_new - float(r @ z)) / rz if flexible else rz_new / rz
        betas.append(beta)
        p = z_new + beta * p
        z, rz = z_new, rz_new
    return PcgResult(x, maxit, hist, False, alphas, betas)
