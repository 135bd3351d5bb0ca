"""Batches of independent MSP solves (oracle side, FP64).

A batch is a list of instances (A_k, lam_k, B_k), B_k holding m_k right-hand
sides. Nothing in Algorithm 1 couples two right-hand sides or two instances:
every column is its own run of the method (Algorithm 1 step 5) with the
sketch, W and level-2 factor of its instance (steps 2-4, computed once per
instance). This module writes that definition out as a loop.

Reading used by the batched CUDA path: the level 2 is applied directly,
y = (C^T C + lambda~ W)^{-1} C^T r (``inner='exact'``; the sketch-and-solve
level-2 system solved exactly, Phi = I), the level-1 method is flexible PCG
and each column is wrapped in FP64 iterative refinement (``refine``).
"""

from __future__ import annotations

import numpy as np

from . import msp


def solve_instance(A: np.ndarray, B: np.ndarray, lam: float, p: msp.MspParams,
                   refine_tol: float | None = None, max_refine: int = 20) -> np.ndarray:
    """X with X[:, j] the MSP solution of (A + lam I) x = B[:, j]; one set-up.
    With ``refine_tol`` each column is refined: correction solves to refine_tol
    until |b - (A + lam I) x| / |b| <= p.tol."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    st = msp.setup(A, lam, p)
    X = np.zeros_like(B)
    for j in range(B.shape[1]):
        b = B[:, j]
        if not np.any(b):
            continue
        if refine_tol is None:
            X[:, j], _ = msp.solve(A, b, lam, p, st)
        else:
            import dataclasses
            q = dataclasses.replace(p, tol=refine_tol)

            def correction(r):
                d, _ = msp.solve(A, r, lam, q, st)
                return d
            X[:, j], _ = msp.refine(A, b, lam, correction, p.tol, max_refine)
    return X


def solve_batch(instances: list[tuple[np.ndarray, np.ndarray, float, msp.MspParams]],
                refine_tol: float | None = None) -> list[np.ndarray]:
    """solve_instance over a list of (A, B, lam, params)."""
    return [solve_instance(A, B, lam, p, refine_tol) for A, B, lam, p in instances]
