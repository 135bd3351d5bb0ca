"""Least squares by sketch-and-precondition with MSP inner solves (Section 3,
the least-squares corollary), FP64 (oracle side; test infrastructure only).

min_x |A x - b| for a tall A (n x d, n >> d):
  1. A~ = Phi A with Phi an s_ls x n sparse embedding (a constant-factor
     subspace embedding, so A~^T A~ is within constant factors of A^T A);
  2. iterate on the normal equations A^T A x = A^T b with the preconditioner
     g -> (A~^T A~)^{-1} g, each application solved only to constant
     accuracy by Theorem 3.1's solver (Algorithm 3 on A~ with lambda = 0).

Readings where the paper is silent (it points to the sketch-and-precondition
literature for the outer method):
* the outer method is flexible PCG on the normal equations (the inner
  solves are inexact, so the preconditioner varies between calls), stopping
  on |A^T (b - A x)| <= tol |A^T b|;
* an inner solve stops at relative residual inner_tol (constant accuracy);
* Phi is a sparse embedding (Definition 2.1) over the n rows of A with
  gamma_ls nonzeros per column, drawn from streams 4 and 5.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import general, krylov, sketch

STREAM_LS = 4


@dataclasses.dataclass
class LsqParams:
    s_ls: int                        # rows of the sketch A~ = Phi A
    gamma_ls: int = 4
    inner: general.GenParams | None = None   # Theorem 3.1 on A~ (lambda = 0)
    inner_tol: float = 1e-2
    inner_maxit: int = 50
    tol: float = 1e-10
    max_outer: int = 200
    seed: int = 0x4D5350
    exact_inner: bool = False        # apply (A~^T A~)^{-1} by a dense solve


def sketch_rows(A: np.ndarray, p: LsqParams) -> np.ndarray:
    """A~ = Phi A (step 1)."""
    n = A.shape[0]
    idx, sgn = sketch.embedding_pattern(n, p.s_ls, p.gamma_ls, p.seed, STREAM_LS)
    Phi = sketch.embedding_matrix(idx, sgn, p.s_ls)
    return np.asarray(Phi @ A)


def solve(A: np.ndarray, b: np.ndarray, p: LsqParams) -> tuple[np.ndarray, krylov.PcgResult, np.ndarray]:
    """Returns (x, outer PCG result, A~)."""
    A = np.asarray(A, dtype=np.float64)
    At = sketch_rows(A, p)
    c = A.T @ b
    if p.exact_inner:
        G = At.T @ At

        def prec(g):
            return np.linalg.solve(G, g)
    else:
        ip = p.inner
        st = general.setup(At, 0.0, ip)
        ip_loose = dataclasses.replace(ip, tol=p.inner_tol, max_outer=p.inner_maxit)

        def prec(g):
            x, _ = general.solve(At, g, 0.0, ip_loose, st)
            return x
    res = krylov.pcg(lambda v: A.T @ (A @ v), c, prec, p.tol, p.max_outer, flexible=True)
    return res.x, res, At
