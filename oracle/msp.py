"""Two-level MSP for (A + lambda I) x = b, A PSD: Algorithm 1 with SolveM1 of
Algorithm 2, in FP64 (oracle side).

Algorithm 1, step by step:
  2. S in R^{s x n}, sparse embedding with gamma nonzeros per column (Def 2.1)
  3. lambda~ = lambda + lambda_0;  C = A S^T;  W = S C
  4. C~ = Phi C;  M2^{-1} = (C~^T C~ + lambda~ W)^{-1}
  5. preconditioned Lanczos on (A + lambda I, b, SolveM1)
Algorithm 2, SolveM1(r):
  2. y^ ~ (C^T C + lambda~ W)^{-1} C^T r by preconditioned Lanczos with M2^{-1};
     the matvec is C^T (C y) + lambda~ (W y), never forming C^T C
  3. w^ = (r - C y^) / lambda~

Readings where the paper is silent (real RAM, Section 2): the outer method is
selectable among Algorithm 6, PCG and flexible PCG (equal in exact arithmetic,
Section 6); the inner solve stops at |res| <= inner_tol * |C^T r| or after
max_inner iterations (the paper gives O(log kappa / eps_0) without constants);
the outer solve stops on the relative residual |b - (A + lam I) x| / |b| <= tol.
``inner='exact'`` replaces the level-2 solve by a dense solve (isolates the
inner-solve error).

``refine`` wraps any solver in FP64 iterative refinement: r = b - (A + lam I) x,
solve for the correction, x += d.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import krylov, nystrom, sketch


@dataclasses.dataclass
class MspParams:
    s: int
    gamma: int = 8
    phi: int | None = None          # default 2 s
    gamma_phi: int = 8
    lam0: float = 0.0
    seed: int = 0x4D5350
    tol: float = 1e-10
    max_outer: int = 2000
    inner_tol: float = 1e-10
    max_inner: int = 50
    outer: str = "fcg"              # 'fcg' | 'pcg' | 'lanczos'
    inner: str = "pcg"              # 'pcg' | 'lanczos' | 'exact'


@dataclasses.dataclass
class MspSetup:
    """Everything Algorithm 1 computes before the outer iteration."""
    S: object
    Phi: object
    C: np.ndarray
    W: np.ndarray
    Ct: np.ndarray
    lam: float
    lam_tilde: float
    M2: np.ndarray
    factor: nystrom.Factor


@dataclasses.dataclass
class MspInfo:
    outer_iters: int = 0
    inner_iters: list = dataclasses.field(default_factory=list)
    rel_residuals: list = dataclasses.field(default_factory=list)
    converged: bool = False


def setup(A: np.ndarray, lam: float, p: MspParams, S=None, Phi=None) -> MspSetup:
    """Algorithm 1 steps 2-4. ``S`` / ``Phi`` override the drawn embeddings (used by
    special-case tests, e.g. a signed permutation for which A^ = A)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    phi = p.phi or 2 * p.s
    if S is None:
        S = sketch.sparse_embedding(n, p.s, p.gamma, p.seed)
    lam_tilde = lam + p.lam0
    C = sketch.sketch_C(A, S)
    W = sketch.core_W(S, C)
    if Phi is None:
        Phi = sketch.level2_embedding(n, phi, p.gamma_phi, p.seed)
    Ct = sketch.level2_sketch(Phi, C)
    M2 = nystrom.level2_matrix(Ct, W, lam_tilde)
    return MspSetup(S, Phi, C, W, Ct, lam, lam_tilde, M2, nystrom.cholesky_with_shift(M2))


def solve_m1(st: MspSetup, r: np.ndarray, p: MspParams, info: MspInfo | None = None) -> np.ndarray:
    """Algorithm 2: w^ = (r - C y^) / lambda~ with y^ from the level-2 solve."""
    C, W, lt = st.C, st.W, st.lam_tilde
    g = C.T @ r
    if p.inner == "exact":
        y = np.linalg.solve(C.T @ C + lt * W, g)
        its = 0
    else:
        def level2_matvec(v):
            return C.T @ (C @ v) + lt * (W @ v)
        if p.inner == "lanczos":
            res = krylov.lanczos_left(level2_matvec, g, st.factor.solve, p.max_inner)
            y, its = res.x, res.iters
        else:
            res = krylov.pcg(level2_matvec, g, st.factor.solve, p.inner_tol, p.max_inner)
            y, its = res.x, res.iters
    if info is not None:
        info.inner_iters.append(its)
    return (r - C @ y) / lt


def solve(A: np.ndarray, b: np.ndarray, lam: float, p: MspParams,
          st: MspSetup | None = None) -> tuple[np.ndarray, MspInfo]:
    """Algorithm 1 (steps 2-5) returning x~ and iteration statistics."""
    A = np.asarray(A, dtype=np.float64)
    if st is None:
        st = setup(A, lam, p)
    info = MspInfo()

    def outer_matvec(v):
        return A @ v + lam * v

    def solve_m(r):
        return solve_m1(st, r, p, info)

    if p.outer == "lanczos":
        res = krylov.lanczos_left(outer_matvec, b, solve_m, p.max_outer)
        x = res.x
        info.outer_iters = res.iters
        rr = np.linalg.norm(b - outer_matvec(x)) / np.linalg.norm(b)
        info.rel_residuals = [rr]
        info.converged = rr <= p.tol
        return x, info
    res = krylov.pcg(outer_matvec, b, solve_m, p.tol, p.max_outer,
                     flexible=(p.outer == "fcg"))
    info.outer_iters = res.iters
    info.rel_residuals = res.rel_residuals
    info.converged = res.converged
    return res.x, info


def refine(A: np.ndarray, b: np.ndarray, lam: float, correction, tol: float,
           max_refine: int = 20) -> tuple[np.ndarray, list]:
    """FP64 iterative refinement: x_0 = 0; r = b - (A + lam I) x; x += correction(r)
    until |r| / |b| <= tol. Returns x and the history of |r| / |b|."""
    A = np.asarray(A, dtype=np.float64)
    x = np.zeros_like(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    hist = []
    for _ in range(max_refine + 1):
        r = b - (A @ x + lam * x)
        hist.append(float(np.linalg.norm(r) / nb))
        if hist[-1] <= tol:
            break
        x = x + correction(r)
    return x, hist
