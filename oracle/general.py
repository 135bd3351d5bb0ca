"""Three-level MSP for (A^T A + lambda I) x = c with A in R^{m x n} of full
column rank: Algorithm 3, with SolveM1 of Algorithm 4 and SolveM2 of
Algorithm 5, in FP64 (oracle side; test infrastructure only).

Algorithm 3, step by step:
  2. lambda~ = lambda + lambda_0
  3. S in R^{s x n}, sparse embedding (Definition 2.1)
  4. A~ = A S^T (m x s);  A^ = Phi A~ (phi x s), Phi a phi x m embedding
  5. M3a = A^^T A^,  M3b = M3a + lambda~ I
  6. their inverses (here: Cholesky factors, applied by triangular solves)
  7. preconditioned Lanczos on (A^T A + lambda I, c, SolveM1)
Algorithm 4, SolveM1(r) -- solves M w = r for M = C W^{-1} C^T + lambda~ I,
with C = A^T A~ and W = A~^T A~ never formed (Section 5):
  2. y^ ~ solution of (A~^T A A^T A~ + lambda~ A~^T A~) y = A~^T A r,
     preconditioned by SolveM2
  3. w^ = (r - A^T A~ y^) / lambda~
Algorithm 5, SolveM2(r) -- solves M2 z = r for M2 = W^2 + lambda~ W through
M2^{-1} = (W^{-1} - (W + lambda~ I)^{-1}) / lambda~ (Section 5):
  2. u^ ~ solution of (A~^T A~) u = r, preconditioned by M3a^{-1}
  3. v^ ~ solution of (A~^T A~ + lambda~ I) v = r, preconditioned by M3b^{-1}
  4. z^ = (u^ - v^) / lambda~

Readings where the paper is silent or garbled:
* The text writes the level-3 preconditioners as "M3a^{-1} := A^^T A^";
  Algorithm 3 step 5 defines M3a = A^^T A^ and the Lanczos calls take
  M3a^{-1}: the preconditioner matrix is A^^T A^ and its inverse is applied.
* Phi (phi x m) is a sparse embedding drawn from the level-2 streams, as in
  the PSD case (Lemma 2.2 names an oblivious embedding without construction).
* The inner iteration counts are fixed: t2 level-2 steps and t3 level-3
  steps (the paper gives O(log(kappa/eps_0)) and O(log(kappa l/eps_0))
  without constants). Every level is (flexible where its preconditioner is
  inexact) PCG, which Section 6 notes is equivalent to Lanczos in exact
  arithmetic. Level 1 stops on |c - (A^T A + lam I) x| <= tol |c|.
* ``level2='exact'`` / ``level3='exact'`` replace a level's iteration by a
  dense solve (isolates the error of each level in the pins).
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import krylov, sketch


@dataclasses.dataclass
class GenParams:
    s: int
    gamma: int = 8
    phi: int | None = None          # default 4 s
    gamma_phi: int = 8
    lam0: float = 0.0
    seed: int = 0x4D5350
    tol: float = 1e-10
    max_outer: int = 500
    t2: int = 12                    # level-2 iterations (Algorithm 4 step 2)
    t3: int = 12                    # level-3 iterations (Algorithm 5 steps 2-3)
    level2: str = "pcg"             # 'pcg' | 'exact'
    level3: str = "pcg"             # 'pcg' | 'exact'


@dataclasses.dataclass
class GenSetup:
    """Everything Algorithm 3 computes before the level-1 iteration."""
    A: np.ndarray
    S: object
    Phi: object
    At: np.ndarray            # A~ = A S^T, m x s
    Ah: np.ndarray            # A^ = Phi A~, phi x s
    lam: float
    lam_tilde: float
    L3a: np.ndarray           # Cholesky factor of M3a = A^^T A^
    L3b: np.ndarray           # Cholesky factor of M3b = M3a + lambda~ I


def setup(A: np.ndarray, lam: float, p: GenParams, S=None, Phi=None) -> GenSetup:
    """Algorithm 3 steps 2-6."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    lam_tilde = lam + p.lam0
    if not lam_tilde > 0.0:
        raise ValueError("lambda + lambda0 must be positive (SolveM1 divides by it)")
    if S is None:
        S = sketch.sparse_embedding(n, p.s, p.gamma, p.seed)
    At = np.asarray((S @ A.T).T)                       # A S^T
    phi = p.phi or 4 * p.s
    if Phi is None:
        Phi = sketch.level2_embedding(m, phi, p.gamma_phi, p.seed)
    Ah = np.asarray(Phi @ At)
    M3a = Ah.T @ Ah
    M3b = M3a + lam_tilde * np.eye(p.s)
    return GenSetup(A, S, Phi, At, Ah, lam, lam_tilde, np.linalg.cholesky(M3a), np.linalg.cholesky(M3b))


def _chol_solve(L: np.ndarray, v: np.ndarray) -> np.ndarray:
    return sla.solve_triangular(L.T, sla.solve_triangular(L, v, lower=True), lower=False)


def solve_m2(st: GenSetup, r: np.ndarray, p: GenParams) -> np.ndarray:
    """Algorithm 5: z^ = (u^ - v^) / lambda~ with u^, v^ from the two level-3 solves."""
    At, lt = st.At, st.lam_tilde
    if p.level3 == "exact":
        W = At.T @ At
        u = np.linalg.solve(W, r)
        v = np.linalg.solve(W + lt * np.eye(W.shape[0]), r)
    else:
        def op_a(y):
            return At.T @ (At @ y)

        def op_b(y):
            return At.T @ (At @ y) + lt * y
        u = krylov.pcg(op_a, r, lambda v_: _chol_solve(st.L3a, v_), 0.0, p.t3).x
        v = krylov.pcg(op_b, r, lambda v_: _chol_solve(st.L3b, v_), 0.0, p.t3).x
    return (u - v) / lt


def level2_matvec(st: GenSetup, y: np.ndarray) -> np.ndarray:
    """(A~^T A A^T A~ + lambda~ A~^T A~) y, from the right: u = A~ y,
    then A~^T (A (A^T u) + lambda~ u)."""
    u = st.At @ y
    return st.At.T @ (st.A @ (st.A.T @ u) + st.lam_tilde * u)


def solve_m1(st: GenSetup, r: np.ndarray, p: GenParams) -> np.ndarray:
    """Algorithm 4: w^ = (r - A^T A~ y^) / lambda~."""
    A, At, lt = st.A, st.At, st.lam_tilde
    g = At.T @ (A @ r)
    if p.level2 == "exact":
        Cm = A.T @ At
        W = At.T @ At
        y = np.linalg.solve(Cm.T @ Cm + lt * W, g)
    else:
        y = krylov.pcg(lambda v: level2_matvec(st, v), g, lambda v: solve_m2(st, v, p), 0.0, p.t2,
                       flexible=True).x
    return (r - A.T @ (At @ y)) / lt


def matvec(A: np.ndarray, lam: float, x: np.ndarray) -> np.ndarray:
    """(A^T A + lam I) x without forming A^T A."""
    return A.T @ (A @ x) + lam * x


def solve(A: np.ndarray, c: np.ndarray, lam: float, p: GenParams,
          st: GenSetup | None = None) -> tuple[np.ndarray, krylov.PcgResult]:
    """Algorithm 3 step 7: flexible PCG on (A^T A + lam I) x = c with SolveM1."""
    A = np.asarray(A, dtype=np.float64)
    if st is None:
        st = setup(A, lam, p)
    res = krylov.pcg(lambda v: matvec(A, lam, v), np.asarray(c, dtype=np.float64),
                     lambda r: solve_m1(st, r, p), p.tol, p.max_outer, flexible=True)
    return res.x, res


def dense_preconditioner(st: GenSetup) -> np.ndarray:
    """M = C W^{-1} C^T + lambda~ I with C = A^T A~, W = A~^T A~ formed densely
    (what SolveM1 applies the inverse of; small sizes only)."""
    Cm = st.A.T @ st.At
    W = st.At.T @ st.At
    return Cm @ np.linalg.solve(W, Cm.T) + st.lam_tilde * np.eye(st.A.shape[1])
