"""Nystrom preconditioner pieces of Algorithm 1 (oracle side, FP64).

* lambda~ = lambda + lambda_0 (Algorithm 1 step 3; Lemma 4.3 sets
  lambda_0 = (2/l) sum_{i>l} lambda_i).
* M2 = C~^T C~ + lambda~ W, inverted exactly once (Algorithm 1 step 4; Part 3 of
  the proof of Theorem 4.2).
* M^{-1} = (1/lambda~)(I - C (C^T C + lambda~ W)^{-1} C^T) for
  M = C W^{-1} C^T + lambda~ I (Eq. M_inverse in the proof of Lemma 4.4).

The factorisation of M2 adds a stabilising shift only if plain Cholesky fails
(the paper inverts M2 in exact arithmetic; this is the reading for floating
point): nu = s * 2^-52 * |M2|_F, multiplied by 100 per retry, at most 4 retries.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla


class NotPositiveDefinite(RuntimeError):
    pass


def lambda0_from_spectrum(eigs: np.ndarray, l: int) -> float:
    """lambda_0 = (2/l) sum_{i>l} lambda_i with eigenvalues in non-increasing order
    (Lemma 4.3 / Theorem 4.2)."""
    e = np.sort(np.asarray(eigs, dtype=np.float64))[::-1]
    return 2.0 / l * float(e[l:].sum())


def level2_matrix(Ct: np.ndarray, W: np.ndarray, lam_tilde: float) -> np.ndarray:
    """M2 = C~^T C~ + lambda~ W."""
    return Ct.T @ Ct + lam_tilde * W


@dataclasses.dataclass
class Factor:
    L: np.ndarray        # lower Cholesky factor of M2 + shift I
    shift: float
    retries: int

    def solve(self, v: np.ndarray) -> np.ndarray:
        """(M2 + shift I)^{-1} v by two triangular solves."""
        y = sla.solve_triangular(self.L, v, lower=True)
        return sla.solve_triangular(self.L.T, y, lower=False)


def cholesky_with_shift(M2: np.ndarray, max_retries: int = 4) -> Factor:
    s = M2.shape[0]
    try:
        return Factor(np.linalg.cholesky(M2), 0.0, 0)
    except np.linalg.LinAlgError:
        pass
    nu = s * 2.0 ** -52 * float(np.linalg.norm(M2, "fro"))
    for k in range(1, max_retries + 1):
        try:
            return Factor(np.linalg.cholesky(M2 + nu * np.eye(s)), nu, k)
        except np.linalg.LinAlgError:
            nu *= 100.0
    raise NotPositiveDefinite("M2 + shift is not positive definite after retries")


def woodbury_inverse_apply(C: np.ndarray, W: np.ndarray, lam_tilde: float,
                           r: np.ndarray) -> np.ndarray:
    """M^{-1} r = (1/lambda~)(r - C (C^T C + lambda~ W)^{-1} C^T r), dense solve
    (the exact SolveM1 used to isolate inner-solve effects)."""
    G = C.T @ C + lam_tilde * W
    y = np.linalg.solve(G, C.T @ r)
    return (r - C @ y) / lam_tilde


def nystrom_preconditioner_dense(C: np.ndarray, W: np.ndarray, lam_tilde: float) -> np.ndarray:
    """M = C W^{-1} C^T + lambda~ I formed densely (small n only)."""
    n = C.shape[0]
    return C @ np.linalg.solve(W, C.T) + lam_tilde * np.eye(n)
