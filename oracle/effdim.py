"""Effective dimension by Hutchinson over regularised solves (oracle, FP64).

d_lambda = tr(A (A + lambda I)^{-1}) = sum_i sigma_i / (sigma_i + lambda)
(Section 2, Lemma 2.1's quantity; the KRR analysis of Section 3 sets the
sketch size from it). With A (A + lambda I)^{-1} = I - lambda (A + lambda I)^{-1},

    d_lambda = n - lambda tr((A + lambda I)^{-1}),

and the trace is estimated as in the Schatten-1 estimator: the mean over
Rademacher probes g_j of g_j^T (A + lambda I)^{-1} g_j, the solves being the
regularised systems the method solves. Probes are those of ``hutchinson``.
"""

from __future__ import annotations

import numpy as np

from . import reference


def quadratic_forms(A: np.ndarray, lam: float, G: np.ndarray, solve=None) -> np.ndarray:
    """q_j = g_j^T (A + lam I)^{-1} g_j; ``solve(A, G, lam)`` defaults to the
    dense Cholesky solve."""
    X = (solve or reference.solve_dense)(A, G, lam)
    return np.einsum("ij,ij->j", G, X)


def estimate(A: np.ndarray, lam: float, G: np.ndarray, solve=None) -> tuple[float, float]:
    """(estimate of d_lambda, standard error of the mean over probes)."""
    n, m = G.shape
    vals = n - lam * quadratic_forms(A, lam, G, solve)
    se = float(vals.std(ddof=1) / np.sqrt(m)) if m > 1 else float("nan")
    return float(vals.mean()), se


def variance_one_probe(A: np.ndarray, lam: float) -> float:
    """Var(n - lam g^T (A + lam I)^{-1} g) for Rademacher g: with
    B = lam (A + lam I)^{-1} symmetric, Var(g^T B g) = 2 (|B|_F^2 - sum_i B_ii^2)."""
    A = np.asarray(A, dtype=np.float64)
    B = lam * np.linalg.inv(A + lam * np.eye(A.shape[0]))
    return float(2.0 * (np.sum(B * B) - np.sum(np.diag(B) ** 2)))


def params_from_effdim(d: float, n: int, lam: float, s_cap: int = 1024) -> dict:
    """Sketch size and shift from d_lambda, as Section 3 and Lemma 2.1 give them.

    * l = 2 d_lambda (the KRR corollary's choice), taken as the integer
      ceiling; Lemma 2.1(1) with gamma = 1 then gives lambda_l <= lambda.
    * s = l, rounded up to a multiple of 16 (the library's tile), but no
      larger than min(n, s_cap) rounded down to a multiple of 16, and no
      smaller than 16. ``capped`` records s < l.
    * lambda0: the paper's shift is (2/s) sum_{i>s} lambda_i. For s >= d,
      Lemma 2.1(2) bounds the tail sum by lambda d, so 2 lambda d / s is an
      upper bound of that shift computable from d alone; below d the lemma
      gives no bound and the shift is 0.
    * direct: d >= n/4, where the paper inverts A + lambda I directly.
    """
    if not (d >= 0.0 and np.isfinite(d)) or n < 16 or not lam > 0.0:
        raise ValueError("need d >= 0 finite, n >= 16, lam > 0")
    l = max(1, int(np.ceil(2.0 * d)))
    top = (min(n, s_cap) // 16) * 16
    s = min(top, -(-l // 16) * 16)
    s = max(16, s)
    lam0 = 2.0 * lam * d / s if s >= d else 0.0
    return {"d_lambda": float(d), "l": l, "s": s, "lambda0": lam0, "capped": int(s < l),
            "direct": int(4.0 * d >= n)}
