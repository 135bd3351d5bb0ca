"""Schatten-p norms for p in (0, 2) from ridge solves (Section 3.2), FP64
(oracle side; test infrastructure only).

The paper treats the estimator of Musco et al. as a black box whose only
requirement is solving ridge systems (A^T A + t I) x = y (eq. schatten-ridge),
plus a random diagonal shift A + zI that bounds the condition number. The
black box itself is not printed; this oracle uses a published integral
representation instead (Balakrishnan's formula for fractional powers): for
q in (0, 1) and x >= 0,

    x^q = (sin(pi q) / pi) * int_0^inf t^(q-1) x / (x + t) dt.

Applied to the eigenvalues sigma_i^2 of A^T A with q = p / 2,

    |A|_p^p = sum_i sigma_i^p
            = (sin(pi q) / pi) * int_0^inf t^(q-1) d_t dt,
    d_t     = tr(A^T A (A^T A + t I)^{-1}) = n - t tr((A^T A + t I)^{-1}),

the effective dimension of A^T A at t, estimated by Hutchinson over ridge
solves. With u = ln t the integrand f(u) = e^(q u) d_(e^u) is analytic in
the strip |Im u| < pi and decays at both ends, so the trapezoidal rule on
the whole line, h sum_k f(u_0 + k h), converges geometrically in 1/h. The
nodes u_0 .. u_N cover [ln t_min, ln t_max]; beyond them f is replaced by
its asymptotic forms, f ~ n e^(q u) (t -> 0, full column rank) and
f ~ |A|_F^2 e^((q-1) u) (t -> inf), whose trapezoidal sums are geometric:

    below:  h n t_min^q e^(-q h) / (1 - e^(-q h)),
    above:  h |A|_F^2 t_max^(q-1) e^(-(1-q) h) / (1 - e^(-(1-q) h)).

(Halving the end weights and integrating the tails exactly instead leaves
the endpoint terms of the Euler-Maclaurin expansion, O(h^2).)
"""

from __future__ import annotations

import math

import numpy as np

from . import reference


def nodes(t_min: float, t_max: float, count: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes t_j uniform in ln t over [t_min, t_max] and their trapezoidal
    weights h (in u = ln t); count >= 2."""
    u = np.linspace(math.log(t_min), math.log(t_max), count)
    h = np.full(count, (u[-1] - u[0]) / (count - 1))
    return np.exp(u), h


def combine(p: float, t: np.ndarray, h: np.ndarray, d_t: np.ndarray, n: int, fro2: float) -> float:
    """(sin(pi q)/pi) [sum_j h t_j^q d_t(j) + the two geometric tails], q = p/2."""
    q = 0.5 * p
    step = float(h[0])
    body = float(np.sum(h * t ** q * d_t))
    a, b = math.exp(-q * step), math.exp(-(1.0 - q) * step)
    lower = step * n * t[0] ** q * a / (1.0 - a)
    upper = step * fro2 * t[-1] ** (q - 1.0) * b / (1.0 - b)
    return math.sin(math.pi * q) / math.pi * (body + lower + upper)


def exact_effdims(sig: np.ndarray, t: np.ndarray) -> np.ndarray:
    """d_t from the singular values (closed form)."""
    e = np.asarray(sig, dtype=np.float64) ** 2
    return np.array([float(np.sum(e / (e + tj))) for tj in t])


def probe_values(A: np.ndarray, t: np.ndarray, G: np.ndarray) -> np.ndarray:
    """v[j, k] = n - t_j g_k^T (A^T A + t_j I)^{-1} g_k (dense solves)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    AtA = A.T @ A
    out = np.empty((t.shape[0], G.shape[1]))
    for j, tj in enumerate(t):
        X = reference.solve_dense(AtA, G, tj)
        out[j] = n - tj * np.einsum("ij,ij->j", G, X)
    return out


def estimate(A: np.ndarray, p: float, t_min: float, t_max: float, count: int, G: np.ndarray,
             z: float = 0.0) -> tuple[float, float, np.ndarray]:
    """Estimate of |A + z I|_p^p (z only for square A), its standard error
    over the probes, and the per-probe estimates X_k."""
    A = np.asarray(A, dtype=np.float64)
    if z != 0.0:
        if A.shape[0] != A.shape[1]:
            raise ValueError("the shift z I needs a square A")
        A = A + z * np.eye(A.shape[0])
    n = A.shape[1]
    fro2 = float(np.sum(A * A))
    t, h = nodes(t_min, t_max, count)
    V = probe_values(A, t, G)
    X = np.array([combine(p, t, h, V[:, k], n, fro2) for k in range(G.shape[1])])
    se = float(X.std(ddof=1) / math.sqrt(X.shape[0])) if X.shape[0] > 1 else float("nan")
    return float(X.mean()), se, X


def exact(A: np.ndarray, p: float) -> float:
    """sum_i sigma_i^p from the SVD."""
    return reference.schatten(np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False), p) ** p
