"""Hutchinson trace estimation for the Schatten-1 norm of a PSD matrix
(oracle side, FP64).

The paper's norm estimators (Section 3.2, after Musco et al.) combine
stochastic trace estimation g^T f(A) g with regularised solves. For PSD A and
p = 1, |A|_1 = sum_i sigma_i = tr(A), so f is the identity and no solve is
needed: the estimate is (1/m) sum_j g_j^T A g_j with Rademacher probes g_j
(entries +-1 with probability 1/2 each).

Probes come from the counter-based generator of ``prng`` (the reading used on
both sides): probe j, row i is negative iff the top bit of
draw(seed, 7 + 2 (j // 256), i, j mod 256) is set.
"""

from __future__ import annotations

import numpy as np

from . import prng

PROBE_STREAM = 7


def probe_sign(seed: int, i: int, j: int) -> int:
    return -1 if (prng.draw(seed, PROBE_STREAM + 2 * (j // 256), i, j % 256) >> 63) else 1


def probes(n: int, m: int, seed: int) -> np.ndarray:
    """G in {+-1}^{n x m} (column j is probe j)."""
    G = np.empty((n, m), dtype=np.float64)
    for i in range(n):
        for j in range(m):
            G[i, j] = probe_sign(seed, i, j)
    return G


def probes_fast(n: int, m: int, seed: int) -> np.ndarray:
    """``probes`` computed with wrapping uint64 array arithmetic (the same
    SplitMix64 definition as ``prng``, evaluated for all (i, j) at once), for
    sizes where the per-entry loop is too slow. Equal to ``probes`` entry for
    entry (pinned)."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(m, dtype=np.uint64)[None, :]
    stream = np.uint64(PROBE_STREAM) + np.uint64(2) * (j // np.uint64(256))
    k = (stream << np.uint64(56)) | (i << np.uint64(8)) | (j % np.uint64(256))
    with np.errstate(over="ignore"):
        z = np.uint64(seed & prng.MASK64) + (k + np.uint64(1)) * np.uint64(prng.GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) != 0, -1.0, 1.0)


def quadratic_forms(A: np.ndarray, G: np.ndarray) -> np.ndarray:
    """q_j = g_j^T A g_j in FP64."""
    A = np.asarray(A, dtype=np.float64)
    return np.einsum("ij,ij->j", G, A @ G)


def estimate(A: np.ndarray, G: np.ndarray) -> tuple[float, float]:
    """(trace estimate, standard error of the mean over probes)."""
    q = quadratic_forms(A, G)
    m = q.shape[0]
    return float(q.mean()), float(q.std(ddof=1) / np.sqrt(m)) if m > 1 else float("nan")


def rademacher_variance(A: np.ndarray) -> float:
    """Var(g^T A g) = 2 (|A|_F^2 - sum_i A_ii^2) for symmetric A, Rademacher g."""
    A = np.asarray(A, dtype=np.float64)
    return float(2.0 * (np.sum(A * A) - np.sum(np.diag(A) ** 2)))
