"""Seeded generators for the synthetic MSP workloads.

Every array is produced in FP64 on the host with NumPy's PCG64
(``numpy.random.default_rng``), keyed by ``(seed, tag)`` so that the matrix,
the right-hand side and any per-instance draw come from independent streams.
The paper (Section 3, kernel ridge regression; Problem 1.1, matrices with a few
large singular values) names no public dataset; these generators stand in for
its two workload shapes:

* ``spectrum_matrix``: A = Q diag(sigma) Q^T with a prescribed spectrum (a few
  large outliers over a decaying or flat tail) -- the "k large singular values"
  shape of Problem 1.1.
* ``rbf_kernel``: a Gaussian (RBF) kernel matrix on uniform points in [0,1]^3 --
  the kernel ridge regression shape (K + lambda I) x = y.
* ``svd_matrix`` / ``tall_matrix``: rectangular m x n matrices with a few
  large singular values over a flat tail -- the general
  (A^T A + lambda I) x = c shape of the main technical result (Section 3).

Rounding to the storage precision (FP32 or BF16) is the caller's business; the
generated FP64 values are the definition of the problem.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# Stream tags for default_rng([seed, tag]).
_TAG_MATRIX = 0
_TAG_RHS = 1
_TAG_TAIL = 2
_TAG_INSTANCE = 3


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag)])


def outlier_spectrum(n: int, k: int, hi: float = 1e4, lo: float = 1e2,
                     tail_exp: float = 1.5) -> np.ndarray:
    """k outliers log-spaced from ``hi`` down to ``lo``, then sigma_i = i^-tail_exp
    for i = k+1..n (1-based i). Returned in non-increasing order."""
    if not (0 <= k <= n):
        raise ValueError("need 0 <= k <= n")
    out = np.logspace(math.log10(hi), math.log10(lo), k) if k > 0 else np.zeros(0)
    i = np.arange(k + 1, n + 1, dtype=np.float64)
    tail = i ** (-tail_exp)
    return np.concatenate([out, tail])


def householder_spectrum(n: int, k: int, seed: int, hi: float = 1e6,
                         lo: float = 1e2) -> np.ndarray:
    """k outliers log-spaced hi -> lo, then a flat tail 0.5 + 0.5 u, u ~ U(0,1),
    drawn in index order."""
    out = np.logspace(math.log10(hi), math.log10(lo), k)
    u = _rng(seed, _TAG_TAIL).random(n - k)
    return np.concatenate([out, 0.5 + 0.5 * u])


def gaussian_square(n: int, seed: int) -> np.ndarray:
    """The seeded N(0,1) n x n matrix whose orthogonal factor is the Q of
    ``spectrum_matrix`` (for large n the caller may factor it elsewhere)."""
    return _rng(seed, _TAG_MATRIX).standard_normal((n, n))


def spectrum_matrix(sigma: np.ndarray, seed: int) -> np.ndarray:
    """A = Q diag(sigma) Q^T with Q the orthogonal factor of a seeded N(0,1)
    n x n matrix (numpy.linalg.qr). sigma[i] is attached to column i of Q.
    The result is symmetrised exactly."""
    n = sigma.shape[0]
    G = gaussian_square(n, seed)
    Q, _ = np.linalg.qr(G)
    A = (Q * sigma[None, :]) @ Q.T
    return 0.5 * (A + A.T)


def householder_factors(n: int, seed: int, reflectors: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """Q = H_1 H_2 ... H_r, H_i = I - tau_i v_i v_i^T, tau_i = 2 / |v_i|^2, v_i ~ N(0, I)
    (row i of a seeded r x n draw), in compact WY form Q = I - Y T Y^T
    (Schreiber and Van Loan): Y = [v_1 ... v_r] (n x r) and T upper triangular,
    T_k = [[T_{k-1}, -tau_k T_{k-1} Y_{k-1}^T v_k], [0, tau_k]]."""
    V = _rng(seed, _TAG_MATRIX).standard_normal((reflectors, n))
    Y = np.ascontiguousarray(V.T)
    T = np.zeros((reflectors, reflectors))
    for k in range(reflectors):
        v = Y[:, k]
        tau = 2.0 / float(v @ v)
        if k:
            T[:k, k] = -tau * (T[:k, :k] @ (Y[:, :k].T @ v))
        T[k, k] = tau
    return Y, T


def householder_lowrank(sigma: np.ndarray, seed: int, reflectors: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """A = Q diag(sigma) Q^T = diag(sigma) + Z M Z^T with Q = I - Y T Y^T
    (``householder_factors``): U = Y T, P = diag(sigma) Y, S = Y^T diag(sigma) Y,
    Z = [U P] (n x 2r) and M = [[S, -I], [-I, 0]]. Returns (Z, M); a product
    A x then costs O(r n) and forming A one rank-2r update."""
    n = sigma.shape[0]
    Y, T = householder_factors(n, seed, reflectors)
    U = Y @ T
    P = sigma[:, None] * Y
    S = Y.T @ P
    S = 0.5 * (S + S.T)
    r = reflectors
    M = np.zeros((2 * r, 2 * r))
    M[:r, :r] = S
    M[:r, r:] = -np.eye(r)
    M[r:, :r] = -np.eye(r)
    return np.concatenate([U, P], axis=1), M


def householder_matrix(sigma: np.ndarray, seed: int, reflectors: int = 64) -> np.ndarray:
    """A = Q diag(sigma) Q^T with Q = H_1 H_2 ... H_r, H_i = I - 2 v v^T / |v|^2,
    v_i ~ N(0, I), formed as diag(sigma) + Z M Z^T (``householder_lowrank``,
    one rank-2r product, O(r n^2)), then symmetrised exactly."""
    Z, M = householder_lowrank(sigma, seed, reflectors)
    A = Z @ (M @ Z.T)
    A[np.diag_indices_from(A)] += sigma
    return 0.5 * (A + A.T)


def svd_matrix(m: int, n: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T (m x n, m >= n) with U, V the orthogonal factors
    (numpy.linalg.qr) of seeded N(0,1) m x n and n x n matrices: exactly the
    singular values sigma. For the general (A^T A + lambda I) systems."""
    if m < n or sigma.shape[0] != n:
        raise ValueError("need m >= n and n singular values")
    r = _rng(seed, _TAG_MATRIX)
    U, _ = np.linalg.qr(r.standard_normal((m, n)))
    V, _ = np.linalg.qr(r.standard_normal((n, n)))
    return (U * sigma[None, :]) @ V.T


def tall_matrix(m: int, n: int, d: np.ndarray, seed: int, out_dtype=np.float32,
                chunk: int = 8192) -> np.ndarray:
    """A = G diag(d) / sqrt(m) with G seeded N(0,1) (m x n), drawn row chunk by
    row chunk in FP64 and rounded once to ``out_dtype``. For m >> n the
    singular values are d_i (1 + O(sqrt(n/m))): the large-size stand-in for
    ``svd_matrix`` (no QR of an m x n matrix)."""
    if d.shape[0] != n:
        raise ValueError("need n column scales")
    r = _rng(seed, _TAG_MATRIX)
    A = np.empty((m, n), dtype=out_dtype)
    scale = d[None, :] / math.sqrt(m)
    for i in range(0, m, chunk):
        rows = min(chunk, m - i)
        A[i:i + rows] = (r.standard_normal((rows, n)) * scale).astype(out_dtype)
    return A


def rbf_points(n: int, seed: int, dim: int = 3) -> np.ndarray:
    """n points uniform in [0,1]^dim, FP64, shape (n, dim)."""
    return _rng(seed, _TAG_MATRIX).random((n, dim))


def rbf_kernel(P: np.ndarray, ell: float, out_dtype=np.float64,
               block: int = 2048) -> np.ndarray:
    """K_ij = exp(-|p_i - p_j|^2 / (2 ell^2)) evaluated in FP64 and rounded once to
    ``out_dtype``. Built in row blocks to bound host memory."""
    n = P.shape[0]
    K = np.empty((n, n), dtype=out_dtype)
    sq = np.einsum("ij,ij->i", P, P)
    inv = 1.0 / (2.0 * ell * ell)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        d2 = sq[i0:i1, None] + sq[None, :] - 2.0 * (P[i0:i1] @ P.T)
        # exact diagonal and no negative round-off
        np.maximum(d2, 0.0, out=d2)
        for i in range(i0, i1):
            d2[i - i0, i] = 0.0
        K[i0:i1] = np.exp(-d2 * inv).astype(out_dtype)
    return K


def rhs(n: int, seed: int, m: int = 1) -> np.ndarray:
    """b ~ N(0, I), shape (n,) for m == 1 else (n, m) (column j = right-hand side j)."""
    g = _rng(seed, _TAG_RHS).standard_normal((n, m))
    return g[:, 0].copy() if m == 1 else g


@dataclasses.dataclass
class Workload:
    """One synthetic problem instance (A + lam I) x = b."""
    name: str
    A: np.ndarray            # FP64 (or the storage dtype for RBF), n x n, symmetric
    b: np.ndarray            # FP64, (n,) or (n, m)
    lam: float
    s: int                   # sketch size
    gamma: int               # nonzeros per row of Pi = S^T
    sigma: np.ndarray | None = None   # exact spectrum when known
    points: np.ndarray | None = None  # RBF points when applicable
    ell: float | None = None

    @property
    def n(self) -> int:
        return self.A.shape[0]


def make_workload(name: str, seed: int = 0, n: int | None = None,
                  m: int = 1, rbf_dtype=np.float32) -> Workload:
    """Build one of the named synthetic workloads.

    ``outlier``  : config-0 shape, n=1024 default, 32 outliers 1e4->1e2, tail i^-1.5,
                   lam=1e-3, s=64, gamma=8 (FP64).
    ``rbf``      : GP-regression shape, n=16384 default, ell=0.1, lam=1e-2, s=1024,
                   gamma=8; the kernel is rounded once to ``rbf_dtype``.
    ``outlier256``: Schatten-1 shape, n=16384 default, 256 outliers, tail i^-1.5.
    ``householder``: n=32768 default, 1024 outliers 1e6->1e2, tail 0.5+0.5u,
                   lam=1e-4, s=2048.
    ``n`` rescales the size; ``s`` keeps the default ratio n/s (at least 16).
    """
    if name == "outlier":
        n = n or 1024
        k = max(1, (32 * n) // 1024)
        sig = outlier_spectrum(n, min(k, n))
        A = spectrum_matrix(sig, seed)
        s = max(16, (64 * n) // 1024)
        return Workload(name, A, rhs(n, seed, m), 1e-3, s, 8, sigma=sig)
    if name == "rbf":
        n = n or 16384
        P = rbf_points(n, seed)
        K = rbf_kernel(P, 0.1, out_dtype=rbf_dtype)
        s = max(16, (1024 * n) // 16384)
        return Workload(name, K, rhs(n, seed, m), 1e-2, s, 8, points=P, ell=0.1)
    if name == "outlier256":
        n = n or 16384
        k = max(1, (256 * n) // 16384)
        sig = outlier_spectrum(n, k)
        A = spectrum_matrix(sig, seed)
        s = max(16, (1024 * n) // 16384)
        return Workload(name, A, rhs(n, seed, m), 1e-3, s, 8, sigma=sig)
    if name == "householder":
        n = n or 32768
        k = max(1, (1024 * n) // 32768)
        sig = householder_spectrum(n, k, seed)
        A = householder_matrix(sig, seed)
        s = max(16, (2048 * n) // 32768)
        return Workload(name, A, rhs(n, seed, m), 1e-4, s, 8, sigma=sig)
    raise ValueError(f"unknown workload {name!r}")


@dataclasses.dataclass
class BatchSpec:
    """One instance of the batched workload: the RBF kernel of ``rbf_kernel`` on
    n uniform points in [0,1]^3 with length scale ell, (K + lam I) X = B with
    B ~ N(0, I) of shape (n, m), sketch size s."""
    n: int
    ell: float
    lam: float
    s: int
    m: int
    seed: int


def batch_specs(seed: int, count: int = 64, n_lo: int = 512, n_hi: int = 8192, m: int = 16,
                lam: float = 1e-2, ell_lo: float = 0.05, ell_hi: float = 0.2,
                s_max: int = 1024) -> list[BatchSpec]:
    """``count`` instances with n ~ U{n_lo..n_hi} and ell ~ U(ell_lo, ell_hi), drawn
    in instance order; s = min(s_max, n / 4) rounded down to a multiple of 64
    (at least 64, at most n). Instance k draws its points and right-hand sides
    with seed ``seed * 4096 + k + 1``."""
    g = _rng(seed, _TAG_INSTANCE)
    ns = g.integers(n_lo, n_hi + 1, size=count)
    ells = g.uniform(ell_lo, ell_hi, size=count)
    out = []
    for k in range(count):
        n = int(ns[k])
        s = min(s_max, max(64, (n // 4) // 64 * 64), n)
        out.append(BatchSpec(n, float(ells[k]), lam, s, m, seed * 4096 + k + 1))
    return out


def batch_instance(spec: BatchSpec, out_dtype=np.float32) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(points, K rounded once to ``out_dtype``, B (n, m) FP64) of one instance."""
    P = rbf_points(spec.n, spec.seed)
    K = rbf_kernel(P, spec.ell, out_dtype=out_dtype)
    B = _rng(spec.seed, _TAG_RHS).standard_normal((spec.n, spec.m))
    return P, K, B


WORKLOADS = ("outlier", "rbf", "outlier256", "householder")
