"""Sparse embeddings and the sketches of Algorithm 1 (oracle side, FP64).

Definition 2.1 (sparse embedding matrix): S is s x n; its columns are
independent; each column has gamma entries at rows chosen uniformly without
replacement, each set to +-1/sqrt(gamma) with independent signs; all other
entries are zero. The paper writes the sketch of A as C = A S^T, so
Pi := S^T is n x s with gamma nonzeros in every ROW (row j of Pi is column j of
S).

Lemma 2.2 names an oblivious subspace embedding Phi (phi x n) for the level-2
sketch C~ = Phi C but gives no construction. Reading used here: Phi is itself a
sparse embedding matrix (Definition 2.1) with phi rows and gamma_phi nonzeros
per column, drawn from its own streams.

Stream ids: S uses streams 0 (indices) and 1 (signs); Phi uses 2 and 3.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import prng

STREAM_S = 0
STREAM_PHI = 2


def embedding_pattern(n: int, rows: int, gamma: int, seed: int, stream: int):
    """Index/sign pattern of a rows x n sparse embedding (Definition 2.1).

    Returns (idx, sgn): int64 and int8 arrays of shape (n, gamma); column j of the
    embedding has value sgn[j, q] / sqrt(gamma) at row idx[j, q]; idx[j] is
    sorted ascending.
    """
    idx = np.empty((n, gamma), dtype=np.int64)
    sgn = np.empty((n, gamma), dtype=np.int8)
    for j in range(n):
        idx[j] = prng.floyd_sample(seed, stream, j, rows, gamma)
        sgn[j] = prng.signs_for_row(seed, stream, j, gamma)
    return idx, sgn


def embedding_matrix(idx: np.ndarray, sgn: np.ndarray, rows: int) -> sp.csr_matrix:
    """The rows x n sparse matrix with entries sgn/sqrt(gamma) at (idx[j,q], j)."""
    n, gamma = idx.shape
    val = sgn.astype(np.float64).ravel() * (1.0 / math.sqrt(gamma))
    cols = np.repeat(np.arange(n, dtype=np.int64), gamma)
    return sp.csr_matrix((val, (idx.ravel(), cols)), shape=(rows, n))


def sparse_embedding(n: int, s: int, gamma: int, seed: int) -> sp.csr_matrix:
    """S in R^{s x n} (Definition 2.1) from the sketch streams."""
    idx, sgn = embedding_pattern(n, s, gamma, seed, STREAM_S)
    return embedding_matrix(idx, sgn, s)


def level2_embedding(n: int, phi: int, gamma_phi: int, seed: int) -> sp.csr_matrix:
    """Phi in R^{phi x n} (reading of Lemma 2.2: a sparse embedding)."""
    idx, sgn = embedding_pattern(n, phi, gamma_phi, seed, STREAM_PHI)
    return embedding_matrix(idx, sgn, phi)


def sketch_C(A: np.ndarray, S: sp.spmatrix) -> np.ndarray:
    """C = A S^T (Algorithm 1, step 3), FP64."""
    A = np.asarray(A, dtype=np.float64)
    return np.asarray((S @ A.T).T)


def core_W(S: sp.spmatrix, C: np.ndarray) -> np.ndarray:
    """W = S C (Algorithm 1, step 3). S A S^T is symmetric in exact arithmetic;
    the rounding asymmetry is removed by (W + W^T)/2."""
    W = np.asarray(S @ C)
    return 0.5 * (W + W.T)


def level2_sketch(Phi: sp.spmatrix, C: np.ndarray) -> np.ndarray:
    """C~ = Phi C (Algorithm 1, step 4)."""
    return np.asarray(Phi @ C)
