"""Pins of the oracle's batched solve (CPU only).

A batch is independent per-column solves (no coupling between columns or
instances). Pinned against: the dense Cholesky solution through the bound
|x - x*| <= |r| / lambda (A PSD, so |(A + lam I)^{-1}| <= 1 / lam), exact
permutation equivariance of the columns, and the zero right-hand side.
"""

import numpy as np

import workloads
from oracle import batch, msp, reference


def _inst(n, ell, m, seed, s):
    spec = workloads.BatchSpec(n, ell, 1e-2, s, m, seed)
    _, K, B = workloads.batch_instance(spec, out_dtype=np.float64)
    return K, B


def _params(s):
    return msp.MspParams(s=s, gamma=8, phi=0, inner="exact", tol=1e-10)


def test_batch_columns_meet_the_dense_solution():
    K, B = _inst(160, 0.15, 3, 11, 40)
    X = batch.solve_instance(K, B, 1e-2, _params(40), refine_tol=1e-6)
    for j in range(3):
        r = B[:, j] - (K @ X[:, j] + 1e-2 * X[:, j])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[:, j])
        xs = reference.solve_dense(K, B[:, j], 1e-2)
        assert np.linalg.norm(X[:, j] - xs) <= 1.01 * np.linalg.norm(r) / 1e-2 + 1e-14


def test_batch_permutation_and_duplicates():
    K, B = _inst(120, 0.08, 4, 5, 32)
    p = _params(32)
    perm = [2, 0, 3, 1]
    X1, X2, X3 = batch.solve_batch([(K, B, 1e-2, p), (K, B[:, perm], 1e-2, p), (K, B, 1e-2, p)])
    assert np.array_equal(X2, X1[:, perm])
    assert np.array_equal(X3, X1)


def test_batch_zero_column():
    K, B = _inst(96, 0.1, 2, 3, 24)
    B[:, 1] = 0.0
    X = batch.solve_instance(K, B, 1e-2, _params(24))
    assert not np.any(X[:, 1])
    assert np.linalg.norm(B[:, 0] - (K @ X[:, 0] + 1e-2 * X[:, 0])) <= 1e-10 * np.linalg.norm(B[:, 0])


def test_batch_specs_recipe():
    sp = workloads.batch_specs(0, count=64)
    assert len(sp) == 64
    for s in sp:
        assert 512 <= s.n <= 8192 and 0.05 <= s.ell <= 0.2 and s.m == 16
        assert s.s % 64 == 0 and 64 <= s.s <= min(1024, s.n)
        assert s.s == min(1024, (s.n // 4) // 64 * 64)
    assert len({s.seed for s in sp}) == 64
