"""Pins for the seeded input generators: the Householder-product matrix of the
mixed-precision workload (n = 32768, 64 reflectors, 1024 outliers) is formed in
compact WY form; here it must equal the reflectors applied one by one, with Q
orthogonal and the prescribed spectrum."""

import numpy as np

from workloads import householder_factors, householder_lowrank, householder_matrix, householder_spectrum


def _explicit_q(n, seed, r):
    # the definition: Q = H_1 H_2 ... H_r with v_i row i of the seeded draw
    from workloads.generators import _TAG_MATRIX, _rng
    V = _rng(seed, _TAG_MATRIX).standard_normal((r, n))
    Q = np.eye(n)
    for i in range(r):
        v = V[i]
        Q = Q - (2.0 / (v @ v)) * np.outer(Q @ v, v)     # Q H_i
    return Q


def test_wy_form_equals_the_reflector_product():
    n, r, seed = 96, 12, 3
    Y, T = householder_factors(n, seed, r)
    Q = np.eye(n) - Y @ T @ Y.T
    assert np.abs(Q - _explicit_q(n, seed, r)).max() <= 1e-13
    assert np.abs(Q @ Q.T - np.eye(n)).max() <= 1e-13
    assert np.allclose(np.triu(T), T)


def test_householder_matrix_spectrum_and_lowrank_product():
    n, r, seed = 200, 16, 5
    sig = householder_spectrum(n, 8, seed, hi=1e6, lo=1e2)
    A = householder_matrix(sig, seed, r)
    Q = _explicit_q(n, seed, r)
    ref = (Q * sig) @ Q.T
    assert np.abs(A - ref).max() <= 1e-15 * n * sig.max()
    assert np.array_equal(A, A.T)
    ev = np.sort(np.linalg.eigvalsh(A))
    assert np.allclose(ev, np.sort(sig), rtol=1e-9, atol=1e-9 * sig.max())
    # the O(r n) product diag(sigma) x + Z (M (Z^T x)) matches the dense A
    Z, M = householder_lowrank(sig, seed, r)
    x = np.random.default_rng(0).standard_normal(n)
    assert np.allclose(sig * x + Z @ (M @ (Z.T @ x)), A @ x, rtol=0, atol=1e-9 * sig.max())
