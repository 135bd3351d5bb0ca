"""Pins for the oracle's random draws and sketches (Definition 2.1, Algorithm 1
steps 2-4). Every check compares against something other than the oracle's own
formula: published generator outputs, brute force over tiny inputs, exact
structural facts and distributional tests with fixed seeds."""

import itertools
import math

import numpy as np
import pytest

from oracle import prng, sketch


def test_splitmix64_published_vectors():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: the first four outputs
    # of the reference generator (as used to seed the xoshiro family).
    assert [prng.splitmix64_output(0, k) for k in range(4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    # Seeded with 1234567: the test vector of java.util.SplittableRandom's
    # algorithm (same generator), as unsigned decimals.
    assert [prng.splitmix64_output(1234567, k) for k in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_below_edges():
    assert prng.uniform_below(0, 17) == 0
    assert prng.uniform_below((1 << 64) - 1, 17) == 16
    assert prng.uniform_below(1 << 63, 10) == 5


def test_counter_layout_and_ranges():
    assert prng.counter(0, 0, 0) == 0
    assert prng.counter(1, 0, 0) == 1 << 56
    assert prng.counter(0, 1, 0) == 1 << 8
    assert prng.counter(3, 5, 7) == (3 << 56) | (5 << 8) | 7
    with pytest.raises(ValueError):
        prng.counter(0, 1 << 48, 0)
    with pytest.raises(ValueError):
        prng.counter(0, 0, 256)


def test_floyd_full_set_and_structure():
    assert prng.floyd_sample(7, 0, 3, 16, 16) == list(range(16))
    for row in range(200):
        v = prng.floyd_sample(11, 0, row, 1024, 8)
        assert v == sorted(set(v)) and len(v) == 8
        assert 0 <= v[0] and v[-1] < 1024


def test_floyd_uniform_over_subsets():
    # s=5, gamma=2: all C(5,2)=10 subsets equally likely. Chi-square over 20000
    # rows with a fixed seed (deterministic); 99.9% point of chi2(9) is 27.9.
    counts = {c: 0 for c in itertools.combinations(range(5), 2)}
    N = 20000
    for row in range(N):
        counts[tuple(prng.floyd_sample(3, 0, row, 5, 2))] += 1
    e = N / 10
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 27.9


def test_signs_balanced():
    sg = np.array([prng.signs_for_row(5, 0, row, 8) for row in range(4000)])
    frac = (sg > 0).mean()
    assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / sg.size)
    assert set(np.unique(sg)) == {-1, 1}


def test_embedding_structure():
    n, s, g = 300, 40, 6
    S = sketch.sparse_embedding(n, s, g, seed=1).toarray()
    assert S.shape == (s, n)
    nnz = (S != 0).sum(axis=0)
    assert np.all(nnz == g)
    assert np.allclose(np.abs(S[S != 0]), 1 / math.sqrt(g), rtol=0, atol=0)
    # every column has unit norm exactly: gamma entries of 1/gamma
    assert np.allclose((S * S).sum(axis=0), 1.0, rtol=0, atol=1e-15)
    # independent streams: Phi differs from S with the same seed
    P = sketch.level2_embedding(n, s, g, seed=1).toarray()
    assert not np.array_equal(P, S)


def test_embedding_second_moment():
    # E[S^T S] = I for a sparse embedding: off-diagonal entries average to 0.
    n, s, g = 64, 512, 8
    acc = np.zeros((n, n))
    reps = 40
    for rep in range(reps):
        S = sketch.sparse_embedding(n, s, g, seed=100 + rep).toarray()
        acc += S.T @ S
    acc /= reps
    off = acc - np.diag(np.diag(acc))
    assert np.allclose(np.diag(acc), 1.0)
    # each off-diagonal entry of S^T S has variance ~ g/s * (1/g)... bounded here
    assert np.abs(off).max() < 0.08


def _brute_sketch(A, S):
    n = A.shape[0]
    s = S.shape[0]
    C = np.zeros((n, s))
    for i in range(n):
        for c in range(s):
            acc = 0.0
            for j in range(n):
                acc += A[i, j] * S[c, j]
            C[i, c] = acc
    return C


def test_sketch_C_W_Ct_brute_force():
    rng = np.random.default_rng(0)
    n, s, phi = 23, 7, 9
    B = rng.standard_normal((n, n))
    A = B @ B.T
    S = sketch.sparse_embedding(n, s, 3, seed=9)
    Phi = sketch.level2_embedding(n, phi, 2, seed=9)
    Sd, Pd = S.toarray(), Phi.toarray()
    C = sketch.sketch_C(A, S)
    assert np.allclose(C, _brute_sketch(A, Sd), rtol=1e-13, atol=1e-12)
    W = sketch.core_W(S, C)
    assert np.allclose(W, Sd @ A @ Sd.T, rtol=1e-12, atol=1e-12)
    assert np.array_equal(W, W.T)
    Ct = sketch.level2_sketch(Phi, C)
    brute = np.array([[sum(Pd[r, j] * C[j, c] for j in range(n)) for c in range(s)]
                      for r in range(phi)])
    assert np.allclose(Ct, brute, rtol=1e-13, atol=1e-12)
