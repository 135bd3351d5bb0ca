"""Schatten-1 norm of a PSD matrix by Hutchinson (row a10): per-probe parity
of q_j = g_j^T A g_j with the FP64 oracle on the same probes, and the estimate
against the exact sum of singular values."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hutchinson, reference
from workloads import make_workload, outlier_spectrum, spectrum_matrix

pytestmark = pytest.mark.gpu
SEED = 0x4D5350


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


# (n, m): rows 16-byte aligned (n % 4 == 0) take the tensor-core path, the
# others the SIMT path; 320 probes are two groups (256 + 64), 1000 leaves a
# ragged last tile row and column
@pytest.mark.parametrize("n,m", [(200, 64), (1000 + 37, 128), (2048, 320), (1000, 320), (4096 + 128, 256),
                                 (130, 192)])
def test_quadratic_forms_match_oracle(ctx, n, m):
    sig = outlier_spectrum(n, max(4, n // 64))
    A = spectrum_matrix(sig, seed=n).astype(np.float32)
    q = ctx.hutchinson(torch.from_numpy(A).cuda(), probes=m, seed=SEED).cpu().numpy()
    G = hutchinson.probes(n, m, SEED)
    A64 = A.astype(np.float64)
    qo = hutchinson.quadratic_forms(A64, G)
    # FP32 128-term tile sums + 128-term contraction, FP64 across tiles:
    # |dq_j| <= c u32 sum_ik |A_ik| (|g_i| = |g_k| = 1)
    bound = 512 * 2.0 ** -24 * np.abs(A64).sum()
    assert np.all(np.abs(q - qo) <= bound)


def test_schatten1_estimate_outlier_spectrum(ctx):
    # 2048 x 2048 PSD, 32 outliers 1e4 -> 1e2, tail i^-1.5: |A|_1 = sum sigma
    n = 2048
    sig = outlier_spectrum(n, 32)
    A = spectrum_matrix(sig, seed=7)
    est, se = ctx.schatten(torch.from_numpy(A.astype(np.float32)).cuda(), p=1.0, probes=256)
    exact = reference.schatten(sig, 1.0)
    sd = np.sqrt(hutchinson.rademacher_variance(A) / 256)
    assert abs(est - exact) <= 4 * sd
    assert se == pytest.approx(sd, rel=0.3)


def test_schatten1_rbf_trace_is_n(ctx):
    # RBF kernel: K_ii = 1, so |K|_1 = tr K = n exactly
    w = make_workload("rbf", seed=3, n=4096)
    K = torch.from_numpy(w.A.astype(np.float32)).cuda()
    est, se = ctx.schatten(K, p=1.0, probes=256)
    assert abs(est - 4096) <= 4 * se + 1e-9 * 4096


def test_schatten_rejects_other_p(ctx):
    from paper_2405_05865_gb300 import MspError
    A = torch.eye(128, dtype=torch.float32, device="cuda")
    with pytest.raises(MspError) as e:
        ctx.schatten(A, p=0.5)
    assert e.value.status == 1


def test_quadratic_forms_full_size(ctx):
    # the bench's size: n = 16384, 256 probes, every q_j against the FP64
    # oracle on the same probes (RBF matrix, FP64 values rounded once to FP32)
    w = make_workload("rbf", seed=2, n=16384)
    A = np.ascontiguousarray(w.A, dtype=np.float32)
    q = ctx.hutchinson(torch.from_numpy(A).cuda(), probes=256, seed=SEED).cpu().numpy()
    G = hutchinson.probes_fast(16384, 256, SEED)
    A64 = A.astype(np.float64)
    qo = hutchinson.quadratic_forms(A64, G)
    bound = 512 * 2.0 ** -24 * np.abs(A64).sum()
    assert np.all(np.abs(q - qo) <= bound)
    # and far inside it: the three BF16 terms carry the whole FP32 significand
    assert np.abs(q - qo).max() <= 1e-5 * np.abs(qo).max()


def test_schatten1_outlier_spectrum_tensor_core_sizes(ctx):
    # |A|_1 = sum sigma of a 4096 x 4096 PSD matrix (64 outliers 1e4 -> 1e2,
    # tail i^-1.5) within 4 Rademacher standard deviations
    n = 4096
    sig = outlier_spectrum(n, 64)
    A = spectrum_matrix(sig, seed=9)
    est, se = ctx.schatten(torch.from_numpy(A.astype(np.float32)).cuda(), p=1.0, probes=256)
    sd = np.sqrt(hutchinson.rademacher_variance(A) / 256)
    assert abs(est - reference.schatten(sig, 1.0)) <= 4 * sd


def test_fp16_two_term_and_bf16_three_term_products(ctx):
    # default: two FP16 terms of s a (22 significant bits); three BF16 terms
    # hold the FP32 significand exactly; both against the FP64 oracle
    n, m = 3000, 256
    sig = outlier_spectrum(n, 40)
    A = spectrum_matrix(sig, seed=17).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    q2 = ctx.hutchinson(Ad, probes=m, seed=SEED).cpu().numpy()
    ctx.set_hutchinson_terms(3)
    try:
        q3 = ctx.hutchinson(Ad, probes=m, seed=SEED).cpu().numpy()
    finally:
        ctx.set_hutchinson_terms(2)
    qo = hutchinson.quadratic_forms(A.astype(np.float64), hutchinson.probes_fast(n, m, SEED))
    s = np.abs(A.astype(np.float64)).sum()
    # per entry |da| <= 2^-22 |a| + 2^-25 / s_scale, s_scale = 2^(14 - e) with 2^e > max a_kk
    e = int(np.frexp(float(A.diagonal().max()))[1])
    floor = 2.0 ** -25 / 2.0 ** (14 - e) * n * n
    assert np.all(np.abs(q2 - qo) <= (2.0 ** -22 + 64 * 2.0 ** -24) * s + floor)
    assert np.all(np.abs(q3 - qo) <= 64 * 2.0 ** -24 * s)
    with pytest.raises(Exception):
        ctx.set_hutchinson_terms(4)


def test_fp16_range_fallback_for_matrices_beyond_the_diagonal_bound(ctx):
    # symmetric, zero diagonal, large off-diagonal entries: |a_ij| > max a_kk,
    # so the FP16 terms would overflow; the call must detect it and return
    # the three-term BF16 result
    n, m = 640, 64
    rng = np.random.default_rng(5)
    B = rng.standard_normal((n, n))
    A = ((B + B.T) * 1e3).astype(np.float32)
    np.fill_diagonal(A, 0.0)
    A[0, 0] = 1e-3
    q = ctx.hutchinson(torch.from_numpy(A).cuda(), probes=m, seed=SEED).cpu().numpy()
    qo = hutchinson.quadratic_forms(A.astype(np.float64), hutchinson.probes_fast(n, m, SEED))
    assert np.all(np.isfinite(q))
    assert np.all(np.abs(q - qo) <= 64 * 2.0 ** -24 * np.abs(A.astype(np.float64)).sum())
