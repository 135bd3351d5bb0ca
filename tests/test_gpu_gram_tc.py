"""The level-2 Gram M2 = C~^T C~ + lambda~ W (Algorithm 1, step 4) on the
tensor cores, against the FP64 oracle.

The tensor-core Gram splits q C~ (q a power of two) into three FP16 terms
h + m + l and accumulates in FP32 in tensor memory: hh alone, drained every
64 rows, and hm, mh, mm, hl, lh (each at most 2^-11 of hh) together, drained
every 512 rows; the drains go into float-float (TwoSum) running sums,
written per slice in FP64 and added in FP64. Error per entry (a, b), with
v = |C~| and V = v^T v:
  dropped ml, lm, ll                     (2 * 2^-33 + 2^-44) V_ab
  hh, 64 products per drain              (64 + 2) * 2^-23 V_ab
  the small products, 2560 per drain     (2560 + 2) * 2^-23 * 2^-10 V_ab
(the recursive-summation bound with a unit error of 2^-23, which holds for
round-to-nearest and for truncating accumulation alike), plus float-float
and FP64 rounding. On data whose scaled entries fit
in 11 bits and whose sums fit in 24 bits the split is exact, m = l = 0 and
every sum is exact: M2 then equals the oracle's bit for bit.

What the preconditioner needs is that M2 - C~^T C~ = lambda~ W + (Gram
error) stays positive definite (the Woodbury form of Algorithm 1 is SPD only
then); the PSD-margin test checks that on the RBF workload.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nystrom as onys
from oracle import reference, sketch
from workloads import make_workload

pytestmark = pytest.mark.gpu

SEED = 0x4D5350


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _oracle_parts(A_used, n, s, gamma, phi, gamma_phi, lam_tilde):
    S = sketch.sparse_embedding(n, s, gamma, SEED)
    Co = sketch.sketch_C(A_used, S)
    Wo = sketch.core_W(S, Co)
    if phi:
        Cto = sketch.level2_sketch(sketch.level2_embedding(n, phi, gamma_phi, SEED), Co)
    else:
        Cto = Co
    return Cto, Wo, onys.level2_matrix(Cto, Wo, lam_tilde)


def _m2(ctx, sk, lam, lam0, phi, tc, gamma_phi=8):
    """(M2, W) of the factor, the Gram on the tensor cores or not."""
    ctx.set_gram_tensor_cores(tc)
    try:
        f = ctx.nystrom(sk, lam, lam0, phi=phi, gamma_phi=gamma_phi, seed=SEED)
        parts = f.parts()
        M2, W = parts["M2"].cpu().numpy(), parts["W"].cpu().numpy()
        f.close()
    finally:
        ctx.set_gram_tensor_cores(True)
    return M2, W


@pytest.mark.parametrize("n,s,phi", [(512, 64, 0), (1000, 200, 0), (2048, 320, 1024)])
def test_gram_tc_integer_data_bit_exact(ctx, n, s, phi):
    # A = B^T B with B in {-1, 0, 1}: integer PSD. gamma = 1 keeps C = A S^T
    # integer (scale 1) and gamma_phi = 4 makes C~ = Phi C a multiple of 1/2
    # (scale 1/2): the FP16 split and every FP32 sum are exact, so the
    # tensor-core Gram equals the oracle's exactly.
    rng = np.random.default_rng(n + s)
    B = rng.integers(-1, 2, size=(24, n)).astype(np.float64)
    A = B.T @ B
    sk = ctx.sketch(_cuda(A, torch.float32), s, 1, SEED)
    Cg = sk.C().double().cpu().numpy()
    Cto, Wo, M2o = _oracle_parts(A, n, s, 1, phi, 4, 0.25)
    assert np.array_equal(Cg, sketch.sketch_C(A, sketch.sparse_embedding(n, s, 1, SEED)))
    assert np.abs(2 * Cto).max() < 2 ** 11 and 4 * (np.abs(Cto).T @ np.abs(Cto)).max() < 2 ** 24
    M2, _ = _m2(ctx, sk, 0.25, 0.0, phi, True, gamma_phi=4)
    assert M2.shape == (s, s)
    assert np.array_equal(M2, M2o)


def _acc_coef(K):
    return 2 * 2.0 ** -33 + 2.0 ** -44 + (66 + 2562 * 2.0 ** -10) * 2.0 ** -23 + 2.0 ** -40


@pytest.mark.parametrize("n,s,phi,lam0", [(3000, 256, 0, 0.0), (2500, 384, 0, 0.05), (4096, 128, 2048, 0.0),
                                          (20000, 128, 0, 0.0)])
def test_gram_tc_matches_oracle(ctx, n, s, phi, lam0):
    # a kernel-like matrix with a decaying spectrum; n = 20000: a ragged
    # last chunk (20000 = 625 x 32) and several slices per tile pair
    rng = np.random.default_rng(n ^ s)
    G = rng.standard_normal((n, 48)) * np.logspace(0, -3, 48)
    A = G @ G.T + 1e-3 * np.eye(n)
    A_dev = _cuda(A, torch.float32)
    A_used = A_dev.double().cpu().numpy()
    lam = 1e-3
    lt = lam + lam0
    sk = ctx.sketch(A_dev, s, 8, SEED)
    M2, W = _m2(ctx, sk, lam, lam0, phi, True)
    assert np.array_equal(M2, M2.T)
    # the Gram part of the GPU's M2 against the FP64 Gram of the GPU's own
    # C~: the FP32 C from the sketch pass, Phi applied in FP32 (gamma_phi
    # terms per row, error (gamma_phi + 2) 2^-24 |Phi| |C|)
    Cg = sk.C().double().cpu().numpy()
    if phi:
        Phi = sketch.level2_embedding(n, phi, 8, SEED)
        Ctg = sketch.level2_sketch(Phi, Cg)
        Va = np.asarray(abs(Phi) @ np.abs(Cg))
        phi_err = 2 * 10 * 2.0 ** -24 * (Va.T @ Va)
    else:
        Ctg = Cg
        phi_err = 0.0
    V = np.abs(Ctg).T @ np.abs(Ctg)
    K = Ctg.shape[0]
    gram = M2 - lt * W
    err = np.abs(gram - Ctg.T @ Ctg)
    bound = _acc_coef(K) * V + phi_err + 2.0 ** -50 * np.abs(M2)
    assert np.all(err <= bound), float((err / bound).max())
    # typical accuracy far inside the worst case (and near the FP32 unit)
    assert np.median(err / V) < 2.0 ** -24
    # end to end against the FP64 oracle: the size of the FP32 sketch rounding
    Cto, Wo, M2o = _oracle_parts(A_used, n, s, 8, phi, 8, lt)
    assert np.abs(M2 - M2o).max() <= 4 * (K + 64) * 2.0 ** -24 * np.abs(M2o).max()


def test_gram_tc_agrees_with_fp32_pipe(ctx):
    # the two Gram paths of the factor give the same M2 to the accuracy of
    # the tensor-core one (the FP32-pipe Gram uses compensated sums)
    n, s = 6000, 512
    rng = np.random.default_rng(5)
    G = rng.standard_normal((n, 96)) / np.sqrt(n)
    A = G @ G.T + 0.01 * np.eye(n)
    sk = ctx.sketch(_cuda(A, torch.float32), s, 8, SEED)
    tc, _ = _m2(ctx, sk, 1e-2, 0.0, 0, True)
    simt, _ = _m2(ctx, sk, 1e-2, 0.0, 0, False)
    Cg = sk.C().double().cpu().numpy()
    V = np.abs(Cg).T @ np.abs(Cg)
    d = np.abs(tc - simt)
    assert np.all(d <= (_acc_coef(n) + 2.0 ** -40) * V + 2.0 ** -50 * np.abs(simt))
    assert not np.array_equal(tc, simt)      # two different paths ran


def test_gram_tc_power_of_two_scale_invariance(ctx):
    # q follows max |C~| by a power of two: scaling A by 2^k scales M2's Gram
    # part by exactly 4^k (lambda~ scaled by 2^k keeps M2 = 4^k M2)
    n, s = 2000, 256
    rng = np.random.default_rng(9)
    G = rng.standard_normal((n, 40))
    A = G @ G.T / n + 0.1 * np.eye(n)
    base = None
    for k in (0, 7, -9):
        sk = ctx.sketch(_cuda(A * 2.0 ** k, torch.float32), s, 8, SEED)
        M2, _ = _m2(ctx, sk, 0.1 * 2.0 ** k, 0.0, 0, True)
        if base is None:
            base = M2
        else:
            assert np.array_equal(M2, base * 4.0 ** k)


def test_gram_tc_keeps_the_preconditioner_spd_margin(ctx):
    # M2 - C^T C = lambda~ W + E: its smallest eigenvalue stays within a few
    # percent of lambda~ lambda_min(W) (a Gram error E of FP32-GEMM size,
    # ~2^-17 V here, makes it negative on this workload)
    w = make_workload("rbf", seed=1, n=8192)
    s = max(128, w.s)
    sk = ctx.sketch(_cuda(w.A, torch.float32), s, 8, SEED)
    Cg = sk.C().double().cpu().numpy()
    M2, W = _m2(ctx, sk, w.lam, 0.0, 0, True)
    lw = np.linalg.eigvalsh(w.lam * W).min()
    assert lw > 0
    assert np.linalg.eigvalsh(M2 - Cg.T @ Cg).min() >= 0.9 * lw


@pytest.mark.parametrize("n", [3000, 8192])
def test_solve_with_tc_gram_matches_fp32_pipe_iterations(ctx, n):
    # the preconditioner built on either Gram path gives the same solve
    w = make_workload("rbf", seed=1, n=n)
    A_dev = _cuda(w.A, torch.float32)
    A_used = A_dev.double().cpu().numpy()
    s = max(128, w.s)
    its = []
    for tc in (True, False):
        ctx.set_gram_tensor_cores(tc)
        try:
            sk = ctx.sketch(A_dev, s, 8, SEED)
            f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
            x, info = ctx.solve(f, A_dev, torch.as_tensor(w.b).cuda(), w.lam, precision="mixed", tol=1e-10)
            its.append(info["outer_iters"])
            xh = x.cpu().numpy()
            assert reference.rel_residual(A_used, xh, w.b, w.lam) <= 1.2e-10
            f.close()
        finally:
            ctx.set_gram_tensor_cores(True)
    # the two Gram roundings steer the FP32 recurrences apart by a few steps
    # over hundreds of iterations (refinement restarts included)
    assert abs(its[0] - its[1]) <= max(2, 0.02 * its[1]), its
