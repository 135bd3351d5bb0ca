"""Schatten-p (p in (0, 2)) from ridge solves through msp_schatten_p against
the FP64 oracle (same quadrature nodes, same Rademacher probes).

* per probe, the device estimate X_k against the oracle's (dense FP64 solves
  of the same systems on the same FP32-rounded matrix): every ridge solve
  stops at relative residual 1e-10 in FP64, so each d_t term is within
  n t |g|^2 1e-10 / (sigma_min^2 + t) of the oracle's; summed with the
  quadrature weights that is far below 1e-6 X_k -- asserted at 1e-6;
* the estimate within 5 standard errors of the exact sum sigma_i^p;
* the shift z I on a square matrix: the estimate of |A + zI|_p^p.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hutchinson, schatten
from workloads import householder_spectrum, svd_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("p", [0.6, 1.0, 1.4])
def test_schatten_p_matches_oracle(ctx, p):
    m, n = 600, 128
    sig = householder_spectrum(n, 6, 5, hi=1e2, lo=1e1)
    A32 = svd_matrix(m, n, sig, 6).astype(np.float32)
    A64 = A32.astype(np.float64)
    sv = np.linalg.svd(A64, compute_uv=False)
    t0, t1 = 1e-4 * sv.min() ** 2, 1e4 * sv.max() ** 2
    nodes, probes = 24, 12
    est, se, X = ctx.schatten_p(torch.from_numpy(A32).cuda(), p, t0, t1, nodes=nodes, probes=probes, s=32,
                                tol=1e-10, refine_tol=1e-4, level2_iters=0, level3_iters=0)
    G = hutchinson.probes(n, probes, 0x4D5350)
    o_est, o_se, o_X = schatten.estimate(A64, p, t0, t1, nodes, G)
    assert np.allclose(X, o_X, rtol=1e-6, atol=0)
    assert est == pytest.approx(o_est, rel=1e-6)
    ex = float(np.sum(sv ** p))
    assert abs(est - ex) <= 5 * se


def test_schatten_p_three_level_solves(ctx):
    m, n = 600, 128
    sig = householder_spectrum(n, 6, 5, hi=1e2, lo=1e1)
    A32 = svd_matrix(m, n, sig, 6).astype(np.float32)
    sv = np.linalg.svd(A32.astype(np.float64), compute_uv=False)
    t0, t1 = 1e-4 * sv.min() ** 2, 1e4 * sv.max() ** 2
    est, se, X = ctx.schatten_p(torch.from_numpy(A32).cuda(), 1.0, t0, t1, nodes=16, probes=6, s=32,
                                tol=1e-8, refine_tol=1e-3)
    G = hutchinson.probes(n, 6, 0x4D5350)
    _, _, o_X = schatten.estimate(A32.astype(np.float64), 1.0, t0, t1, 16, G)
    assert np.allclose(X, o_X, rtol=1e-5, atol=0)


def test_schatten_p_shift(ctx):
    n = 160
    rng = np.random.default_rng(4)
    A32 = rng.standard_normal((n, n)).astype(np.float32)
    z = 0.8
    sv = np.linalg.svd(A32.astype(np.float64) + z * np.eye(n), compute_uv=False)
    t0, t1 = 1e-4 * sv.min() ** 2, 1e4 * sv.max() ** 2
    est, se, X = ctx.schatten_p(torch.from_numpy(A32).cuda(), 1.0, t0, t1, nodes=24, probes=8, s=32, z=z,
                                tol=1e-10, refine_tol=1e-4, level2_iters=0, level3_iters=0)
    G = hutchinson.probes(n, 8, 0x4D5350)
    _, _, o_X = schatten.estimate(A32.astype(np.float64), 1.0, t0, t1, 24, G, z=z)
    # the device adds z to the FP32 diagonal (one rounding per diagonal entry)
    assert np.allclose(X, o_X, rtol=1e-5, atol=0)


def test_schatten_p_bad_arguments(ctx):
    from paper_2405_05865_gb300 import MspError
    A = torch.randn((100, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(MspError):
        ctx.schatten_p(A, 2.0, 1e-3, 1e3)
    with pytest.raises(MspError):
        ctx.schatten_p(A, 1.0, 1e-3, 1e3, z=0.5)      # shift needs a square A
    with pytest.raises(MspError):
        ctx.schatten_p(A, 1.0, 1e3, 1e-3)
