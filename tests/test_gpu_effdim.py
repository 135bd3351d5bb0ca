"""Effective dimension d_lambda = tr(A (A + lam I)^{-1}) through
msp_effective_dimension against the FP64 oracle.

* per probe, the device value n - lam g^T x against the oracle's value on the
  same Rademacher probes and the same (FP32-rounded) matrix, within the bound
  the solve's backward error gives: with r = g - (A + lam I) x,
  |lam g^T (x - x*)| <= |g| |r| and |r| <= tol ((L + lam) |x| + |g|);
* the estimate within 5 standard errors of the closed form
  sum_i sigma_i / (sigma_i + lam) over the eigenvalues of that matrix;
* a probe count that is not a multiple of 16 (a ragged last instance).

The system is the kernel ridge regression one d_lambda is defined for
(Section 3): an RBF kernel matrix, n = 2048, length scale 0.2, lam = 1e-2
(d_lambda ~ 323), sketch size s = 768.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import effdim, hutchinson, reference

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def system():
    _, A32, _ = workloads.batch_instance(workloads.BatchSpec(2048, 0.2, 1e-2, 768, 1, 7))
    A64 = A32.astype(np.float64)
    return A32, A64, np.linalg.eigvalsh(A64), reference.norm_lower_bound(A64)


@pytest.mark.parametrize("m,seed", [(64, 11), (40, 12)])
def test_effective_dimension(ctx, system, m, seed):
    A32, A64, eig, L = system
    n, lam = A32.shape[0], 1e-2
    A = torch.from_numpy(A32).cuda()
    est, se, q = ctx.effective_dimension(A, lam, s=768, probes=m, seed=seed, tol=TOL, refine_tol=1e-6,
                                         criterion="backward")
    q = q.cpu().numpy()
    G = hutchinson.probes(n, m, seed)
    X = reference.solve_dense(A64, G, lam)
    ref = n - lam * np.einsum("ij,ij->j", G, X)
    for j in range(m):
        bound = np.sqrt(n) * TOL * ((L + lam) * np.linalg.norm(X[:, j]) + np.sqrt(n))
        assert abs(q[j] - ref[j]) <= 1.01 * bound, (j, q[j], ref[j], bound)
    o_est, o_se = effdim.estimate(A64, lam, G)
    assert est == pytest.approx(float(q.mean()), rel=1e-14)
    assert se == pytest.approx(float(q.std(ddof=1) / np.sqrt(m)), rel=1e-10)
    assert abs(est - o_est) <= 1e-6 * o_est
    assert se == pytest.approx(o_se, rel=1e-3)
    exact = reference.effective_dimension(eig, lam)
    assert abs(est - exact) <= 5 * se


def test_effective_dimension_bad_arguments(ctx, system):
    A = torch.from_numpy(system[0]).cuda()
    with pytest.raises(Exception):
        ctx.effective_dimension(A, 0.0, s=256, probes=16)
    with pytest.raises(Exception):
        ctx.effective_dimension(A, 1e-2, s=256, probes=1)


def test_auto_params_then_solve(ctx, system):
    """msp_auto_params: the estimate is within 5 standard errors of the
    closed form, the chosen (l, s, lambda0) are the oracle's rule applied to
    that estimate, and the system solves with them to backward error 1e-10."""
    A32, A64, eig, L = system
    n, lam = A32.shape[0], 1e-2
    A = torch.from_numpy(A32).cuda()
    p = ctx.auto_params(A, lam, probes=64, seed=5, tol=TOL, refine_tol=1e-6, criterion="backward")
    exact = reference.effective_dimension(eig, lam)
    assert abs(p["d_lambda"] - exact) <= 5 * p["d_std_err"]
    want = effdim.params_from_effdim(min(float(n), max(0.0, p["d_lambda"])), n, lam)
    for key in ("l", "s", "capped", "direct"):
        assert p[key] == want[key], key
    assert p["lambda0"] == want["lambda0"]
    assert 0.0 < p["lambda0"] <= lam and not p["capped"]
    b = np.random.default_rng(9).standard_normal(n)
    sk = ctx.sketch(A, s=p["s"])
    f = ctx.nystrom(sk, lam=lam, lam0=p["lambda0"], phi=0)
    x, info = ctx.solve(f, A, torch.from_numpy(b).cuda(), lam=lam, max_inner=0, criterion="backward", tol=TOL)
    f.close()
    sk.close()
    x = x.cpu().numpy()
    r = b - (A64 @ x + lam * x)
    assert info["status"] == 0
    assert np.linalg.norm(r) <= TOL * ((L + lam) * np.linalg.norm(x) + np.linalg.norm(b))
