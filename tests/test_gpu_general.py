"""Three-level MSP for (A^T A + lam I) x = c on the GPU against the FP64
oracle (Algorithms 3-5).

Inputs: A = U diag(sigma) V^T with 8 outlier singular values log-spaced
1e2 -> 1e1 over a flat tail in [0.5, 1] (the "few large singular values"
shape of Section 3), rounded once to FP32; the oracle works on the same FP32
values in FP64. lambda0 = (2/l) sum_{i>l} sigma_i^2 with l = 16 (Theorem 3.1).

Tolerances (u = 2^-24):
* A~ = A S^T element by element within (gamma + 1) u (|A| |S|^T), the
  rounding of the FP32 sum of gamma signed terms;
* M3a, M3b (FP64 Grams of the device A^) against the oracle's within
  8 u |M3|_F (A^ differs from the oracle's by FP32 rounding);
* one SolveM2 with t3 steps against the oracle's with the same t3: the FP32
  level-3 iterates carry relative rounding of a few u, amplified by the
  cancellation in (u - v) / lam~ by 1 + |W| / lam~; bound 4 u (1 + |W|/lam~)
  per unit norm (a CPU FP32 simulation of the same steps lands 80x inside);
* one SolveM1 likewise, with the second cancellation of
  w = (r - A^T A~ y) / lam~ (factor 1 + |A|^2 / lam~);
* the full mixed-precision solve: |c - (A^T A + lam I) x| <= 1e-10 |c|
  recomputed here in FP64, and |x - x*| <= |r| / (sigma_min^2 + lam).
"""

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import general, sketch
from workloads import householder_spectrum, svd_matrix

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
LAM = 1e-3


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _problem(m, n, seed):
    sig = householder_spectrum(n, 8, seed, hi=1e2, lo=1e1)
    A32 = svd_matrix(m, n, sig, seed + 1).astype(np.float32)
    lam0 = 2.0 / 16 * float(np.sum(sig[16:] ** 2))
    return A32, sig, lam0


CASES = [(3000, 256, 128, 4), (2001, 203, 100, 7)]   # aligned; odd n (padded copy), ragged s


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"m{c[0]}n{c[1]}s{c[2]}")
def system(request, ctx):
    m, n, s, seed = request.param
    A32, sig, lam0 = _problem(m, n, seed)
    A = torch.from_numpy(A32).cuda()
    g = ctx.general(A, LAM, s, lam0=lam0)
    p = general.GenParams(s=s, lam0=lam0)
    st = general.setup(A32.astype(np.float64), LAM, p)
    yield A32, sig, lam0, g, p, st
    g.close()


def test_setup_matches_oracle(system):
    A32, sig, lam0, g, p, st = system
    got = g.setup(p.s)
    At = got["At"].cpu().numpy().astype(np.float64)
    S = sketch.sparse_embedding(A32.shape[1], p.s, p.gamma, p.seed)
    bound = (p.gamma + 1) * U32 * np.asarray((abs(S) @ np.abs(A32.astype(np.float64)).T).T)
    assert np.all(np.abs(At - st.At) <= bound + 1e-30)
    # A^ = Phi A~ inherits the bound on A~ through |Phi|, plus the FP32
    # rounding of its own gamma_phi-term sums; the Gram then moves by at most
    # 2 |A^|_2 |dA^|_F + |dA^|_F^2 (its FP64 accumulation adds far less)
    Phi = sketch.level2_embedding(A32.shape[0], p.phi or 4 * p.s, p.gamma_phi, p.seed)
    dAh = np.asarray(abs(Phi) @ bound) + (p.gamma_phi + 1) * U32 * np.asarray(abs(Phi) @ np.abs(st.At))
    eps = float(np.linalg.norm(dAh))
    gram_bound = 2 * np.linalg.norm(st.Ah, 2) * eps + eps ** 2
    for key, L in (("M3a", st.L3a), ("M3b", st.L3b)):
        ref = L @ L.T
        dev = got[key].cpu().numpy()
        assert np.linalg.norm(dev - ref) <= gram_bound + 1e-13 * np.linalg.norm(ref), key
    assert g.lambda_tilde == pytest.approx(LAM + lam0, rel=1e-15)


@pytest.mark.parametrize("t3", [1, 8])
def test_solve_m2_matches_oracle(system, t3):
    A32, sig, lam0, g, p, st = system
    r = np.random.default_rng(11).standard_normal(p.s).astype(np.float32)
    z = g.solve_m2(torch.from_numpy(r).cuda(), t3).cpu().numpy().astype(np.float64)
    ref = general.solve_m2(st, r.astype(np.float64), general.GenParams(s=p.s, lam0=lam0, t3=t3))
    W = st.At.T @ st.At
    amp = 1.0 + np.linalg.eigvalsh(W)[-1] / st.lam_tilde
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= 4 * U32 * amp, (err, 4 * U32 * amp)


def test_solve_m1_matches_oracle(system):
    A32, sig, lam0, g, p, st = system
    n = A32.shape[1]
    r = np.random.default_rng(12).standard_normal(n).astype(np.float32)
    w = g.solve_m1(torch.from_numpy(r).cuda(), 4, 6).cpu().numpy().astype(np.float64)
    ref = general.solve_m1(st, r.astype(np.float64), general.GenParams(s=p.s, lam0=lam0, t2=4, t3=6))
    W = st.At.T @ st.At
    amp = (1.0 + np.linalg.eigvalsh(W)[-1] / st.lam_tilde) * (1.0 + sig[0] ** 2 / st.lam_tilde)
    err = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    assert err <= 4 * U32 * amp, (err, 4 * U32 * amp)


def test_solve_m2_direct_matches_exact(system):
    """level3_iters = 0: M2^{-1} = (W^{-1} - (W + lam~ I)^{-1}) / lam~ applied
    exactly, against the oracle's dense solve with W^2 + lam~ W."""
    A32, sig, lam0, g, p, st = system
    r = np.random.default_rng(17).standard_normal(p.s).astype(np.float32)
    z = g.solve_m2(torch.from_numpy(r).cuda(), 0).cpu().numpy().astype(np.float64)
    ref = general.solve_m2(st, r.astype(np.float64), general.GenParams(s=p.s, lam0=lam0, level3="exact"))
    W = st.At.T @ st.At
    amp = 1.0 + np.linalg.eigvalsh(W)[-1] / st.lam_tilde
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= 4 * U32 * amp, (err, 4 * U32 * amp)


def test_solve_m1_direct_matches_exact(system):
    """level2_iters = 0: C = A^T A~ formed, M^{-1} r by the Woodbury form with
    (C^T C + lam~ W)^{-1}, against the oracle's exact level 2."""
    A32, sig, lam0, g, p, st = system
    n = A32.shape[1]
    r = np.random.default_rng(18).standard_normal(n).astype(np.float32)
    w = g.solve_m1(torch.from_numpy(r).cuda(), 0, 0).cpu().numpy().astype(np.float64)
    ref = general.solve_m1(st, r.astype(np.float64), general.GenParams(s=p.s, lam0=lam0, level2="exact"))
    W = st.At.T @ st.At
    amp = (1.0 + np.linalg.eigvalsh(W)[-1] / st.lam_tilde) * (1.0 + sig[0] ** 2 / st.lam_tilde)
    err = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    assert err <= 4 * U32 * amp, (err, 4 * U32 * amp)


@pytest.mark.parametrize("t2,t3", [(8, 0), (0, 0)])
def test_full_solve_direct_modes(system, t2, t3):
    A32, sig, lam0, g, p, st = system
    A64 = A32.astype(np.float64)
    n = A32.shape[1]
    c = np.random.default_rng(19).standard_normal(n)
    x, info = g.solve(torch.from_numpy(c).cuda(), tol=1e-10, refine_tol=1e-3, level2_iters=t2, level3_iters=t3)
    x = x.cpu().numpy()
    r = c - (A64.T @ (A64 @ x) + LAM * x)
    assert info["status"] == 0
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c)


def test_matvec64(system):
    A32, sig, lam0, g, p, st = system
    A64 = A32.astype(np.float64)
    x = np.random.default_rng(13).standard_normal(A32.shape[1])
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = A64.T @ (A64 @ x) + LAM * x
    # FP64 accumulation of m + n terms per entry
    bound = 4 * (A32.shape[0] + A32.shape[1]) * 2.0 ** -53 * (np.abs(A64).T @ (np.abs(A64) @ np.abs(x)))
    assert np.all(np.abs(y - ref) <= bound + LAM * np.abs(x) * 2.0 ** -52)


def test_op_fp32(system):
    A32, sig, lam0, g, p, st = system
    A64 = A32.astype(np.float64)
    x = np.random.default_rng(16).standard_normal(A32.shape[1]).astype(np.float32)
    y = g.op(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    ref = A64.T @ (A64 @ x64) + LAM * x64
    # FP32: row dots of n terms, then sums of m products (the partials per
    # CTA in FP32, combined in FP64), each entry within (n + m) u |A|^T (|A| |x|)
    m, n = A32.shape
    bound = (n + m) * U32 * (np.abs(A64).T @ (np.abs(A64) @ np.abs(x64))) + 4 * U32 * LAM * np.abs(x64)
    assert np.all(np.abs(y - ref) <= bound)


def test_full_solve_reaches_tolerance(system):
    A32, sig, lam0, g, p, st = system
    A64 = A32.astype(np.float64)
    n = A32.shape[1]
    c = np.random.default_rng(14).standard_normal(n)
    x, info = g.solve(torch.from_numpy(c).cuda(), tol=1e-10, refine_tol=1e-3)
    x = x.cpu().numpy()
    r = c - (A64.T @ (A64 @ x) + LAM * x)
    assert info["status"] == 0
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c)
    assert abs(info["rel_resid"] - np.linalg.norm(r) / np.linalg.norm(c)) <= 1e-12
    xs = np.linalg.solve(A64.T @ A64 + LAM * np.eye(n), c)
    lmin = np.linalg.svd(A64, compute_uv=False)[-1] ** 2 + LAM
    assert np.linalg.norm(x - xs) <= 1.01 * np.linalg.norm(r) / lmin + 1e-12 * np.linalg.norm(xs)
    assert info["outer_iters"] >= 1 and info["refine_steps"] >= 1


def test_fp32_solve_and_zero_rhs(system):
    A32, sig, lam0, g, p, st = system
    n = A32.shape[1]
    c = np.random.default_rng(15).standard_normal(n)
    x, info = g.solve(torch.from_numpy(c).cuda(), tol=1e-4, precision="fp32")
    # the FP32 recurrence residual meets tol; the true residual can differ by
    # the FP32 rounding of the operator, about u kappa(A^T A + lam I)
    kappa = (sig[0] ** 2 + LAM) / (np.min(sig) ** 2 + LAM)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-4 + 4 * U32 * kappa
    x0, info0 = g.solve(torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert info0["status"] == 0 and not torch.any(x0)


def test_bad_arguments(ctx):
    from paper_2405_05865_gb300 import MspError
    A = torch.zeros((100, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(MspError):
        ctx.general(A, 0.0, 16, lam0=0.0)            # lambda~ = 0
    with pytest.raises(MspError):
        ctx.general(A.t().contiguous(), 1e-2, 16)    # m < n
    with pytest.raises(MspError):
        ctx.general(A, 1e-2, 64)                     # s > n
    A2 = torch.randn((200, 40), dtype=torch.float32, device="cuda")
    g = ctx.general(A2, 1e-2, 16)
    with pytest.raises(MspError):
        g.solve(torch.ones(40, dtype=torch.float64, device="cuda"), level2_iters=-1)
    with pytest.raises(MspError):
        g.solve(torch.ones(40, dtype=torch.float64, device="cuda"), criterion="backward")
    g.close()
