"""The Cholesky inverse of M2 + nu I (Algorithm 1, step 4) of an FP32 sketch
in float-float arithmetic, against the FP64 factorisation and the oracle.

The factor's inverse X = L^{-1} of a computed Cholesky factor of
M = M2 + nu I satisfies |X M X^T - I|_2 <= c s u kappa(M) for a unit
roundoff u; float-float has u about 2^-46 (FP64: 2^-53), so the test
allows s 2^-40 kappa(M) (a margin of 2^6 over the unit). The shift nu =
2^-24 |M2|_F is the same on both paths (the FP32 data needs it), and the
solves built on either factor reach the tolerance asked for.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nystrom as onys
from oracle import reference
from workloads import make_workload

pytestmark = pytest.mark.gpu

SEED = 0x4D5350


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_05865_gb300 import Context
    c = Context(0)
    yield c
    c.set_factor_float_float(True)
    c.close()


def _cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _factor(ctx, sk, lam, lam0, phi, ff):
    ctx.set_factor_float_float(ff)
    try:
        f = ctx.nystrom(sk, lam, lam0, phi=phi, seed=SEED)
        p = f.parts()
        out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in p.items()}
        f.close()
    finally:
        ctx.set_factor_float_float(True)
    return out


def _inverse_residual(p, s):
    M = p["M2"][:s, :s] + p["shift"] * np.eye(s)
    X = np.tril(p["Linv"][:s, :s])
    E = X @ M @ X.T - np.eye(s)
    ev = np.linalg.eigvalsh(M)
    return np.linalg.norm(E, 2), ev.max() / ev.min()


@pytest.mark.parametrize("work,n,s,phi", [("rbf", 2048, 256, 0), ("rbf", 5000, 640, 0), ("rbf", 3000, 128, 1024),
                                          ("outlier", 1024, 64, 0)])
def test_ff_inverse_meets_the_unit_bound(ctx, work, n, s, phi):
    w = make_workload(work, seed=3, n=n) if work == "rbf" else make_workload(work, seed=0)
    lam0 = onys.lambda0_from_spectrum(w.sigma, 32) if work == "outlier" else 0.0
    sk = ctx.sketch(_cuda(w.A, torch.float32), s, 8, SEED)
    pf = _factor(ctx, sk, w.lam, lam0, phi, True)
    pd = _factor(ctx, sk, w.lam, lam0, phi, False)
    sk.close()
    # the same M2 and shift on both paths (the Gram is not part of the change)
    assert np.array_equal(pf["M2"], pd["M2"]) and pf["shift"] == pd["shift"] > 0
    ef, kappa = _inverse_residual(pf, s)
    ed, _ = _inverse_residual(pd, s)
    assert ef <= s * 2.0 ** -40 * kappa, (ef, kappa)
    assert ed <= s * 2.0 ** -44 * kappa, (ed, kappa)
    # the two inverses agree to the float-float bound, entry by entry relative
    # to the size of L^{-1}
    Xf, Xd = np.tril(pf["Linv"][:s, :s]), np.tril(pd["Linv"][:s, :s])
    assert np.abs(Xf - Xd).max() <= s * 2.0 ** -40 * kappa * np.abs(Xd).max()
    assert not np.array_equal(Xf, Xd)          # two different paths ran


def test_ff_power_of_four_scaling_is_exact(ctx):
    # M2 scaled by 4^k (A by 2^k) gives L^{-1} scaled by exactly 2^-k: the
    # float-float path scales M to |M|_F in [1, 4) by a power of four first
    w = make_workload("rbf", seed=5, n=1500)
    base = None
    for k in (0, 6, -5):
        sk = ctx.sketch(_cuda(w.A * 2.0 ** k, torch.float32), 128, 8, SEED)
        p = _factor(ctx, sk, w.lam * 2.0 ** k, 0.0, 0, True)
        sk.close()
        if base is None:
            base = p["Linv"]
        else:
            assert np.array_equal(p["Linv"], base * 2.0 ** -k)


@pytest.mark.parametrize("n", [3000, 8192])
def test_solves_on_either_factor_agree(ctx, n):
    w = make_workload("rbf", seed=1, n=n)
    A_dev = _cuda(w.A, torch.float32)
    A_used = A_dev.double().cpu().numpy()
    s = max(128, w.s)
    its = []
    for ff in (True, False):
        ctx.set_factor_float_float(ff)
        try:
            sk = ctx.sketch(A_dev, s, 8, SEED)
            f = ctx.nystrom(sk, w.lam, 0.0, phi=0)
            x, info = ctx.solve(f, A_dev, torch.as_tensor(w.b).cuda(), w.lam, precision="mixed", tol=1e-10)
            assert reference.rel_residual(A_used, x.cpu().numpy(), w.b, w.lam) <= 1.2e-10
            its.append(info["outer_iters"])
            f.close()
            sk.close()
        finally:
            ctx.set_factor_float_float(True)
    assert abs(its[0] - its[1]) <= max(2, 0.02 * its[1]), its
