"""The no-allocation gradient entry point (msp_rbf_grad_ell_static).

It serves callers that cannot allocate device memory where they need the
RBF length-scale gradient (a framework allocator owning the device, a loop
that forbids allocation after start-up). It keeps its scratch in a fixed
array inside the library; here it is called through the C ABI twice in a row
and must reproduce the allocating entry point msp_rbf_grad_ell, and it must
refuse sizes beyond its limit. This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import rbf_points

pytestmark = pytest.mark.gpu


def test_static_variant_matches_allocating_entry_point():
    from paper_2405_05865_gb300 import Context, _lib
    ctx = Context(0)
    lib = ctx.lib
    n, ell = 3001, 0.1
    P = torch.from_numpy(rbf_points(n, seed=21)).cuda()
    rng = np.random.default_rng(21)
    a = torch.from_numpy(rng.standard_normal(n)).cuda()
    x = torch.from_numpy(rng.standard_normal(n)).cuda()
    ref = float(ctx.rbf_grad_ell(P, ell, a, x))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vals = []
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.msp_rbf_grad_ell_static(ctypes.c_void_p(P.data_ptr()), n, 3, ell,
                                         ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.msp_last_error(None)
        torch.cuda.synchronize()
        vals.append(float(out))
    for v in vals:
        assert v == pytest.approx(ref, rel=1e-12, abs=0.0)
    ctx.close()


def test_static_variant_at_the_size_limit():
    # n = 8 * 65536 - 3: the last scratch slot (block 65535) holds a partial
    # block of 5 points and the final warp is ragged
    from paper_2405_05865_gb300 import Context
    ctx = Context(0)
    lib = ctx.lib
    n, ell = 8 * 65536 - 3, 0.05
    P = torch.from_numpy(rbf_points(n, seed=22)).cuda()
    rng = np.random.default_rng(22)
    a = torch.from_numpy(rng.standard_normal(n)).cuda()
    x = torch.from_numpy(rng.standard_normal(n)).cuda()
    ref = float(ctx.rbf_grad_ell(P, ell, a, x))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.msp_rbf_grad_ell_static(ctypes.c_void_p(P.data_ptr()), n, 3, ell,
                                         ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.msp_last_error(None)
        torch.cuda.synchronize()
        assert float(out) == pytest.approx(ref, rel=1e-12, abs=0.0)
    ctx.close()


def test_static_variant_rejects_oversized_input():
    from paper_2405_05865_gb300 import _lib
    lib = _lib.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.msp_rbf_grad_ell_static(p, 8 * 65536 + 1, 3, 0.1, p, p, p, None)
    assert st == 1
    assert b"exceeds the static scratch limit" in lib.msp_last_error(None)
