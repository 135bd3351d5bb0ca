"""The error convention of the C ABI, checked without a GPU: every entry
point that returns a status answers a NULL context or handle (and zero
sizes) with MSP_EINVAL and a message in msp_last_error(NULL), before it
touches a device; nothing aborts, traps or prints. Without a CUDA device,
msp_create refuses cleanly."""

import ctypes

import pytest

from paper_2405_05865_gb300 import _lib

MSP_EINVAL = 1


def _zero(t):
    if t is None:
        return None
    if isinstance(t, type) and issubclass(t, ctypes._Pointer):
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p):
        return None
    if t in (ctypes.c_double, ctypes.c_float):
        return t(0.0)
    if isinstance(t, type) and issubclass(t, ctypes.Structure):
        return t()
    return t(0)


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_null_context_or_handle_is_einval(lib):
    checked = 0
    for name, (res, args) in sorted(_lib._SIGS.items()):
        if res is not ctypes.c_int or not args:
            continue
        rc = getattr(lib, name)(*[_zero(a) for a in args])
        assert rc == MSP_EINVAL, (name, rc)
        msg = lib.msp_last_error(None)
        assert msg and len(msg) > 3, name
        checked += 1
    assert checked >= 40


def test_create_without_a_device_refuses_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    ctx = ctypes.c_void_p()
    rc = lib.msp_create(ctypes.byref(ctx), 0, None)
    assert rc == MSP_EINVAL and not ctx.value
    assert b"no CUDA device" in lib.msp_last_error(None)
    # the destroy functions take NULL
    lib.msp_destroy(None)
    lib.msp_sketch_destroy(None)
    lib.msp_factor_destroy(None)
