"""Two-level Multi-level Sketched Preconditioning (MSP) on one GB300 (sm_103a).

The hot path is the CUDA library ``lib/libmsp.so`` (C ABI in include/msp.h),
built by ``python -m paper_2405_05865_gb300.build``. ``api`` is the Python
layer over it (PyTorch supplies device memory and streams). There is no CPU
or PyTorch fallback: without the built library or a CUDA device the API
raises.
"""

__all__ = ["Context", "Sketch", "Factor", "Batch", "General", "LeastSquares", "DEFAULT_SEED", "MspError", "params_from_effdim"]


def __getattr__(name):
    if name in ("Context", "Sketch", "Factor", "Batch", "General", "LeastSquares", "DEFAULT_SEED", "params_from_effdim"):
        from . import api
        return getattr(api, name)
    if name == "MspError":
        from ._lib import MspError
        return MspError
    raise AttributeError(name)
