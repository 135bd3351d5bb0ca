"""ctypes binding of libmsp (include/msp.h): argument marshalling only.

Every array argument is passed as a raw pointer; every computation happens in
the library's CUDA kernels. Loading fails loudly if the shared library has not
been built (``python -m paper_2405_05865_gb300.build``); there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmsp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "msp.h")

MSP_F64, MSP_F32, MSP_BF16 = 0, 1, 2
MSP_PREC_FP64, MSP_PREC_FP32, MSP_PREC_MIXED = 0, 1, 2
MSP_STOP_RESIDUAL, MSP_STOP_BACKWARD = 0, 1
STATUS = {0: "MSP_OK", 1: "MSP_EINVAL", 2: "MSP_ENOMEM", 3: "MSP_ECUDA", 4: "MSP_ENOTPD",
          5: "MSP_ENOCONV", 6: "MSP_ENONFINITE", 7: "MSP_ETIMEOUT"}


class MspOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_outer", C.c_int), ("max_refine", C.c_int),
                ("refine_tol", C.c_double), ("inner_tol", C.c_double), ("max_inner", C.c_int),
                ("precision", C.c_int), ("check_every", C.c_int), ("profile", C.c_int),
                ("criterion", C.c_int), ("level2_iters", C.c_int), ("level3_iters", C.c_int)]


class MspInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters", C.c_int), ("refine_steps", C.c_int),
                ("shift_retries", C.c_int), ("rel_resid", C.c_double),
                ("lambda_tilde", C.c_double), ("shift", C.c_double), ("status", C.c_int),
                ("gemv_launches", C.c_int), ("level2_launches", C.c_int), ("resid_launches", C.c_int),
                ("level1_graph_iters", C.c_int), ("gemv_ms", C.c_double), ("level2_ms", C.c_double),
                ("resid_ms", C.c_double), ("backward_err", C.c_double), ("norm_lb", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class MspInstance(C.Structure):
    """One instance of a batch (msp_instance)."""
    _fields_ = [("A", C.c_void_p), ("n", C.c_int64), ("lda", C.c_int64), ("lam", C.c_double),
                ("lam0", C.c_double), ("B", C.c_void_p), ("ldb", C.c_int64), ("X", C.c_void_p),
                ("ldx", C.c_int64), ("m", C.c_int), ("gamma", C.c_int), ("s", C.c_int64),
                ("phi", C.c_int64), ("gamma_phi", C.c_int), ("pad_", C.c_int), ("seed", C.c_uint64)]


class MspAutoParams(C.Structure):
    """Sketch size and shift chosen from d_lambda (msp_auto_params)."""
    _fields_ = [("d_lambda", C.c_double), ("d_std_err", C.c_double), ("l", C.c_int64), ("s", C.c_int64),
                ("lambda0", C.c_double), ("capped", C.c_int), ("direct", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class MspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


P = C.c_void_p
I64 = C.c_int64
_SIGS = {
    "msp_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
    "msp_destroy": (None, [P]),
    "msp_last_error": (C.c_char_p, [P]),
    "msp_default_opts": (None, [C.POINTER(MspOpts)]),
    "msp_version": (C.c_char_p, []),
    "msp_launch_count": (C.c_int64, [P]),
    "msp_sketch_pattern": (C.c_int, [P, I64, I64, C.c_int, C.c_uint64, C.c_int, P, P]),
    "msp_sketch": (C.c_int, [P, P, C.c_int, I64, I64, I64, C.c_int, C.c_uint64, C.POINTER(P)]),
    "msp_sketch_destroy": (None, [P]),
    "msp_sketch_info": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64),
                                  C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "msp_sketch_get_C": (C.c_int, [P, P, P, I64]),
    "msp_nystrom": (C.c_int, [P, P, C.c_double, C.c_double, I64, C.c_int, C.c_uint64,
                              C.POINTER(P)]),
    "msp_nystrom_ex": (C.c_int, [P, P, C.c_double, C.c_double, I64, C.c_int, C.c_uint64, C.c_int,
                                 C.POINTER(P)]),
    "msp_factor_destroy": (None, [P]),
    "msp_factor_get": (C.c_int, [P, P, P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_int)]),
    "msp_solve_m1": (C.c_int, [P, P, P, P, C.POINTER(MspOpts), C.POINTER(C.c_int)]),
    "msp_solve": (C.c_int, [P, P, P, C.c_int, I64, I64, C.c_double, P, P, C.POINTER(MspOpts),
                            C.POINTER(MspInfo)]),
    "msp_set_grid_wait_limit": (C.c_int, [P, C.c_double]),
    "msp_set_gram_tensor_cores": (C.c_int, [P, C.c_int]),
    "msp_set_level1_graphs": (C.c_int, [P, C.c_int]),
    "msp_set_factor_float_float": (C.c_int, [P, C.c_int]),
    "msp_set_sketch_one_pass": (C.c_int, [P, C.c_int]),
    "msp_solve_refined": (C.c_int, [P, P, P, C.c_int, I64, I64, P, C.c_int, I64, C.c_double, P, P,
                                    C.POINTER(MspOpts), C.POINTER(MspInfo)]),
    "msp_solve_full": (C.c_int, [P, P, C.c_int, I64, I64, C.c_double, P, P, I64, C.c_int,
                                 C.c_double, I64, C.c_int, C.c_uint64, C.POINTER(MspOpts),
                                 C.POINTER(MspInfo)]),
    "msp_matvec_f64": (C.c_int, [P, P, C.c_int, I64, I64, C.c_double, P, P]),
    "msp_dot": (C.c_int, [P, P, P, I64, C.c_double, P]),
    "msp_params_from_effdim": (C.c_int, [C.c_double, I64, C.c_double, C.POINTER(MspAutoParams)]),
    "msp_auto_params": (C.c_int, [P, P, I64, I64, C.c_double, I64, C.c_uint64, C.c_int, C.POINTER(MspOpts),
                                  C.POINTER(MspAutoParams)]),
    "msp_effective_dimension": (C.c_int, [P, P, I64, I64, C.c_double, I64, C.c_uint64, I64, C.c_int,
                                          C.POINTER(MspOpts), C.POINTER(C.c_double), C.POINTER(C.c_double), P]),
    "msp_norm_lower_bound": (C.c_int, [P, P, C.c_int, I64, I64, C.POINTER(C.c_double)]),
    "msp_general_create": (C.c_int, [P, P, I64, I64, I64, C.c_double, C.c_double, I64, C.c_int, I64, C.c_int,
                                     C.c_uint64, C.POINTER(P)]),
    "msp_general_destroy": (None, [P]),
    "msp_general_info": (C.c_int, [P, C.POINTER(I64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
    "msp_general_get": (C.c_int, [P, P, P, I64, P, P]),
    "msp_general_solve": (C.c_int, [P, P, P, P, C.POINTER(MspOpts), C.POINTER(MspInfo)]),
    "msp_general_solve_m1": (C.c_int, [P, P, P, P, C.c_int, C.c_int]),
    "msp_general_solve_m2": (C.c_int, [P, P, P, P, C.c_int]),
    "msp_general_matvec64": (C.c_int, [P, P, P, P]),
    "msp_general_op": (C.c_int, [P, P, P, P]),
    "msp_solve_many": (C.c_int, [P, P, P, C.c_int, I64, I64, C.c_double, P, I64, P, I64, I64, C.POINTER(MspOpts),
                                 C.POINTER(MspInfo)]),
    "msp_general_set_lambda": (C.c_int, [P, P, C.c_double, C.c_double]),
    "msp_schatten_p": (C.c_int, [P, P, I64, I64, I64, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                 I64, C.c_uint64, I64, C.c_double, C.POINTER(MspOpts), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), P]),
    "msp_lsq_create": (C.c_int, [P, P, I64, I64, I64, I64, C.c_int, C.c_double, I64, C.c_int, I64, C.c_int,
                                 C.c_uint64, C.POINTER(P)]),
    "msp_lsq_destroy": (None, [P]),
    "msp_lsq_solve": (C.c_int, [P, P, P, P, C.POINTER(MspOpts), C.POINTER(MspInfo), C.POINTER(C.c_double)]),
    "msp_batch_create": (C.c_int, [P, C.c_int, C.POINTER(MspInstance), C.POINTER(P)]),
    "msp_batch_destroy": (None, [P]),
    "msp_batch_solve": (C.c_int, [P, P, C.POINTER(MspOpts), C.POINTER(MspInfo)]),
    "msp_batch_info": (C.c_int, [P, P, C.POINTER(MspInfo)]),
    "msp_batch_stats": (C.c_int, [P, P, P]),
    "msp_batch_autotune": (C.c_int, [P, P, C.POINTER(C.c_int)]),
    "msp_solve_batched": (C.c_int, [P, C.c_int, C.POINTER(MspInstance), C.POINTER(MspOpts),
                                    C.POINTER(MspInfo)]),
    "msp_schatten": (C.c_int, [P, P, C.c_int, I64, I64, C.c_double, I64, C.c_uint64,
                               C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "msp_hutchinson": (C.c_int, [P, P, C.c_int, I64, I64, I64, C.c_uint64, P]),
    "msp_set_hutchinson_terms": (C.c_int, [P, C.c_int]),
    "msp_rbf_kernel": (C.c_int, [P, P, I64, C.c_int, C.c_double, P, I64]),
    "msp_rbf_grad_ell": (C.c_int, [P, P, I64, C.c_int, C.c_double, P, P, P]),
    "msp_rbf_grad_ell_static": (C.c_int, [P, I64, C.c_int, C.c_double, P, P, P, P]),
}

_lib = None


def header_symbols() -> list[str]:
    """Function names declared in include/msp.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^MSP_API\s+[\w\s\*]+?\b(msp_\w+)\s*\(", txt, flags=re.M)))


def load() -> C.CDLL:
    """Load libmsp.so (built in-tree) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmsp.so is not built ({LIB_PATH}); run "
                          "`python -m paper_2405_05865_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(ctx, status: int) -> None:
    if status != 0:
        msg = load().msp_last_error(ctx)
        raise MspError(status, msg.decode() if msg else "")
