"""Python API over libmsp: PyTorch supplies device memory and the stream; every
step of MSP runs in the library's CUDA kernels (see include/msp.h).

    ctx = Context()                         # device 0, torch's current stream
    sk = ctx.sketch(A, s=1024, gamma=8)     # Algorithm 1 steps 2-3: C = A S^T
    f = ctx.nystrom(sk, lam=1e-2)           # steps 3-4: W, C~, M2 and its factor
    x, info = ctx.solve(f, A, b, lam=1e-2)  # step 5 (+ FP64 refinement)
"""

from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L

DEFAULT_SEED = 0x4D5350      # "MSP"

_DT = {torch.float32: L.MSP_F32, torch.float64: L.MSP_F64, torch.bfloat16: L.MSP_BF16}
_PREC = {"fp64": L.MSP_PREC_FP64, "fp32": L.MSP_PREC_FP32, "mixed": L.MSP_PREC_MIXED}
_STOP = {"residual": L.MSP_STOP_RESIDUAL, "backward": L.MSP_STOP_BACKWARD}


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def make_opts(lib, **kw) -> L.MspOpts:
    o = L.MspOpts()
    lib.msp_default_opts(C.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "precision" and isinstance(v, str):
            v = _PREC[v]
        if k == "criterion" and isinstance(v, str):
            v = _STOP[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _check_matrix(A: torch.Tensor, need_cuda: bool = True) -> tuple[int, int, int]:
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square 2-D tensor")
    if A.dtype not in _DT:
        raise TypeError("A must be float32, float64 or bfloat16")
    if need_cuda and not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.stride(1) != 1:
        raise ValueError("A must be row-major with unit column stride")
    return A.shape[0], A.stride(0), _DT[A.dtype]


def params_from_effdim(d: float, n: int, lam: float) -> dict:
    """The library's rule from d_lambda to (l, s, lambda0, capped, direct);
    host only (msp_params_from_effdim)."""
    lib = L.load()
    out = L.MspAutoParams()
    st = lib.msp_params_from_effdim(float(d), int(n), float(lam), C.byref(out))
    if st != 0:
        raise L.MspError(st, "params_from_effdim: invalid arguments")
    return out.as_dict()


class Sketch:
    def __init__(self, ctx: "Context", handle: C.c_void_p, n: int, s: int, dtype: torch.dtype):
        self.ctx, self.handle, self.n, self.s, self.dtype = ctx, handle, n, s, dtype

    def C(self) -> torch.Tensor:
        out = torch.empty((self.n, self.s), dtype=self.dtype, device=self.ctx.device)
        L.check(self.ctx.ptr, self.ctx.lib.msp_sketch_get_C(self.ctx.ptr, self.handle, _ptr(out), self.s))
        return out

    def close(self) -> None:
        if self.handle:
            self.ctx.lib.msp_sketch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    def __init__(self, ctx: "Context", handle: C.c_void_p, sketch: Sketch):
        self.ctx, self.handle, self.sketch = ctx, handle, sketch

    def parts(self) -> dict:
        s = self.sketch.s
        dev = self.ctx.device
        W = torch.empty((s, s), dtype=torch.float64, device=dev)
        M2 = torch.empty_like(W)
        Li = torch.empty_like(W)
        lt, sh, rt = C.c_double(), C.c_double(), C.c_int()
        L.check(self.ctx.ptr, self.ctx.lib.msp_factor_get(self.ctx.ptr, self.handle, _ptr(W), _ptr(M2),
                                                          _ptr(Li), C.byref(lt), C.byref(sh), C.byref(rt)))
        return {"W": W, "M2": M2, "Linv": Li, "lambda_tilde": lt.value, "shift": sh.value,
                "retries": rt.value}

    def close(self) -> None:
        if self.handle:
            self.ctx.lib.msp_factor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A set-up batch (msp_batch_create). Holds the caller tensors whose
    pointers the library keeps: A, and the column-major copies of B and the
    solution X (``X(k)`` returns instance k's solution as an (n, m) view)."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, keep: list):
        self.ctx, self.handle, self.keep = ctx, handle, keep
        self.count = len(keep)

    def X(self, k: int) -> torch.Tensor:
        return self.keep[k][2].t()

    def solve(self, sync: bool = True, raise_on_noconv: bool = True, **opts) -> list[dict] | None:
        """One persistent launch over every instance; sync=False returns at
        once (no host synchronisation; the call can be captured in a CUDA
        graph on the context's stream)."""
        o = make_opts(self.ctx.lib, **opts)
        if not sync:
            L.check(self.ctx.ptr, self.ctx.lib.msp_batch_solve(self.ctx.ptr, self.handle, C.byref(o), None))
            return None
        infos = (L.MspInfo * self.count)()
        st = self.ctx.lib.msp_batch_solve(self.ctx.ptr, self.handle, C.byref(o), infos)
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ctx.ptr, st)
        return [i.as_dict() for i in infos]

    def info(self) -> list[dict]:
        infos = (L.MspInfo * self.count)()
        st = self.ctx.lib.msp_batch_info(self.ctx.ptr, self.handle, infos)
        if st not in (0, 5):
            L.check(self.ctx.ptr, st)
        return [i.as_dict() for i in infos]

    def autotune(self, unit_tiles: int = 0) -> int:
        """Set (unit_tiles > 0) or search (0) the unit width of the batched A
        passes; returns the width in use. A search overwrites the X buffers."""
        v = C.c_int(unit_tiles)
        L.check(self.ctx.ptr, self.ctx.lib.msp_batch_autotune(self.ctx.ptr, self.handle, C.byref(v)))
        return v.value

    def stats(self) -> dict:
        """Counters and device-timer split of the last solve (msp_batch_stats)."""
        v = (C.c_double * 16)()
        L.check(self.ctx.ptr, self.ctx.lib.msp_batch_stats(self.ctx.ptr, self.handle, v))
        keys = ("a_passes", "resid_passes", "a_bytes", "resid_bytes", "a_ms", "g_ms", "tri_ms",
                "z_ms", "vec_ms", "resid_ms", "check_ms", "dense_pass_bytes", "nn_bytes", "g_bytes",
                "z_bytes", "unit_tiles")
        return dict(zip(keys, list(v)))

    def close(self) -> None:
        if self.handle:
            self.ctx.lib.msp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class General:
    """Three-level MSP for (A^T A + lam I) x = c (msp_general_create). Keeps
    the caller's A alive: the library reads it on every solve."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, A: torch.Tensor):
        self.ctx, self.handle, self.A = ctx, handle, A
        self.m, self.n = A.shape
        sp, lt, sa, sb = L.I64(), C.c_double(), C.c_double(), C.c_double()
        L.check(ctx.ptr, ctx.lib.msp_general_info(handle, C.byref(sp), C.byref(lt), C.byref(sa), C.byref(sb)))
        self.s_pad, self.lambda_tilde, self.shift_a, self.shift_b = sp.value, lt.value, sa.value, sb.value

    def solve(self, c: torch.Tensor, raise_on_noconv: bool = True, **opts) -> tuple[torch.Tensor, dict]:
        if not c.is_cuda or c.dtype != torch.float64 or c.shape != (self.n,):
            raise ValueError("c must be a CUDA float64 vector of length n")
        c = c.contiguous()
        x = torch.empty_like(c)
        o = make_opts(self.ctx.lib, **opts)
        info = L.MspInfo()
        st = self.ctx.lib.msp_general_solve(self.ctx.ptr, self.handle, _ptr(c), _ptr(x), C.byref(o), C.byref(info))
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ctx.ptr, st)
        return x, info.as_dict()

    def solve_m1(self, r: torch.Tensor, t2: int, t3: int) -> torch.Tensor:
        r = r.to(torch.float32).contiguous()
        w = torch.empty(self.n, dtype=torch.float32, device=r.device)
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_solve_m1(self.ctx.ptr, self.handle, _ptr(r), _ptr(w), t2, t3))
        return w

    def solve_m2(self, r: torch.Tensor, t3: int) -> torch.Tensor:
        r = r.to(torch.float32).contiguous()
        z = torch.empty(r.shape[0], dtype=torch.float32, device=r.device)
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_solve_m2(self.ctx.ptr, self.handle, _ptr(r), _ptr(z), t3))
        return z

    def op(self, p: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """q = (A^T A + lam I) p in FP32 (the level-1 operator, one row pass)."""
        p = p.to(torch.float32).contiguous()
        q = out if out is not None else torch.empty_like(p)
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_op(self.ctx.ptr, self.handle, _ptr(p), _ptr(q)))
        return q

    def matvec(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(torch.float64).contiguous()
        y = torch.empty_like(x)
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_matvec64(self.ctx.ptr, self.handle, _ptr(x), _ptr(y)))
        return y

    def set_lambda(self, lam: float, lam0: float = 0.0) -> None:
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_set_lambda(self.ctx.ptr, self.handle, float(lam), float(lam0)))
        self.lambda_tilde = lam + lam0

    def setup(self, s: int) -> dict:
        """A~ (m x s FP32) and the FP64 Grams M3a, M3b (s x s) as device tensors."""
        dev = self.A.device
        At = torch.empty((self.m, s), dtype=torch.float32, device=dev)
        M3a = torch.empty((s, s), dtype=torch.float64, device=dev)
        M3b = torch.empty_like(M3a)
        L.check(self.ctx.ptr, self.ctx.lib.msp_general_get(self.ctx.ptr, self.handle, _ptr(At), s, _ptr(M3a),
                                                           _ptr(M3b)))
        return {"At": At, "M3a": M3a, "M3b": M3b}

    def close(self) -> None:
        if self.handle:
            self.ctx.lib.msp_general_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LeastSquares:
    """min |A x - b| by sketch-and-precondition with three-level inner solves
    (msp_lsq_create). Keeps the caller's A alive."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, A: torch.Tensor):
        self.ctx, self.handle, self.A = ctx, handle, A
        self.n_rows, self.d = A.shape

    def solve(self, b: torch.Tensor, raise_on_noconv: bool = True, **opts) -> tuple[torch.Tensor, dict]:
        if not b.is_cuda or b.dtype != torch.float64 or b.shape != (self.n_rows,):
            raise ValueError("b must be a CUDA float64 vector of length n_rows")
        b = b.contiguous()
        x = torch.empty(self.d, dtype=torch.float64, device=b.device)
        opts.setdefault("inner_tol", 1e-2)
        o = make_opts(self.ctx.lib, **opts)
        info = L.MspInfo()
        rn = C.c_double()
        st = self.ctx.lib.msp_lsq_solve(self.ctx.ptr, self.handle, _ptr(b), _ptr(x), C.byref(o), C.byref(info),
                                        C.byref(rn))
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ctx.ptr, st)
        d = info.as_dict()
        d["resid_norm"] = rn.value
        return x, d

    def close(self) -> None:
        if self.handle:
            self.ctx.lib.msp_lsq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """An MSP context bound to one CUDA device and one stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("MSP needs a CUDA device; none is available")
        self.lib = L.load()
        self.device = torch.device("cuda", device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ptr = C.c_void_p()
        L.check(None, self.lib.msp_create(C.byref(self.ptr), device, C.c_void_p(self.stream.cuda_stream)))

    def close(self) -> None:
        if self.ptr:
            self.lib.msp_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- a1
    def sketch_pattern(self, n: int, rows: int, gamma: int, seed: int = DEFAULT_SEED,
                       stream: int = 0) -> tuple[torch.Tensor, torch.Tensor]:
        idx = torch.empty((n, gamma), dtype=torch.int32, device=self.device)
        sgn = torch.empty((n, gamma), dtype=torch.int8, device=self.device)
        L.check(self.ptr, self.lib.msp_sketch_pattern(self.ptr, n, rows, gamma, seed, stream,
                                                      _ptr(idx), _ptr(sgn)))
        return idx, sgn

    # -- a1-a2
    def sketch(self, A: torch.Tensor, s: int, gamma: int = 8, seed: int = DEFAULT_SEED) -> Sketch:
        n, lda, dt = _check_matrix(A)
        h = C.c_void_p()
        L.check(self.ptr, self.lib.msp_sketch(self.ptr, _ptr(A), dt, n, lda, s, gamma, seed, C.byref(h)))
        # a BF16 A is read in BF16; C and what follows are FP32
        return Sketch(self, h, n, s, torch.float32 if A.dtype == torch.bfloat16 else A.dtype)

    # -- a3-a5
    def nystrom(self, sk: Sketch, lam: float, lam0: float = 0.0, phi: int | None = None,
                gamma_phi: int = 8, seed: int = DEFAULT_SEED, data: str = "fp32") -> Factor:
        """Algorithm 1 steps 3-4; data = "bf16" stores the level-2 data C and W
        in BF16 (msp_nystrom_ex)."""
        if phi is None:
            phi = 4 * sk.s
        h = C.c_void_p()
        dt = {"fp32": L.MSP_F32, "bf16": L.MSP_BF16}[data]
        L.check(self.ptr, self.lib.msp_nystrom_ex(self.ptr, sk.handle, lam, lam0, phi, gamma_phi, seed, dt,
                                                  C.byref(h)))
        return Factor(self, h, sk)

    def solve_m1(self, f: Factor, r: torch.Tensor, **opts) -> tuple[torch.Tensor, int]:
        if not r.is_cuda or r.dtype != f.sketch.dtype or r.numel() != f.sketch.n:
            raise ValueError("r must be a CUDA vector of the sketch's dtype and length n")
        w = torch.empty_like(r)
        o = make_opts(self.lib, **opts)
        it = C.c_int()
        L.check(self.ptr, self.lib.msp_solve_m1(self.ptr, f.handle, _ptr(r.contiguous()), _ptr(w),
                                                C.byref(o), C.byref(it)))
        return w, it.value

    # -- a6-a8
    def solve(self, f: Factor, A: torch.Tensor, b: torch.Tensor, lam: float,
              raise_on_noconv: bool = True, **opts) -> tuple[torch.Tensor, dict]:
        n, lda, dt = _check_matrix(A)
        if not b.is_cuda or b.dtype != torch.float64 or b.numel() != n:
            raise ValueError("b must be a CUDA float64 vector of length n")
        b = b.contiguous()
        x = torch.empty_like(b)
        o = make_opts(self.lib, **opts)
        info = L.MspInfo()
        st = self.lib.msp_solve(self.ptr, f.handle, _ptr(A), dt, n, lda, lam, _ptr(b), _ptr(x),
                                C.byref(o), C.byref(info))
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ptr, st)
        return x, info.as_dict()

    def set_sketch_one_pass(self, on: bool) -> None:
        """FP32 sketch pass: one pass over the symmetric A (default) or separate passes."""
        L.check(self.ptr, self.lib.msp_set_sketch_one_pass(self.ptr, int(bool(on))))

    def set_level1_graphs(self, on: bool) -> None:
        """Level-1 iterations replayed as a CUDA graph (default) or launched one by one."""
        L.check(self.ptr, self.lib.msp_set_level1_graphs(self.ptr, int(bool(on))))

    def set_factor_float_float(self, on: bool) -> None:
        """Cholesky of an FP32 factor in float-float (default) or in FP64."""
        L.check(self.ptr, self.lib.msp_set_factor_float_float(self.ptr, int(bool(on))))

    def set_gram_tensor_cores(self, on: bool) -> None:
        """M2 Gram on the tensor cores (default) or on the FP32 pipe."""
        L.check(self.ptr, self.lib.msp_set_gram_tensor_cores(self.ptr, int(bool(on))))

    def set_grid_wait_limit(self, seconds: float) -> None:
        """Limit of the level-1 / level-2 grid barriers (0: the default 2 s)."""
        L.check(self.ptr, self.lib.msp_set_grid_wait_limit(self.ptr, float(seconds)))

    def solve_refined(self, f: Factor, A: torch.Tensor, A_res: torch.Tensor, b: torch.Tensor, lam: float,
                      raise_on_noconv: bool = True, **opts) -> tuple[torch.Tensor, dict]:
        """msp_solve_refined: the level-1 iteration applies A (FP32, the
        factor's matrix); each FP64 refinement residual applies A_res (the
        problem, FP64 or FP32)."""
        n, lda, dt = _check_matrix(A)
        nr, ldr, dtr = _check_matrix(A_res)
        if nr != n:
            raise ValueError("A and A_res must have the same size")
        if not b.is_cuda or b.dtype != torch.float64 or b.numel() != n:
            raise ValueError("b must be a CUDA float64 vector of length n")
        b = b.contiguous()
        x = torch.empty_like(b)
        o = make_opts(self.lib, **opts)
        info = L.MspInfo()
        st = self.lib.msp_solve_refined(self.ptr, f.handle, _ptr(A), dt, n, lda, _ptr(A_res), dtr, ldr, lam,
                                        _ptr(b), _ptr(x), C.byref(o), C.byref(info))
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ptr, st)
        return x, info.as_dict()

    def solve_many(self, f: Factor, A: torch.Tensor, B: torch.Tensor, lam: float,
                   raise_on_noconv: bool = True, **opts) -> tuple[torch.Tensor, list[dict]]:
        """Columns of B (CUDA float64 (n, m)) solved one by one with the factor f."""
        n, lda, dt = _check_matrix(A)
        if not B.is_cuda or B.dtype != torch.float64 or B.dim() != 2 or B.shape[0] != n:
            raise ValueError("B must be a CUDA float64 (n, m) tensor")
        m = B.shape[1]
        Bc = B.t().contiguous()              # column-major n x m
        Xc = torch.empty_like(Bc)
        o = make_opts(self.lib, **opts)
        infos = (L.MspInfo * max(m, 1))()
        st = self.lib.msp_solve_many(self.ptr, f.handle, _ptr(A), dt, n, lda, lam, _ptr(Bc), n, _ptr(Xc), n, m,
                                     C.byref(o), infos)
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ptr, st)
        return Xc.t(), [infos[j].as_dict() for j in range(m)]

    def solve_full(self, A: torch.Tensor, b: torch.Tensor, lam: float, s: int, gamma: int = 8,
                   lam0: float = 0.0, phi: int | None = None, gamma_phi: int = 8,
                   seed: int = DEFAULT_SEED, out: torch.Tensor | None = None,
                   **opts) -> tuple[torch.Tensor, dict]:
        """Algorithm 1 end to end; A, b, out may live on the host (pinned is fastest)
        or on the device."""
        n, lda, dt = _check_matrix(A, need_cuda=False)
        if b.dtype != torch.float64 or b.numel() != n:
            raise ValueError("b must be a float64 vector of length n")
        if phi is None:
            phi = 4 * s
        x = out if out is not None else torch.empty(n, dtype=torch.float64,
                                                    pin_memory=not b.is_cuda,
                                                    device=b.device if b.is_cuda else "cpu")
        o = make_opts(self.lib, **opts)
        info = L.MspInfo()
        L.check(self.ptr, self.lib.msp_solve_full(self.ptr, _ptr(A), dt, n, lda, lam, _ptr(b.contiguous()),
                                                  _ptr(x), s, gamma, lam0, phi, gamma_phi, seed,
                                                  C.byref(o), C.byref(info)))
        return x, info.as_dict()

    # -- a9: batches of instances, up to 16 right-hand sides each
    def batch(self, instances: list[dict], gamma: int = 8, lam0: float = 0.0, phi: int = 0,
              gamma_phi: int = 8, seed: int = DEFAULT_SEED) -> Batch:
        """instances: dicts with A (CUDA FP32 (n, n)), B (CUDA FP64 (n, m) or
        (n,)), lam, s, and optionally gamma, lam0, phi, gamma_phi, seed."""
        arr = (L.MspInstance * len(instances))()
        keep = []
        for k, d in enumerate(instances):
            A = d["A"]
            n, lda, dt = _check_matrix(A)
            if dt != L.MSP_F32:
                raise TypeError("batched instances need an FP32 A")
            B = d["B"]
            if not B.is_cuda or B.dtype != torch.float64 or B.shape[0] != n:
                raise ValueError("B must be a CUDA float64 (n, m) tensor")
            if B.dim() == 1:
                B = B[:, None]
            Bc = B.t().contiguous()          # column-major n x m
            Xc = torch.empty_like(Bc)
            e = arr[k]
            e.A, e.n, e.lda = A.data_ptr(), n, lda
            e.lam, e.lam0 = float(d["lam"]), float(d.get("lam0", lam0))
            e.B, e.ldb, e.X, e.ldx, e.m = Bc.data_ptr(), n, Xc.data_ptr(), n, Bc.shape[0]
            e.gamma, e.s = int(d.get("gamma", gamma)), int(d["s"])
            e.phi, e.gamma_phi = int(d.get("phi", phi)), int(d.get("gamma_phi", gamma_phi))
            e.seed = int(d.get("seed", seed))
            keep.append((A, Bc, Xc))
        h = C.c_void_p()
        L.check(self.ptr, self.lib.msp_batch_create(self.ptr, len(instances), arr, C.byref(h)))
        return Batch(self, h, keep)

    # -- three-level MSP for (A^T A + lam I) x = c
    def general(self, A: torch.Tensor, lam: float, s: int, lam0: float = 0.0, phi: int | None = None,
                gamma: int = 8, gamma_phi: int = 8, seed: int = DEFAULT_SEED) -> General:
        if not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a CUDA float32 (m, n) tensor with unit column stride")
        m, n = A.shape
        h = C.c_void_p()
        L.check(self.ptr, self.lib.msp_general_create(self.ptr, _ptr(A), m, n, A.stride(0), float(lam), float(lam0),
                                                      s, gamma, phi if phi is not None else 4 * s, gamma_phi, seed,
                                                      C.byref(h)))
        return General(self, h, A)

    # -- Schatten-p, p in (0, 2), from ridge solves (integral representation)
    def schatten_p(self, A: torch.Tensor, p: float, t_min: float, t_max: float, nodes: int = 32, probes: int = 16,
                   s: int = 64, z: float = 0.0, lambda_floor_rel: float = 1e-3, seed: int = DEFAULT_SEED,
                   **opts) -> tuple[float, float, list[float]]:
        """(estimate of |A + zI|_p^p, standard error, per-probe estimates)."""
        if not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a CUDA float32 (m, n) tensor with unit column stride")
        m, n = A.shape
        o = make_opts(self.lib, **opts)
        est, se = C.c_double(), C.c_double()
        X = (C.c_double * probes)()
        L.check(self.ptr, self.lib.msp_schatten_p(self.ptr, _ptr(A), m, n, A.stride(0), float(p), float(z),
                                                  float(t_min), float(t_max), nodes, probes, seed, s,
                                                  float(lambda_floor_rel), C.byref(o), C.byref(est), C.byref(se),
                                                  C.cast(X, C.c_void_p)))
        return est.value, se.value, list(X)

    # -- least squares (sketch-and-precondition, three-level inner solves)
    def lsq(self, A: torch.Tensor, s_ls: int, lam0: float, s: int, gamma_ls: int = 4, phi: int | None = None,
            gamma: int = 8, gamma_phi: int = 8, seed: int = DEFAULT_SEED) -> LeastSquares:
        if not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a CUDA float32 (n_rows, d) tensor with unit column stride")
        n_rows, d = A.shape
        h = C.c_void_p()
        L.check(self.ptr, self.lib.msp_lsq_create(self.ptr, _ptr(A), n_rows, d, A.stride(0), s_ls, gamma_ls,
                                                  float(lam0), s, gamma, phi if phi is not None else 4 * s,
                                                  gamma_phi, seed, C.byref(h)))
        return LeastSquares(self, h, A)

    # -- effective dimension d_lambda by Hutchinson over batched solves
    def effective_dimension(self, A: torch.Tensor, lam: float, s: int, probes: int = 64, gamma: int = 8,
                            seed: int = DEFAULT_SEED, raise_on_noconv: bool = True,
                            **opts) -> tuple[float, float, torch.Tensor]:
        """(estimate of tr(A (A + lam I)^{-1}), standard error, per-probe values)."""
        n, lda, dt = _check_matrix(A)
        if dt != L.MSP_F32:
            raise TypeError("effective_dimension needs an FP32 A")
        o = make_opts(self.lib, **opts)
        est, se = C.c_double(), C.c_double()
        q = torch.empty(probes, dtype=torch.float64, device=self.device)
        st = self.lib.msp_effective_dimension(self.ptr, _ptr(A), n, lda, float(lam), probes, seed, s, gamma,
                                              C.byref(o), C.byref(est), C.byref(se), _ptr(q))
        if st != 0 and not (st == 5 and not raise_on_noconv):
            L.check(self.ptr, st)
        return est.value, se.value, q

    def auto_params(self, A: torch.Tensor, lam: float, probes: int = 64, gamma: int = 8,
                    seed: int = DEFAULT_SEED, **opts) -> dict:
        """Sketch size s ~ 2 d_lambda and shift lambda0 from a d_lambda estimate."""
        n, lda, dt = _check_matrix(A)
        if dt != L.MSP_F32:
            raise TypeError("auto_params needs an FP32 A")
        o = make_opts(self.lib, **opts)
        out = L.MspAutoParams()
        L.check(self.ptr, self.lib.msp_auto_params(self.ptr, _ptr(A), n, lda, float(lam), probes, seed, gamma,
                                                    C.byref(o), C.byref(out)))
        return out.as_dict()

    # -- a10: Schatten-1 norm (PSD A) by Hutchinson
    def schatten(self, A: torch.Tensor, p: float = 1.0, probes: int = 256,
                 seed: int = DEFAULT_SEED) -> tuple[float, float]:
        """(estimate of |A|_p, standard error); p = 1 only."""
        n, lda, dt = _check_matrix(A)
        v, vp, se = C.c_double(), C.c_double(), C.c_double()
        L.check(self.ptr, self.lib.msp_schatten(self.ptr, _ptr(A), dt, n, lda, p, probes, seed,
                                                C.byref(v), C.byref(vp), C.byref(se)))
        return v.value, se.value

    def hutchinson(self, A: torch.Tensor, probes: int = 256, seed: int = DEFAULT_SEED) -> torch.Tensor:
        n, lda, dt = _check_matrix(A)
        q = torch.empty(probes, dtype=torch.float64, device=self.device)
        L.check(self.ptr, self.lib.msp_hutchinson(self.ptr, _ptr(A), dt, n, lda, probes, seed, _ptr(q)))
        return q

    def set_hutchinson_terms(self, terms: int) -> None:
        """BF16 terms per FP32 entry in the tensor-core Hutchinson product (2 or 3)."""
        L.check(self.ptr, self.lib.msp_set_hutchinson_terms(self.ptr, int(terms)))

    # -- a11: RBF kernels and the adjoint of the length scale
    def rbf_kernel(self, points: torch.Tensor, ell: float) -> torch.Tensor:
        if not points.is_cuda or points.dtype != torch.float64 or points.dim() != 2:
            raise ValueError("points must be a CUDA float64 (n, dim) tensor")
        points = points.contiguous()
        n, dim = points.shape
        K = torch.empty((n, n), dtype=torch.float32, device=self.device)
        L.check(self.ptr, self.lib.msp_rbf_kernel(self.ptr, _ptr(points), n, dim, float(ell), _ptr(K), n))
        return K

    def rbf_grad_ell(self, points: torch.Tensor, ell: float, a: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        points = points.contiguous()
        n, dim = points.shape
        out = torch.empty((), dtype=torch.float64, device=self.device)
        L.check(self.ptr, self.lib.msp_rbf_grad_ell(self.ptr, _ptr(points), n, dim, float(ell),
                                                    _ptr(a.contiguous()), _ptr(x.contiguous()), _ptr(out)))
        return out

    def dot(self, x: torch.Tensor, y: torch.Tensor, scale: float = 1.0) -> torch.Tensor:
        """scale * x^T y as a 0-d CUDA float64 tensor (msp_dot)."""
        if not (x.is_cuda and y.is_cuda and x.dtype == y.dtype == torch.float64 and x.numel() == y.numel()):
            raise ValueError("x, y must be CUDA float64 vectors of one length")
        out = torch.empty((), dtype=torch.float64, device=self.device)
        L.check(self.ptr, self.lib.msp_dot(self.ptr, _ptr(x.contiguous()), _ptr(y.contiguous()), x.numel(),
                                           float(scale), _ptr(out)))
        return out

    def norm_lower_bound(self, A: torch.Tensor) -> float:
        """L <= |A|_2 (largest column norm, all-ones Rayleigh quotient)."""
        n, lda, dt = _check_matrix(A)
        v = C.c_double()
        L.check(self.ptr, self.lib.msp_norm_lower_bound(self.ptr, _ptr(A), dt, n, lda, C.byref(v)))
        return v.value

    def matvec_f64(self, A: torch.Tensor, x: torch.Tensor, lam: float = 0.0) -> torch.Tensor:
        n, lda, dt = _check_matrix(A)
        y = torch.empty_like(x)
        L.check(self.ptr, self.lib.msp_matvec_f64(self.ptr, _ptr(A), dt, n, lda, lam, _ptr(x.contiguous()),
                                                  _ptr(y)))
        return y
