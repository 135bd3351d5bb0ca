// Entry points of libmsp (include/msp.h): contexts, handles, argument checks,
// staging of host buffers and the FP64 refinement driver.
#include "msp_internal.cuh"

#include <cstdint>

#include <cuda_bf16.h>

#include <vector>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

namespace {

thread_local std::string g_noctx_error;

using msp::DeviceGuard;

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

msp_status msp_set_error(msp_ctx* ctx, msp_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->last_error = buf;
    else g_noctx_error = buf;
    return st;
}

msp_status msp_alloc(msp_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    MSP_CUDA_TRY(ctx, cudaMallocAsync(p, bytes, ctx->stream));
    return MSP_OK;
}

// Stream-ordered free; the pool keeps the memory for reuse.
static void free_on(msp_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx ? ctx->stream : nullptr);
}

void msp_free(void* p) {
    if (p) cudaFreeAsync(p, nullptr);
}

msp_status msp_scratch(msp_ctx* ctx, size_t bytes, void** out) {
    if (bytes > ctx->scratch_bytes) {
        // grow geometrically (1.5x the old size at least) so a sequence of
        // slightly larger requests does not reallocate every time
        const size_t old = ctx->scratch_bytes;
        free_on(ctx, ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
        size_t want = std::max(bytes, old + old / 2);
        MSP_TRY(msp_alloc(ctx, &ctx->scratch, want));
        ctx->scratch_bytes = want;
    }
    *out = ctx->scratch;
    return MSP_OK;
}

static msp_status stage_alloc(msp_ctx* ctx, size_t bytes) {
    if (bytes > ctx->stage_bytes) {
        free_on(ctx, ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        MSP_TRY(msp_alloc(ctx, &ctx->stage, bytes));
        ctx->stage_bytes = bytes;
    }
    return MSP_OK;
}

extern "C" {

const char* msp_version(void) { return "msp-gb300 0.1 sm_103a"; }

int64_t msp_launch_count(const msp_ctx* ctx) { return ctx ? ctx->launches : 0; }

void msp_default_opts(msp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->tol = 1e-10;
    o->max_outer = 2000;
    o->max_refine = 20;
    o->refine_tol = 1e-6;
    o->inner_tol = 1e-6;
    o->max_inner = 50;
    o->precision = MSP_PREC_MIXED;
    o->check_every = 8;
    o->level2_iters = 8;
    o->level3_iters = 8;
}

const char* msp_last_error(const msp_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_noctx_error.c_str();
}

msp_status msp_create(msp_ctx** out, int device, void* stream) {
    if (!out) return msp_set_error(nullptr, MSP_EINVAL, "msp_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return msp_set_error(nullptr, MSP_EINVAL, "msp_create: no CUDA device %d", device);
    }
    DeviceGuard g(device);
    msp_ctx* ctx = new (std::nothrow) msp_ctx();
    if (!ctx) return msp_set_error(nullptr, MSP_ENOMEM, "msp_create: out of host memory");
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return msp_set_error(nullptr, MSP_ECUDA, "msp_create: cudaGetDeviceProperties failed");
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    // keep freed pool memory for reuse (stream-ordered allocations are made
    // and released once per solve)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMalloc(&ctx->ctl, sizeof(CtlBlock)) != cudaSuccess ||
        cudaMallocHost(&ctx->host_flags, 256) != cudaSuccess) {
        cudaGetLastError();
        msp_destroy(ctx);
        return msp_set_error(nullptr, MSP_ENOMEM, "msp_create: allocation failed");
    }
    cudaMemset(ctx->ctl, 0, sizeof(CtlBlock));
    *out = ctx;
    return MSP_OK;
}

void msp_destroy(msp_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->ctl) cudaFree(ctx->ctl);
    if (ctx->host_flags) cudaFreeHost(ctx->host_flags);
    msp_l1_graph_release(ctx);
    msp_fac_graph_release(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (int i = 0; i < ctx->n_events; ++i) cudaEventDestroy(ctx->events[i]);
    delete[] ctx->events;
    for (int i = 0; i < ctx->n_lanes; ++i) {
        msp_destroy(ctx->lanes[i]);
        cudaStreamDestroy(ctx->lane_streams[i]);
    }
    delete[] ctx->lanes;
    delete[] ctx->lane_streams;
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    for (cudaEvent_t e : ctx->aux_ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : ctx->fac_side)
        if (s) cudaStreamDestroy(s);
    for (auto& pair : ctx->fac_ev)
        for (cudaEvent_t e : pair)
            if (e) cudaEventDestroy(e);
    delete ctx;
}

// ------------------------------------------------------------------ a1

msp_status msp_sketch_pattern(msp_ctx* ctx, int64_t n, int64_t rows, int gamma, uint64_t seed,
                              int stream, int32_t* idx, int8_t* sgn) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!idx || !sgn) return msp_set_error(ctx, MSP_EINVAL, "pattern: NULL output");
    DeviceGuard g(ctx->device);
    return msp_pattern_launch(ctx, n, rows, gamma, seed, stream, idx, sgn, nullptr);
}

// --------------------------------------------------------------- a1-a2

// The one-pass sketch of a symmetric FP32 A, then (with stats) the
// norm-bound row statistics. Both only read A. The statistics pass is
// HBM-bound with many small blocks, while the sketch kernel holds one
// 1024-thread block per SM and runs n / 32 blocks in waves, the last one
// partly filled (512 blocks on 152 SMs at n = 16384). So the statistics are
// enqueued on a side stream that forks from the main stream before the
// sketch launch and joins it after: their blocks take the SMs the sketch's
// last wave leaves idle. The sketch is submitted first.
static msp_status sym_pass_and_stats(msp_ctx* ctx, const float* A, msp_dtype dtype, int64_t n, int64_t lda,
                                     int64_t sp, const int32_t* ptr, const int32_t* ent, int gamma, float* C,
                                     float* packed, double* stats) {
    cudaStream_t side = nullptr;
    if (stats) {
        if ((ctx->aux_stream ||
             cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking) == cudaSuccess) &&
            (ctx->aux_ev[0] || cudaEventCreateWithFlags(&ctx->aux_ev[0], cudaEventDisableTiming) == cudaSuccess) &&
            (ctx->aux_ev[1] || cudaEventCreateWithFlags(&ctx->aux_ev[1], cudaEventDisableTiming) == cudaSuccess) &&
            cudaEventRecord(ctx->aux_ev[0], ctx->stream) == cudaSuccess &&
            cudaStreamWaitEvent(ctx->aux_stream, ctx->aux_ev[0], 0) == cudaSuccess)
            side = ctx->aux_stream;
        else
            cudaGetLastError();   // the statistics stay on the main stream
    }
    msp_status st = msp_sketch_sym_pass(ctx, A, n, lda, sp, ptr, ent, gamma, C, packed);
    if (stats && st == MSP_OK) {
        if (side) {
            cudaStream_t main_stream = ctx->stream;
            ctx->stream = side;
            st = msp_norm_lb_launch(ctx, A, dtype, n, lda, stats, stats + 3 * n);
            ctx->stream = main_stream;
            if (st == MSP_OK && (cudaEventRecord(ctx->aux_ev[1], side) != cudaSuccess ||
                                 cudaStreamWaitEvent(ctx->stream, ctx->aux_ev[1], 0) != cudaSuccess))
                st = msp_set_error(ctx, MSP_ECUDA, "sketch: side stream join failed");
        } else {
            st = msp_norm_lb_launch(ctx, A, dtype, n, lda, stats, stats + 3 * n);
        }
    }
    if (side && st != MSP_OK) cudaStreamSynchronize(side);
    return st;
}

void msp_sketch_destroy(msp_sketch_t* sk) {
    if (!sk) return;
    for (void* p : {(void*)sk->idx, (void*)sk->sgn, (void*)sk->csr_ptr, (void*)sk->csr_ent, sk->C,
                    (void*)sk->packed, (void*)sk->stats})
        if (p) cudaFreeAsync(p, sk->stream);
    delete sk;
}

}  // extern "C"

// The passes over A that only the solve needs: the packed upper tiles of an
// FP32 A (unless the chunked host copy packed them already) and the row
// statistics of the norm bound, which every solve with this sketch's
// factors then reuses. (Run on a side stream beside the factor they gained
// nothing: their blocks took the SMs the factor's kernels wait for.)
static msp_status sketch_solve_prep(msp_ctx* ctx, msp_sketch_s* sk, const void* A, msp_dtype dtype,
                                    int64_t lda, bool do_pack) {
    const int64_t n = sk->n;
    MSP_TRY(msp_alloc(ctx, (void**)&sk->stats, (size_t)(3 * n + 1) * 8));
    if (do_pack && sk->packed) MSP_TRY(msp_pack_upper(ctx, (const float*)A, lda, n, sk->packed));
    return msp_norm_lb_launch(ctx, A, dtype, n, lda, sk->stats, sk->stats + 3 * n);
}

msp_status msp_sketch_impl(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                           int64_t lda, int64_t s, int gamma, uint64_t seed, bool pack,
                           msp_sketch_t** out, const void* host_chunks) {
    if (dtype != MSP_F32 && dtype != MSP_F64 && dtype != MSP_BF16)
        return msp_set_error(ctx, MSP_EINVAL, "sketch: dtype must be MSP_F32, MSP_F64 or MSP_BF16");
    // BF16 A: read in BF16, C and everything after it in FP32; no packed copy
    // and no norm statistics (a solve applies an FP32 A of its own)
    const msp_dtype a_dt = dtype;
    if (dtype == MSP_BF16) {
        if (host_chunks) return msp_set_error(ctx, MSP_EINVAL, "sketch: a BF16 A must be in device memory");
        dtype = MSP_F32;
        pack = false;
    }
    const int64_t s_max = dtype == MSP_F32 ? MSP_MAX_S_SINGLE : MSP_MAX_S;
    if (n < 1 || lda < n || s < 16 || s > s_max || s > n || gamma < 1 ||
        gamma > MSP_MAX_GAMMA || gamma > s || n >= (1ll << 30))
        return msp_set_error(ctx, MSP_EINVAL,
                             "sketch: need 16 <= s <= min(n, %lld), 1 <= gamma <= min(s, %d), "
                             "lda >= n (n=%lld lda=%lld s=%lld gamma=%d)",
                             (long long)s_max, MSP_MAX_GAMMA, (long long)n, (long long)lda,
                             (long long)s, gamma);
    const int64_t sp = round_up(s, MSP_S_ALIGN);
    if (dtype == MSP_F64 && sp > 1024)
        return msp_set_error(ctx, MSP_EINVAL, "sketch: FP64 supports s <= 1024");
    msp_sketch_s* sk = new (std::nothrow) msp_sketch_s();
    if (!sk) return msp_set_error(ctx, MSP_ENOMEM, "sketch: host allocation failed");
    sk->n = n; sk->s = s; sk->s_pad = sp; sk->gamma = gamma; sk->dtype = dtype; sk->seed = seed;
    sk->stream = ctx->stream;
    const size_t ts = dtype_size(dtype);
    msp_status st = MSP_OK;
    bool prep_done = false;    // packed tiles (one-pass kernel) and statistics (their pass) formed
    if ((st = msp_alloc(ctx, (void**)&sk->idx, (size_t)n * gamma * 4)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&sk->sgn, (size_t)n * gamma)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&sk->csr_ptr, (size_t)(sp + 1) * 4)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&sk->csr_ent, (size_t)n * gamma * 4)) != MSP_OK ||
        (st = msp_alloc(ctx, &sk->C, (size_t)n * sp * ts)) != MSP_OK ||
        (st = msp_pattern_launch(ctx, n, s, gamma, seed, 0, sk->idx, sk->sgn, nullptr)) != MSP_OK ||
        (st = msp_build_csr(ctx, n, sp, gamma, sk->idx, sk->sgn, sk->csr_ptr, sk->csr_ent)) !=
            MSP_OK ||
        (dtype == MSP_F32 && pack &&
         (st = msp_alloc(ctx, (void**)&sk->packed, (size_t)msp_packed_tiles(n) * 128 * 128 * 4)) != MSP_OK)) {
        cudaStreamSynchronize(ctx->stream);
        msp_sketch_destroy(sk);
        return st;
    }
    if (host_chunks) {
        // A arrives from the host in row chunks on the copy stream (staged at
        // A_dev, ld n); each chunk's rows of C and its tile rows of the packed
        // copy are formed as soon as it lands
        if (!ctx->copy_stream && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx->copy_stream = nullptr;
            msp_sketch_destroy(sk);
            return msp_set_error(ctx, MSP_ECUDA, "sketch: copy stream creation failed");
        }
        const int64_t rows = std::max<int64_t>(128, round_up((n + 7) / 8, 128));
        const int nchunk = (int)((n + rows - 1) / rows);
        std::vector<cudaEvent_t> ev(nchunk, nullptr);
        cudaEvent_t ready = nullptr;
        bool ok = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventRecord(ready, ctx->stream) == cudaSuccess &&
                  cudaStreamWaitEvent(ctx->copy_stream, ready, 0) == cudaSuccess;
        // FP32 (the symmetric A the packed A pass assumes): only the upper
        // trapezoid of each 128-row block crosses the host link (about half of
        // A); the lower tiles are mirrored on the device once their source
        // rows have landed. FP64: whole rows.
        const bool half = (dtype == MSP_F32);
        // FP32 one-pass: once chunk k has landed, the lower tiles of its tile
        // columns are mirrored from its own rows, which completes the column
        // block A[:, r0 .. r0 + nr); the one-pass kernel then forms those rows
        // of C and the packed tiles of those columns on a side stream, while
        // the later chunks are still being copied. The same kernel on the same
        // blocks: bit for bit the result of a device-resident A.
        const bool one_pass = half && ctx->sketch_sym && msp_sketch_sym_ok(A, n, n, sp, gamma);
        cudaStream_t side = nullptr;
        if (one_pass) {
            if ((ctx->aux_stream ||
                 cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking) == cudaSuccess) &&
                (ctx->aux_ev[0] || cudaEventCreateWithFlags(&ctx->aux_ev[0], cudaEventDisableTiming) == cudaSuccess) &&
                (ctx->aux_ev[1] || cudaEventCreateWithFlags(&ctx->aux_ev[1], cudaEventDisableTiming) == cudaSuccess))
                side = ctx->aux_stream;
            else
                cudaGetLastError();   // the sketch launches stay on the main stream
            if (pack) {
                st = msp_alloc(ctx, (void**)&sk->stats, (size_t)(3 * n + 1) * 8);
                ok = ok && st == MSP_OK;
            }
        }
        for (int k = 0; ok && k < nchunk; ++k) {
            const int64_t r0 = k * rows, nr = std::min(rows, n - r0);
            ok = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
            if (half) {
                for (int64_t b0 = r0; ok && b0 < r0 + nr; b0 += 128) {
                    const int64_t bn = std::min<int64_t>(128, n - b0);
                    ok = cudaMemcpy2DAsync((char*)A + ((size_t)b0 * n + b0) * ts, n * ts,
                                           (const char*)host_chunks + ((size_t)b0 * lda + b0) * ts, lda * ts,
                                           (n - b0) * ts, bn, cudaMemcpyHostToDevice, ctx->copy_stream) == cudaSuccess;
                }
            } else {
                ok = ok && cudaMemcpy2DAsync((char*)A + (size_t)r0 * n * ts, n * ts,
                                             (const char*)host_chunks + (size_t)r0 * lda * ts, lda * ts, n * ts, nr,
                                             cudaMemcpyHostToDevice, ctx->copy_stream) == cudaSuccess;
            }
            ok = ok && cudaEventRecord(ev[k], ctx->copy_stream) == cudaSuccess;
        }
        for (int k = 0; ok && k < nchunk; ++k) {
            const int64_t r0 = k * rows, nr = std::min(rows, n - r0);
            ok = cudaStreamWaitEvent(ctx->stream, ev[k], 0) == cudaSuccess;
            if (!ok) break;
            if (one_pass) {
                if ((st = msp_mirror_lower_cols(ctx, (float*)A, n, n, r0 / 128, (r0 + nr + 127) / 128)) != MSP_OK) {
                    ok = false;
                    break;
                }
                // 32-row blocks of C: this chunk's; the last chunk also takes
                // the padding blocks up to the last tile column
                const int64_t ib0 = r0 / 32, ib1 = (k == nchunk - 1) ? INT64_MAX : (r0 + nr) / 32;
                if (side) {
                    if (cudaEventRecord(ctx->aux_ev[0], ctx->stream) != cudaSuccess ||
                        cudaStreamWaitEvent(side, ctx->aux_ev[0], 0) != cudaSuccess) {
                        ok = false;
                        break;
                    }
                    cudaStream_t main_stream = ctx->stream;
                    ctx->stream = side;
                    st = msp_sketch_sym_blocks(ctx, (const float*)A, n, n, sp, sk->csr_ptr, sk->csr_ent, gamma,
                                               (float*)sk->C, pack ? sk->packed : nullptr, ib0, ib1);
                    ctx->stream = main_stream;
                } else {
                    st = msp_sketch_sym_blocks(ctx, (const float*)A, n, n, sp, sk->csr_ptr, sk->csr_ent, gamma,
                                               (float*)sk->C, pack ? sk->packed : nullptr, ib0, ib1);
                }
                if (st != MSP_OK) {
                    ok = false;
                    break;
                }
                continue;
            }
            if (half && (st = msp_mirror_lower_rows(ctx, (float*)A, n, n, r0 / 128, (r0 + nr + 127) / 128)) != MSP_OK) {
                ok = false;
                break;
            }
            if ((st = msp_sketch_apply_rows(ctx, (const char*)A + (size_t)r0 * n * ts, dtype, nr, n, n, sp,
                                            sk->csr_ptr, sk->csr_ent, gamma, (char*)sk->C + (size_t)r0 * sp * ts)) !=
                    MSP_OK ||
                (sk->packed && (st = msp_pack_upper_rows(ctx, (const float*)A, n, n, r0 / 128, (r0 + nr + 127) / 128,
                                                         sk->packed)) != MSP_OK))
                ok = false;
        }
        if (ok && one_pass) {
            // every row has landed and every lower tile is mirrored: the row
            // statistics on the main stream, beside the side stream's last
            // sketch launches, then the join
            if (pack) st = msp_norm_lb_launch(ctx, A, dtype, n, n, sk->stats, sk->stats + 3 * n);
            if (st == MSP_OK && side &&
                (cudaEventRecord(ctx->aux_ev[1], side) != cudaSuccess ||
                 cudaStreamWaitEvent(ctx->stream, ctx->aux_ev[1], 0) != cudaSuccess))
                st = msp_set_error(ctx, MSP_ECUDA, "sketch: side stream join failed");
            ok = (st == MSP_OK);
            prep_done = true;
        }
        if (!ok && st == MSP_OK) {
            cudaGetLastError();
            st = msp_set_error(ctx, MSP_ECUDA, "sketch: chunked copy failed");
        }
        // (destroying a pending event is safe: its resources go once it completes)
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (ready) cudaEventDestroy(ready);
        if (st != MSP_OK) {
            cudaStreamSynchronize(ctx->copy_stream);
            if (side) cudaStreamSynchronize(side);
            cudaStreamSynchronize(ctx->stream);
            msp_sketch_destroy(sk);
            return st;
        }
    } else if (a_dt == MSP_F32 && ctx->sketch_sym && msp_sketch_sym_ok(A, n, lda, sp, gamma)) {
        // one pass over the symmetric A: C and the packed tiles together;
        // the norm-bound row statistics are a pass of their own
        if (pack) st = msp_alloc(ctx, (void**)&sk->stats, (size_t)(3 * n + 1) * 8);
        if (st == MSP_OK)
            st = sym_pass_and_stats(ctx, (const float*)A, dtype, n, lda, sp, sk->csr_ptr, sk->csr_ent, gamma,
                                    (float*)sk->C, pack ? sk->packed : nullptr, pack ? sk->stats : nullptr);
        if (st != MSP_OK) {
            cudaStreamSynchronize(ctx->stream);
            msp_sketch_destroy(sk);
            return st;
        }
        prep_done = true;
    } else if ((st = msp_sketch_apply(ctx, A, a_dt, n, lda, sp, sk->csr_ptr, sk->csr_ent, gamma, sk->C)) !=
               MSP_OK) {
        cudaStreamSynchronize(ctx->stream);
        msp_sketch_destroy(sk);
        return st;
    }
    if (pack && !prep_done &&
        (st = sketch_solve_prep(ctx, sk, A, dtype, host_chunks ? n : lda, !host_chunks)) != MSP_OK) {
        cudaStreamSynchronize(ctx->stream);
        msp_sketch_destroy(sk);
        return st;
    }
    sk->A_src = pack ? A : nullptr;
    *out = sk;
    return MSP_OK;
}

extern "C" {

msp_status msp_sketch(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda,
                      int64_t s, int gamma, uint64_t seed, msp_sketch_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !out) return msp_set_error(ctx, MSP_EINVAL, "sketch: NULL argument");
    DeviceGuard g(ctx->device);
    *out = nullptr;
    return msp_sketch_impl(ctx, A, dtype, n, lda, s, gamma, seed, true, out, nullptr);
}

msp_status msp_sketch_info(const msp_sketch_t* sk, int64_t* n, int64_t* s, int64_t* s_pad,
                           int* gamma, int* dtype) {
    if (!sk) return msp_set_error(nullptr, MSP_EINVAL, "sketch is NULL");
    if (n) *n = sk->n;
    if (s) *s = sk->s;
    if (s_pad) *s_pad = sk->s_pad;
    if (gamma) *gamma = sk->gamma;
    if (dtype) *dtype = sk->dtype;
    return MSP_OK;
}

msp_status msp_sketch_get_C(msp_ctx* ctx, const msp_sketch_t* sk, void* C, int64_t ldc) {
    if (!ctx || !sk || !C || ldc < sk->s) return msp_set_error(ctx, MSP_EINVAL, "get_C: bad argument");
    DeviceGuard g(ctx->device);
    const size_t ts = dtype_size(sk->dtype);
    MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(C, ldc * ts, sk->C, sk->s_pad * ts, sk->s * ts, sk->n,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

// --------------------------------------------------------------- a3-a5

void msp_factor_destroy(msp_factor_t* f) {
    if (!f) return;
    for (void* p : {f->W, f->B, f->Bt, (void*)f->W64, (void*)f->M2, (void*)f->Linv64, f->Cb, f->Wb})
        if (p) cudaFreeAsync(p, f->stream);
    delete f;
}

}  // extern "C"

namespace {

// Cb = bf16(C) (round to nearest even) and Cr = float(Cb), n x s_pad.
__global__ void k_round_bf16(const float* __restrict__ C, int64_t len, __nv_bfloat16* __restrict__ Cb,
                             float* __restrict__ Cr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const __nv_bfloat16 v = __float2bfloat16_rn(C[e]);
    if (Cb) Cb[e] = v;
    if (Cr) Cr[e] = __bfloat162float(v);
}

}  // namespace

msp_status msp_nystrom_impl(msp_ctx* ctx, const msp_sketch_s* sk, double lambda, double lambda0,
                            int64_t phi, int gamma_phi, uint64_t seed, msp_factor_t** out, msp_dtype data) {
    if (!(lambda > 0.0) || !(lambda0 >= 0.0) || !std::isfinite(lambda) || !std::isfinite(lambda0))
        return msp_set_error(ctx, MSP_EINVAL, "nystrom: need lambda > 0 and lambda0 >= 0");
    if (data != MSP_F32 && !(data == MSP_BF16 && sk->dtype == MSP_F32))
        return msp_set_error(ctx, MSP_EINVAL, "nystrom: preconditioner data must be MSP_F32, or MSP_BF16 for an "
                                              "FP32 sketch");
    if (sk->dtype == MSP_F64) data = MSP_F32;
    if (phi < 0 || (phi > 0 && (gamma_phi < 1 || gamma_phi > MSP_MAX_GAMMA || gamma_phi > phi ||
                                phi >= (1ll << 30))))
        return msp_set_error(ctx, MSP_EINVAL, "nystrom: need phi >= 0 and 1 <= gamma_phi <= min(phi, %d)",
                             MSP_MAX_GAMMA);
    const int64_t n = sk->n, sp = sk->s_pad;
    const size_t ts = dtype_size(sk->dtype);
    msp_factor_s* f = new (std::nothrow) msp_factor_s();
    if (!f) return msp_set_error(ctx, MSP_ENOMEM, "nystrom: host allocation failed");
    f->sk = sk; f->s = sk->s; f->s_pad = sp; f->phi = phi; f->dtype = sk->dtype;
    f->stream = ctx->stream;
    f->lambda = lambda; f->lambda0 = lambda0; f->lam_tilde = lambda + lambda0;
    f->data = (sk->dtype == MSP_F32) ? data : MSP_F32;
    const size_t mat_t = (size_t)sp * sp * ts, mat_d = (size_t)sp * sp * 8;
    msp_status st = MSP_OK;
    void* phi_mem = nullptr;
    float* Cr = nullptr;         // BF16 data: float(bf16(C)), the C every later step uses
    auto fail = [&](msp_status s2) {
        cudaStreamSynchronize(ctx->stream);
        if (phi_mem) free_on(ctx, phi_mem);
        if (Cr) free_on(ctx, Cr);
        msp_factor_destroy(f);
        return s2;
    };
    const void* Csrc = sk->C;
    if (f->data == MSP_BF16) {
        const int64_t len = n * sp;
        if ((st = msp_alloc(ctx, &f->Cb, (size_t)len * 2)) != MSP_OK ||
            (st = msp_alloc(ctx, &f->Wb, (size_t)sp * sp * 2)) != MSP_OK ||
            (st = msp_alloc(ctx, (void**)&Cr, (size_t)len * 4)) != MSP_OK)
            return fail(st);
        k_round_bf16<<<(unsigned)((len + 255) / 256), 256, 0, ctx->stream>>>((const float*)sk->C, len,
                                                                            (__nv_bfloat16*)f->Cb, Cr);
        MSP_CHECK_LAUNCH(ctx);
        Csrc = Cr;
    }
    if ((st = msp_alloc(ctx, &f->W, mat_t)) != MSP_OK || (st = msp_alloc(ctx, &f->B, mat_t)) != MSP_OK ||
        (st = msp_alloc(ctx, &f->Bt, mat_t)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&f->W64, mat_d)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&f->M2, mat_d)) != MSP_OK ||
        (st = msp_alloc(ctx, (void**)&f->Linv64, mat_d)) != MSP_OK)
        return fail(st);
    // W = S C = Pi^T C: row c of W gathers the rows j of C listed for column c
    const double sc = 1.0 / std::sqrt((double)sk->gamma);
    if ((st = msp_gather_rows(ctx, sk->dtype, sp, sp, sk->csr_ptr, sk->csr_ent, Csrc, sp, sc, f->W,
                              sp)) != MSP_OK)
        return fail(st);
    const void* Ct = Csrc;
    int64_t phi_rows = n;
    if (phi > 0) {
        // Phi: phi x n sparse embedding (stream 2); C~ = Phi C
        size_t b_idx = round_up((int64_t)n * gamma_phi * 4, 256);
        size_t b_sgn = round_up((int64_t)n * gamma_phi, 256);
        size_t b_ptr = round_up((phi + 1) * 4, 256);
        size_t b_ent = round_up((int64_t)n * gamma_phi * 4, 256);
        size_t b_ct = (size_t)phi * sp * ts;
        if ((st = msp_alloc(ctx, &phi_mem, b_idx + b_sgn + b_ptr + b_ent + b_ct)) != MSP_OK)
            return fail(st);
        char* c = (char*)phi_mem;
        int32_t* pidx = (int32_t*)c; c += b_idx;
        int8_t* psgn = (int8_t*)c; c += b_sgn;
        int32_t* pptr = (int32_t*)c; c += b_ptr;
        int32_t* pent = (int32_t*)c; c += b_ent;
        void* ct = c;
        if ((st = msp_pattern_launch(ctx, n, phi, gamma_phi, seed, 2, pidx, psgn, nullptr)) != MSP_OK ||
            (st = msp_build_csr(ctx, n, phi, gamma_phi, pidx, psgn, pptr, pent)) != MSP_OK ||
            (st = msp_gather_rows(ctx, sk->dtype, phi, sp, pptr, pent, Csrc, sp,
                                  1.0 / std::sqrt((double)gamma_phi), ct, sp)) != MSP_OK)
            return fail(st);
        Ct = ct;
        phi_rows = phi;
    }
    if ((st = msp_build_factor(ctx, f, Ct, phi_rows)) != MSP_OK) return fail(st);
    if (f->data == MSP_BF16) {
        // Wb = bf16 of the symmetrised W (for the iterative level 2)
        k_round_bf16<<<(unsigned)((sp * sp + 255) / 256), 256, 0, ctx->stream>>>((const float*)f->W, sp * sp,
                                                                                (__nv_bfloat16*)f->Wb, nullptr);
        MSP_CHECK_LAUNCH(ctx);
    }
    if (phi_mem) free_on(ctx, phi_mem);
    if (Cr) free_on(ctx, Cr);
    *out = f;
    return MSP_OK;
}

extern "C" {

msp_status msp_nystrom(msp_ctx* ctx, const msp_sketch_t* sk, double lambda, double lambda0,
                       int64_t phi, int gamma_phi, uint64_t seed, msp_factor_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!sk || !out) return msp_set_error(ctx, MSP_EINVAL, "nystrom: NULL argument");
    DeviceGuard g(ctx->device);
    *out = nullptr;
    return msp_nystrom_impl(ctx, sk, lambda, lambda0, phi, gamma_phi, seed, out);
}

msp_status msp_nystrom_ex(msp_ctx* ctx, const msp_sketch_t* sk, double lambda, double lambda0, int64_t phi,
                          int gamma_phi, uint64_t seed, msp_dtype data, msp_factor_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!sk || !out) return msp_set_error(ctx, MSP_EINVAL, "nystrom: NULL argument");
    DeviceGuard g(ctx->device);
    *out = nullptr;
    return msp_nystrom_impl(ctx, sk, lambda, lambda0, phi, gamma_phi, seed, out, data);
}

msp_status msp_factor_get(msp_ctx* ctx, const msp_factor_t* f, double* W, double* M2, double* Linv,
                          double* lam_tilde, double* shift, int* retries) {
    if (!ctx || !f) return msp_set_error(ctx, MSP_EINVAL, "factor_get: NULL argument");
    DeviceGuard g(ctx->device);
    const int64_t s = f->s, sp = f->s_pad;
    if (W) MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(W, s * 8, f->W64, sp * 8, s * 8, s,
                                               cudaMemcpyDeviceToDevice, ctx->stream));
    if (M2) MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(M2, s * 8, f->M2, sp * 8, s * 8, s,
                                                cudaMemcpyDeviceToDevice, ctx->stream));
    if (Linv) MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(Linv, s * 8, f->Linv64, sp * 8, s * 8, s,
                                                  cudaMemcpyDeviceToDevice, ctx->stream));
    if (lam_tilde) *lam_tilde = f->lam_tilde;
    if (shift) *shift = f->shift;
    if (retries) *retries = f->retries;
    return MSP_OK;
}

msp_status msp_solve_m1(msp_ctx* ctx, const msp_factor_t* f, const void* r, void* w,
                        const msp_opts* opts, int* inner_iters) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!f || !r || !w) return msp_set_error(ctx, MSP_EINVAL, "solve_m1: NULL argument");
    DeviceGuard g(ctx->device);
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    return msp_solve_m1_impl(ctx, f, r, w, &o, inner_iters);
}

// --------------------------------------------------------------- a6-a8

// A is the matrix the level-1 iteration applies (the factor's working
// precision); Ares (dtype dres, ld ldres) the matrix of the FP64 refinement
// residual and of the backward-error bound, A itself unless the caller gives
// the problem's FP64 matrix beside a reduced working copy.
static msp_status solve_impl(msp_ctx* ctx, const msp_factor_s* f, const void* A, msp_dtype dtype,
                             int64_t n, int64_t lda, double lambda, const double* b, double* x,
                             const msp_opts* o, msp_info* info, const void* Ares = nullptr,
                             msp_dtype dres = MSP_F64, int64_t ldres = 0) {
    if (!Ares) {
        Ares = A;
        dres = dtype;
        ldres = lda;
    }
    msp_info inf{};
    inf.lambda_tilde = f->lam_tilde;
    inf.shift = f->shift;
    inf.shift_retries = f->retries;
    if (n != f->sk->n || lda < n)
        return msp_set_error(ctx, MSP_EINVAL, "solve: n does not match the factor, or lda < n");
    if (!(lambda > 0.0) || !std::isfinite(lambda))
        return msp_set_error(ctx, MSP_EINVAL, "solve: need lambda > 0");
    const int prec = o->precision;
    if (prec == MSP_PREC_FP64) {
        if (dtype != MSP_F64 || f->dtype != MSP_F64)
            return msp_set_error(ctx, MSP_EINVAL, "solve: MSP_PREC_FP64 needs an FP64 A and factor");
    } else if (prec == MSP_PREC_FP32 || prec == MSP_PREC_MIXED) {
        if (dtype != MSP_F32 || f->dtype != MSP_F32)
            return msp_set_error(ctx, MSP_EINVAL, "solve: FP32/MIXED precision needs an FP32 A and factor");
    } else {
        return msp_set_error(ctx, MSP_EINVAL, "solve: unknown precision %d", prec);
    }
    if (!(o->tol > 0.0) || o->max_outer < 1 || o->max_inner < 0 || o->max_refine < 0)
        return msp_set_error(ctx, MSP_EINVAL, "solve: bad options");
    const msp_dtype wt = f->dtype;
    const size_t ts = dtype_size(wt);
    // the sketch's packed upper tiles and norm-bound statistics stand in for A
    // when A is the sketched matrix
    const bool sketched_A = (A == f->sk->A_src);
    const bool same_res = (Ares == A);
    if (ldres < n) return msp_set_error(ctx, MSP_EINVAL, "solve: residual matrix leading dimension < n");
    const float* packed = (dtype == MSP_F32 && f->sk->packed && sketched_A) ? f->sk->packed : nullptr;
    if (o->criterion != MSP_STOP_RESIDUAL && o->criterion != MSP_STOP_BACKWARD)
        return msp_set_error(ctx, MSP_EINVAL, "solve: unknown criterion %d", o->criterion);
    const bool crit_bw = o->criterion == MSP_STOP_BACKWARD;
    // per-solve buffers: r64 (n), rhs_w (n), sol_w (n), scalars, |A| bound work
    void* mem = nullptr;
    size_t b_r = round_up(n * 8, 256), b_w = round_up(n * ts, 256);
    const size_t b_nw = crit_bw ? (size_t)round_up(3 * n * 8, 256) : 0;
    MSP_TRY(msp_alloc(ctx, &mem, b_r + 2 * b_w + 256 + b_nw));
    char* c = (char*)mem;
    double* r64 = (double*)c; c += b_r;
    void* rhs_w = c; c += b_w;
    void* sol_w = c; c += b_w;
    double* scal = (double*)c;    // [0] |b|^2, [1] |r|^2, [2] L <= |A|_2, [3] |x|^2
    double* nwork = (double*)(c + 256);
    double* hs = (double*)ctx->host_flags + 8;
    msp_status st = MSP_OK;
    int outer_total = 0, inner_total = 0, steps = 0;
    double bb = 0.0, rr = 0.0;
    ProfSlot slots[3];
    Profiler pr;
    pr.ctx = ctx;
    pr.on = o->profile != 0;
    if (pr.on) MSP_TRY(msp_profiler_reserve(ctx, 4096));
    const int64_t graph_iters0 = ctx->l1_graph_iters;
    auto finish = [&](msp_status s2) {
        cudaStreamSynchronize(ctx->stream);
        inf.level1_graph_iters = (int)(ctx->l1_graph_iters - graph_iters0);
        if (pr.on) {
            inf.gemv_launches = slots[0].launches;
            inf.gemv_ms = slots[0].ms;
            inf.level2_launches = slots[1].launches;
            inf.level2_ms = slots[1].ms;
            inf.resid_launches = slots[2].launches;
            inf.resid_ms = slots[2].ms;
        }
        free_on(ctx, mem);
        inf.outer_iters = outer_total;
        inf.inner_iters = inner_total;
        inf.refine_steps = steps;
        inf.status = s2;
        if (info) *info = inf;
        return s2;
    };
    double Lb = 0.0, xx = 0.0;
    auto read2 = [&](double* a0, double* a1) -> msp_status {
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hs, scal, 32, cudaMemcpyDeviceToHost, ctx->stream));
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        *a0 = hs[0];
        *a1 = hs[1];
        Lb = hs[2];
        xx = hs[3];
        return MSP_OK;
    };
    // the stopping rule of the solve
    auto met = [&]() {
        if (crit_bw) return std::sqrt(rr) <= o->tol * ((Lb + lambda) * std::sqrt(xx) + std::sqrt(bb));
        return rr <= o->tol * o->tol * bb;
    };
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(scal, 0, 32, ctx->stream));
    if (crit_bw && sketched_A && same_res && f->sk->stats) {
        if (cudaMemcpyAsync(scal + 2, f->sk->stats + 3 * n, 8, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return finish(msp_set_error(ctx, MSP_ECUDA, "solve: norm bound copy failed"));
        }
    } else if (crit_bw && (st = msp_norm_lb_launch(ctx, Ares, dres, n, ldres, nwork, scal + 2)) != MSP_OK) {
        return finish(st);
    }
    if ((st = msp_norm2(ctx, b, n, scal + 0)) != MSP_OK) return finish(st);
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(r64, b, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(scal + 1, scal + 0, 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((st = read2(&bb, &rr)) != MSP_OK) return finish(st);
    inf.norm_lb = Lb;
    if (!std::isfinite(bb)) return finish(msp_set_error(ctx, MSP_ENONFINITE, "solve: b is not finite"));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, n * 8, ctx->stream));
    if (bb == 0.0) {
        inf.rel_resid = 0.0;
        return finish(MSP_OK);
    }
    // MIXED: every correction solve to refine_tol. FP64: the first solve to
    // tol; its recurrence residual can drift from the true one, so further
    // steps correct from the FP64 residual, each asked for just the remaining
    // factor (with a margin of 2). FP32: one solve.
    const int max_steps = (prec == MSP_PREC_FP32) ? 1 : o->max_refine + 1;
    const double mixed_tol = std::max(o->refine_tol, o->tol);
    msp_status kst = MSP_OK;
    bool have_resid = true;   // r64 / rr hold the residual of the current x (x = 0: r = b)
    for (int k = 0; k < max_steps; ++k) {
        if (!have_resid) {
            // r = b - (A + lam I) x, FP64 accumulation
            if ((st = pr.begin(0)) != MSP_OK) return finish(st);
            if ((st = msp_matvec64(ctx, Ares, dres, n, ldres, lambda, x, b, r64, scal + 1, prec == MSP_PREC_FP64)) != MSP_OK)
                return finish(st);
            if ((st = pr.end()) != MSP_OK) return finish(st);
            if ((st = pr.finish(&slots[2], 1)) != MSP_OK) return finish(st);
            if (crit_bw && (st = msp_norm2(ctx, x, n, scal + 3)) != MSP_OK) return finish(st);
            if ((st = read2(&bb, &rr)) != MSP_OK) return finish(st);
            if (!std::isfinite(rr))
                return finish(msp_set_error(ctx, MSP_ENONFINITE, "solve: residual is not finite"));
            have_resid = true;
        }
        if (met()) break;
        double step_tol = o->tol;
        if (prec == MSP_PREC_MIXED) step_tol = mixed_tol;
        else if (prec == MSP_PREC_FP64 && k > 0)
            step_tol = std::min(0.5, std::max(o->tol, 0.5 * o->tol * std::sqrt(bb / rr)));
        // correction solve on the normalised residual: (A + lam I) d = r / |r|
        if ((st = msp_scale_cast(ctx, r64, scal + 1, n, wt, rhs_w)) != MSP_OK) return finish(st);
        int it = 0, in = 0;
        kst = msp_krylov_solve(ctx, f, A, dtype, n, lda, lambda, rhs_w, sol_w, step_tol,
                               o->max_outer, o, &it, &in, pr.on ? slots : nullptr, packed);
        outer_total += it;
        inner_total += in;
        if (kst != MSP_OK && kst != MSP_ENOCONV) return finish(kst);
        if ((st = msp_axpy_back(ctx, x, sol_w, wt, scal + 1, n, k > 0)) != MSP_OK) return finish(st);
        steps = k + 1;
        have_resid = false;
        if (prec == MSP_PREC_FP32) break;
    }
    if (!have_resid) {
        if ((st = pr.begin(0)) != MSP_OK) return finish(st);
        if ((st = msp_matvec64(ctx, Ares, dres, n, ldres, lambda, x, b, r64, scal + 1, prec == MSP_PREC_FP64)) != MSP_OK)
            return finish(st);
        if ((st = pr.end()) != MSP_OK) return finish(st);
        if ((st = pr.finish(&slots[2], 1)) != MSP_OK) return finish(st);
        if (crit_bw && (st = msp_norm2(ctx, x, n, scal + 3)) != MSP_OK) return finish(st);
        if ((st = read2(&bb, &rr)) != MSP_OK) return finish(st);
    }
    inf.rel_resid = std::sqrt(rr / bb);
    if (crit_bw) inf.backward_err = std::sqrt(rr) / ((Lb + lambda) * std::sqrt(xx) + std::sqrt(bb));
    if (!met() && prec != MSP_PREC_FP32)
        return finish(msp_set_error(ctx, MSP_ENOCONV,
                                    "solve: relative residual %.3e (backward error bound %.3e) "
                                    "above tol %.3e after %d steps",
                                    inf.rel_resid, inf.backward_err, o->tol, steps));
    if (kst == MSP_ENOCONV) return finish(kst);
    return finish(MSP_OK);
}

msp_status msp_solve(msp_ctx* ctx, const msp_factor_t* f, const void* A, msp_dtype dtype, int64_t n,
                     int64_t lda, double lambda, const double* b, double* x, const msp_opts* opts,
                     msp_info* info) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!f || !A || !b || !x) return msp_set_error(ctx, MSP_EINVAL, "solve: NULL argument");
    DeviceGuard g(ctx->device);
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    return solve_impl(ctx, f, A, dtype, n, lda, lambda, b, x, &o, info);
}

msp_status msp_set_grid_wait_limit(msp_ctx* ctx, double seconds) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!(seconds >= 0.0) || seconds > 60.0)
        return msp_set_error(ctx, MSP_EINVAL, "grid wait limit must be in [0, 60] s (0: the default)");
    DeviceGuard g(ctx->device);
    const unsigned long long ns = (unsigned long long)(seconds * 1e9);
    return msp_grid_wait_limit_krylov(ctx, seconds > 0.0 && ns == 0 ? 1ull : ns);
}

msp_status msp_solve_refined(msp_ctx* ctx, const msp_factor_t* f, const void* A, msp_dtype dtype,
                             int64_t n, int64_t lda, const void* A_res, msp_dtype res_dtype, int64_t ld_res,
                             double lambda, const double* b, double* x, const msp_opts* opts, msp_info* info) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!f || !A || !A_res || !b || !x) return msp_set_error(ctx, MSP_EINVAL, "solve_refined: NULL argument");
    if (res_dtype != MSP_F64 && res_dtype != MSP_F32)
        return msp_set_error(ctx, MSP_EINVAL, "solve_refined: residual matrix must be MSP_F64 or MSP_F32");
    DeviceGuard g(ctx->device);
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    return solve_impl(ctx, f, A, dtype, n, lda, lambda, b, x, &o, info, A_res, res_dtype, ld_res);
}

msp_status msp_solve_many(msp_ctx* ctx, const msp_factor_t* f, const void* A, msp_dtype dtype, int64_t n,
                          int64_t lda, double lambda, const double* B, int64_t ldb, double* X, int64_t ldx,
                          int64_t m, const msp_opts* opts, msp_info* infos) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!f || !A || (m > 0 && (!B || !X)) || m < 0 || ldb < n || ldx < n)
        return msp_set_error(ctx, MSP_EINVAL, "solve_many: NULL argument, m < 0, or ldb / ldx < n");
    DeviceGuard g(ctx->device);
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    // every column is its own run of Algorithm 1 step 5 with the shared factor
    msp_status worst = MSP_OK;
    for (int64_t j = 0; j < m; ++j) {
        msp_info inf;
        const msp_status st = solve_impl(ctx, f, A, dtype, n, lda, lambda, B + j * ldb, X + j * ldx, &o, &inf);
        if (infos) infos[j] = inf;
        if (st != MSP_OK && st != MSP_ENOCONV) return st;
        if (st == MSP_ENOCONV) worst = MSP_ENOCONV;
    }
    if (worst == MSP_ENOCONV) return msp_set_error(ctx, MSP_ENOCONV, "solve_many: a column did not converge");
    return MSP_OK;
}

msp_status msp_solve_full(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda,
                          double lambda, const double* b, double* x, int64_t s, int gamma,
                          double lambda0, int64_t phi, int gamma_phi, uint64_t seed,
                          const msp_opts* opts, msp_info* info) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !b || !x) return msp_set_error(ctx, MSP_EINVAL, "solve_full: NULL argument");
    if (n < 1 || lda < n) return msp_set_error(ctx, MSP_EINVAL, "solve_full: need lda >= n >= 1");
    DeviceGuard g(ctx->device);
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    const size_t ts = dtype_size(dtype);
    const bool dA = is_device_ptr(A), db = is_device_ptr(b), dx = is_device_ptr(x);
    size_t need = (dA ? 0 : round_up(n * n * ts, 256)) + (db ? 0 : round_up(n * 8, 256)) +
                  (dx ? 0 : round_up(n * 8, 256));
    const void* Ad = A;
    const double* bd = b;
    double* xd = x;
    int64_t ldd = lda;
    // a host A is copied in row chunks overlapped with the sketch and the
    // packing (which read only the chunk's rows)
    const bool chunked = !dA;
    if (need) {
        MSP_TRY(stage_alloc(ctx, need));
        char* c = (char*)ctx->stage;
        if (!dA) {
            Ad = c;
            ldd = n;
            c += round_up(n * n * ts, 256);
        }
        if (!db) {
            MSP_CUDA_TRY(ctx, cudaMemcpyAsync(c, b, n * 8, cudaMemcpyHostToDevice, ctx->stream));
            bd = (const double*)c;
            c += round_up(n * 8, 256);
        }
        if (!dx) xd = (double*)c;
    }
    msp_sketch_t* sk = nullptr;
    msp_factor_t* f = nullptr;
    msp_status st = msp_sketch_impl(ctx, Ad, dtype, n, chunked ? lda : ldd, s, gamma, seed, true, &sk,
                                    chunked ? A : nullptr);
    if (st == MSP_OK) st = msp_nystrom_impl(ctx, sk, lambda, lambda0, phi, gamma_phi, seed, &f);
    msp_status st2 = MSP_OK;
    if (st == MSP_OK) st2 = solve_impl(ctx, f, Ad, dtype, n, ldd, lambda, bd, xd, &o, info);
    if (st == MSP_OK && (st2 == MSP_OK || st2 == MSP_ENOCONV) && !dx) {
        cudaError_t e = cudaMemcpyAsync(x, xd, n * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st2 = msp_set_error(ctx, MSP_ECUDA, "solve_full: copy-out failed");
    }
    cudaStreamSynchronize(ctx->stream);
    msp_factor_destroy(f);
    msp_sketch_destroy(sk);
    return st != MSP_OK ? st : st2;
}

msp_status msp_matvec_f64(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda,
                          double lambda, const double* x, double* y) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !x || !y || n < 1 || lda < n)
        return msp_set_error(ctx, MSP_EINVAL, "matvec: bad argument");
    DeviceGuard g(ctx->device);
    return msp_matvec64(ctx, A, dtype, n, lda, lambda, x, nullptr, y, nullptr);
}

}  // extern "C"
