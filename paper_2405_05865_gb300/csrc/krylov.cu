// Level-1 and level-2 iterations of MSP on sm_103a (Algorithm 1 step 5 and
// Algorithm 2).
//
// One level-1 (outer) iteration is two launches:
//   k_gemv      q = (A + lam I) p, one pass over A, with the dot p^T q fused;
//               the last block to finish forms alpha = (r^T z) / (p^T q).
//   k_level2    persistent cooperative kernel: x += alpha p, r -= alpha q,
//               convergence test on |r|, then SolveM1(r) (Algorithm 2):
//               g = C^T r; level-2 PCG on (C^T C + lam~ W) y = g
//               preconditioned by M2^{-1} v = B^T (B v); w = (r - C y)/lam~;
//               finally the flexible (Polak-Ribiere) beta and p = w + beta p.
// Level-2 vectors (length s) are held redundantly in every block's shared
// memory; every block computes the same scalars from the same partial sums
// in the same order, so all blocks take identical branches and the number of
// grid barriers always matches. Reductions use fixed orders (deterministic).
#include "msp_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace {

constexpr int kNW = 8;             // warps per block in k_level2
constexpr int kThreads = kNW * 32;

enum { MODE_INIT = 0, MODE_ITER = 1, MODE_APPLY = 2 };

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T>
__device__ inline void load16(const T* p, T* out) {
    typename Vec16<T>::type v = *reinterpret_cast<const typename Vec16<T>::type*>(p);
    if constexpr (Vec16<T>::W == 4) { out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w; }
    else { out[0] = v.x; out[1] = v.y; }
}

// One vector load of a row slice: 16 bytes of FP32 / FP64, or 8 bytes of
// BF16 (4 values, widened to FP32 exactly), so that every storage type puts
// the same 4 (FP64: 2) consecutive values in each lane step.
template <typename T>
__device__ inline void load_vec(const T* p, T* out) { load16(p, out); }
__device__ inline void load_vec(const __nv_bfloat16* p, float* out) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    out[0] = __uint_as_float(v.x << 16);
    out[1] = __uint_as_float(v.x & 0xFFFF0000u);
    out[2] = __uint_as_float(v.y << 16);
    out[3] = __uint_as_float(v.y & 0xFFFF0000u);
}

// Values per vector load of a storage type.
template <typename TS> struct StoreW { static constexpr int W = 16 / (int)sizeof(TS); };
template <> struct StoreW<__nv_bfloat16> { static constexpr int W = 4; };

// Streaming (evict-first) 16-byte load: A is read once per pass, so it should
// not displace the sketch C, which the level-2 iteration re-reads from L2.
template <typename T>
__device__ inline void load16_stream(const T* p, T* out) {
    typename Vec16<T>::type v = __ldcs(reinterpret_cast<const typename Vec16<T>::type*>(p));
    if constexpr (Vec16<T>::W == 4) { out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w; }
    else { out[0] = v.x; out[1] = v.y; }
}

// Deterministic block-wide sum of one double per thread (all threads get it).
__device__ inline double block_sum(double v, double* red) {
    v = msp::warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) t += red[k];
    return t;
}

// Sum of a per-block partial array in fixed order (all threads get it).
__device__ inline double sum_parts(const double* parts, int stride, int G, double* red) {
    double v = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) v += __ldcg(&parts[(int64_t)k * stride]);
    return block_sum(v, red);
}

// Two block sums at once (red holds 64 doubles): per value the order of
// block_sum, with one pair of barriers.
__device__ inline void block_sum2(double& v0, double& v1, double* red) {
    v0 = msp::warp_sum(v0);
    v1 = msp::warp_sum(v1);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[w] = v0;
        red[32 + w] = v1;
    }
    __syncthreads();
    double t0 = 0.0, t1 = 0.0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) {
        t0 += red[k];
        t1 += red[32 + k];
    }
    v0 = t0;
    v1 = t1;
}

// sum_parts of the entries at offsets o0 and o1 of every block's record.
__device__ inline void sum_parts2(const double* parts, int stride, int G, double* red, double& s0, double& s1) {
    double v0 = 0.0, v1 = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        v0 += __ldcg(&parts[(int64_t)k * stride]);
        v1 += __ldcg(&parts[(int64_t)k * stride + 1]);
    }
    block_sum2(v0, v1, red);
    s0 = v0;
    s1 = v1;
}

// ------------------------------------------------------------------ GEMV

// q = (A + lam I) p; warp per row (grid-stride); lane reads 16 B vectors.
// The block partials of p^T q are combined by the last block, which writes
// ctl->pq and ctl->alpha = ctl->rz / pq (or flags an error).
template <typename TA, typename T, bool VEC>
__global__ void __launch_bounds__(256) k_gemv(const TA* __restrict__ A, int64_t lda, int64_t n,
                                             double lam, const T* __restrict__ p,
                                             T* __restrict__ q, double* __restrict__ part,
                                             CtlBlock* ctl) {
    if (ctl->done | ctl->error) return;
    __shared__ double red[32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double pq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
         i += warps) {
        const TA* row = A + i * lda;
        T acc = T(0);
        if constexpr (VEC) {
            constexpr int W = Vec16<TA>::W;
            int64_t j = (int64_t)lane * W;
            // 4 independent 16 B loads in flight per lane
            for (; j + 3 * 32 * W < n; j += 4 * 32 * W) {
                TA a[4][W];
                T pv[4][W];
#pragma unroll
                for (int u = 0; u < 4; ++u) load16_stream(row + j + u * 32 * W, a[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int e = 0; e < W; ++e) pv[u][e] = p[j + u * 32 * W + e];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int e = 0; e < W; ++e) acc += (T)a[u][e] * pv[u][e];
            }
            for (; j < n; j += 32 * W) {
                TA a[W];
                load16_stream(row + j, a);
#pragma unroll
                for (int e = 0; e < W; ++e) acc += (T)a[e] * p[j + e];
            }
        } else {
            for (int64_t j = lane; j < n; j += 32) acc += (T)__ldcs(&row[j]) * p[j];
        }
        acc = msp::warp_sum(acc);
        if (lane == 0) {
            T qi = acc + (T)lam * p[i];
            q[i] = qi;
            pq += (double)p[i] * (double)qi;
        }
    }
    double tot = block_sum(pq, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();
        unsigned int t = atomicAdd(&ctl->last_block_counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double all = sum_parts(part, 1, gridDim.x, red);
    if (threadIdx.x == 0) {
        ctl->last_block_counter = 0;
        ctl->pq = all;
        if (!isfinite(all)) { ctl->error = MSP_ENONFINITE; }
        else if (!(all > 0.0)) { ctl->error = MSP_ENOTPD; }
        else ctl->alpha = ctl->rz / all;
    }
}

// Exact binary32 -> binary64 widening with integer instructions (the FP64
// pipe, which bounds the residual, then only executes the FMAs). Subnormal
// inputs are flushed to zero (their products are below 1e-37 |x|); infinities
// and NaNs keep their class.
__device__ inline double widen_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = u & 0x7f800000u;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    uint64_t bits;
    if (ex == 0u) bits = sign;                                               // zero / subnormal
    else if (ex == 0x7f800000u) bits = sign | 0x7ff0000000000000ull | ((uint64_t)(u & 0x007fffffu) << 29);
    else bits = sign | (((uint64_t)(u & 0x7fffffffu) << 29) + ((uint64_t)(1023 - 127) << 52));
    return __longlong_as_double((long long)bits);
}

// A entry widened to FP64 (exact for every storage type).
__device__ inline double wide64(double v) { return v; }
__device__ inline double wide64(float v) { return (double)v; }
__device__ inline double wide64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// out = b - (A + lam I) x  (or (A + lam I) x if b == nullptr), FP64
// accumulation; |out|^2 into *norm2 (last block, fixed order). The FP64 FMA
// rate bounds this kernel on this part (two FMAs per clock per SM): loads are
// vectorised (16 B of A, 32 B of x per lane step) and A is widened with
// integer instructions so that the FP64 pipe issues only the FMAs.
template <typename TA, bool VEC>
__global__ void __launch_bounds__(256) k_matvec64(const TA* __restrict__ A, int64_t lda, int64_t n,
                                                 double lam, const double* __restrict__ x,
                                                 const double* __restrict__ b,
                                                 double* __restrict__ out, double* __restrict__ part,
                                                 unsigned int* counter, double* norm2) {
    __shared__ double red[32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double nn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
         i += warps) {
        const TA* row = A + i * lda;
        double acc0 = 0.0, acc1 = 0.0;
        if constexpr (VEC && sizeof(TA) == 4) {
            int64_t j = (int64_t)lane * 4;
            for (; j + 32 * 4 < n; j += 2 * 32 * 4) {
                const float4 a0 = __ldcs(reinterpret_cast<const float4*>(row + j));
                const float4 a1 = __ldcs(reinterpret_cast<const float4*>(row + j + 128));
                const double2 x0 = *reinterpret_cast<const double2*>(x + j);
                const double2 x1 = *reinterpret_cast<const double2*>(x + j + 2);
                const double2 x2 = *reinterpret_cast<const double2*>(x + j + 128);
                const double2 x3 = *reinterpret_cast<const double2*>(x + j + 130);
                acc0 = fma(widen_f32(a0.x), x0.x, acc0);
                acc1 = fma(widen_f32(a1.x), x2.x, acc1);
                acc0 = fma(widen_f32(a0.y), x0.y, acc0);
                acc1 = fma(widen_f32(a1.y), x2.y, acc1);
                acc0 = fma(widen_f32(a0.z), x1.x, acc0);
                acc1 = fma(widen_f32(a1.z), x3.x, acc1);
                acc0 = fma(widen_f32(a0.w), x1.y, acc0);
                acc1 = fma(widen_f32(a1.w), x3.y, acc1);
            }
            for (; j < n; j += 32 * 4) {
                const float4 a0 = __ldcs(reinterpret_cast<const float4*>(row + j));
                acc0 = fma(widen_f32(a0.x), x[j], acc0);
                acc0 = fma(widen_f32(a0.y), x[j + 1], acc0);
                acc0 = fma(widen_f32(a0.z), x[j + 2], acc0);
                acc0 = fma(widen_f32(a0.w), x[j + 3], acc0);
            }
        } else {
            for (int64_t j = lane; j < n; j += 32) acc0 = fma(wide64(__ldcs(&row[j])), x[j], acc0);
        }
        double acc = msp::warp_sum(acc0 + acc1);
        if (lane == 0) {
            double v = acc + lam * x[i];
            if (b) v = b[i] - v;
            out[i] = v;
            nn += v * v;
        }
    }
    double tot = block_sum(nn, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double all = sum_parts(part, 1, gridDim.x, red);
    if (threadIdx.x == 0) {
        *counter = 0;
        if (norm2) *norm2 = all;
    }
}

// ---------------------------------------------------------- level 2

// TC: storage type of C and W (T, or BF16 preconditioner data with T = float)
template <typename T, typename TC = T>
struct L2Args {
    int64_t n, s_pad;
    int mode;
    const TC* C;
    const TC* W;
    const T* B;
    const T* Bt;
    T lam_t;
    double tol_rel2;        // level-1 tolerance^2 (MODE_INIT sets ctl->tol2)
    double inner_tol2;
    int max_inner;
    T* x;
    T* r;
    const T* q;
    T* p;
    T* z;                   // level-1 preconditioned residual (in/out)
    const float* qpart;     // packed A pass: q_i = sum_slot qpart[slot][i] + lam p_i
    int q_slots;
    int64_t q_ld;
    T lam;
    CtlBlock* ctl;
    T* part;                // G x s_pad
    T* gvec;                // s_pad
    T* uvec;
    T* tvec;
    T* zvec;
    T* wdvec;
    double* dpart;          // G x 4
};

// Per-lane slice of an s_pad row stored as TS: PL elements as PL/W vectors of
// W elements (one vector load each), element index of vector v, component
// e: v*32*W + lane*W + e; values held as T.
template <typename T, int PL, typename TS = T>
struct RowSlice {
    static constexpr int W = StoreW<TS>::W;
    static constexpr int NVEC = PL / W;
    T v[PL];
    __device__ inline void load(const TS* row, int lane) {
#pragma unroll
        for (int k = 0; k < NVEC; ++k) load_vec(row + k * 32 * W + lane * W, v + k * W);
    }
    __device__ inline T dot_smem(const T* s, int lane) const {
        T a = T(0);
#pragma unroll
        for (int k = 0; k < NVEC; ++k)
#pragma unroll
            for (int e = 0; e < W; ++e) a += v[k * W + e] * s[k * 32 * W + lane * W + e];
        return a;
    }
};

template <typename T, int PL, typename TS = T>
__device__ inline void store_slice(T* dst, const T* src, int lane) {
    constexpr int W = StoreW<TS>::W;
#pragma unroll
    for (int k = 0; k < PL / W; ++k)
#pragma unroll
        for (int e = 0; e < W; ++e) dst[k * 32 * W + lane * W + e] = src[k * W + e];
}

// Row pass over this block's rows of C.
//   kind 0: acc += r_i c_i                     (g = C^T r)
//   kind 1: acc += (c_i . d) c_i               (u = C^T C d)
//   kind 2: w_i = (r_i - c_i . y) / lam~; dots r.w and r.z_old  (no acc)
// Per-warp accumulators are combined through shared memory into part[b].
constexpr int kRowChunk = 256;   // rows of C staged per round (r, z, w in shared memory)

template <typename T, typename TC, int PL>
__device__ inline void row_one(const L2Args<T, TC>& a, int kind, int64_t il, const RowSlice<T, PL, TC>& c,
                               const T* svec, T* acc, const T* sr, T* sw, int lane) {
    T coef;
    if (kind == 0) {
        coef = sr[il];
    } else {
        T t = msp::warp_sum(c.dot_smem(svec, lane));
        if (kind == 1) {
            coef = t;
        } else {
            if (lane == 0) sw[il] = (sr[il] - t) / a.lam_t;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < PL; ++k) acc[k] += coef * c.v[k];
}

// Row pass over this block's rows of C, two rows in flight per warp, in
// chunks of kRowChunk rows whose r (and z_old, w) live in shared memory so no
// per-row global access sits on the critical path.
//   kind 0: acc += r_i c_i                     (g = C^T r)
//   kind 1: acc += (c_i . d) c_i               (u = C^T C d)
//   kind 2: w_i = (r_i - c_i . y) / lam~ into z; per-thread dots r.w, r.z_old
// Per-warp accumulators are combined through shared memory into part[b].
template <typename T, typename TC, int PL>
__device__ void row_pass(const L2Args<T, TC>& a, int kind, int64_t row0, int64_t row1, const T* svec,
                         T* swarp, T* srow, double* rw, double* rzo) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T* sr = srow;                 // kRowChunk
    T* sw = srow + kRowChunk;     // kRowChunk
    T acc[PL];
#pragma unroll
    for (int k = 0; k < PL; ++k) acc[k] = T(0);
    double d_rw = 0.0, d_rzo = 0.0;
    for (int64_t base = row0; base < row1; base += kRowChunk) {
        const int64_t end = min(row1, base + kRowChunk);
        const int nr = (int)(end - base);
        if (kind != 1) {
            for (int e = threadIdx.x; e < nr; e += blockDim.x) sr[e] = a.r[base + e];
            __syncthreads();
        }
        int il = w;
        for (; il + kNW < nr; il += 2 * kNW) {
            RowSlice<T, PL, TC> c0, c1;
            c0.load(a.C + (base + il) * a.s_pad, lane);
            c1.load(a.C + (base + il + kNW) * a.s_pad, lane);
            row_one<T, TC, PL>(a, kind, il, c0, svec, acc, sr, sw, lane);
            row_one<T, TC, PL>(a, kind, il + kNW, c1, svec, acc, sr, sw, lane);
        }
        if (il < nr) {
            RowSlice<T, PL, TC> c0;
            c0.load(a.C + (base + il) * a.s_pad, lane);
            row_one<T, TC, PL>(a, kind, il, c0, svec, acc, sr, sw, lane);
        }
        if (kind != 1) __syncthreads();
        if (kind == 2) {
            for (int e = threadIdx.x; e < nr; e += blockDim.x) {
                const T ri = sr[e], wi = sw[e];
                const T zo = a.z[base + e];
                d_rw += (double)ri * (double)wi;
                d_rzo += (double)ri * (double)zo;
                a.z[base + e] = wi;
            }
            __syncthreads();
        }
    }
    if (kind == 2) {
        *rw = d_rw;
        *rzo = d_rzo;
        return;
    }
    store_slice<T, PL, TC>(swarp + (int64_t)w * a.s_pad, acc, lane);
}

// Butterfly reduce-scatter: lane l ends with the sum over the 32 lanes of
// v[l] (31 shuffles, v overwritten).
template <typename T>
__device__ inline T reduce_scatter32(T* v, int lane) {
#pragma unroll
    for (int wd = 16; wd >= 1; wd >>= 1) {
        const bool upper = (lane & wd) != 0;
#pragma unroll
        for (int i = 0; i < wd; ++i) {
            const T send = upper ? v[i] : v[i + wd];
            const T keep = upper ? v[i + wd] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, wd);
        }
    }
    return v[0];
}

// Row pass of kind 2 (w_i = (r_i - c_i . y) / lam~, dots r.w and r.z_old)
// for PL <= 32: a warp takes the rows w, w + kNW, ... of a chunk (at most 32
// when kRowChunk = 32 kNW), holds its slice of y in registers, keeps one
// partial dot per row and reduces all of them at once by a reduce-scatter, so
// no per-row warp reduction sits in a dependency chain (the per-row
// reductions of row_one held this pass to the latency of one shuffle chain
// per row).
template <typename T, typename TC, int PL>
__device__ void row_pass_w(const L2Args<T, TC>& a, int64_t row0, int64_t row1, const T* svec, T* srow,
                           double* rw, double* rzo) {
    static_assert(PL <= 32, "y slice and 32 partial dots in registers");
    static_assert(kRowChunk == 32 * kNW, "a warp's rows of a chunk fit one reduce-scatter");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int W = StoreW<TC>::W;
    T* sr = srow;
    T* sw = srow + kRowChunk;
    T ys[PL];
#pragma unroll
    for (int k = 0; k < PL / W; ++k)
#pragma unroll
        for (int e = 0; e < W; ++e) ys[k * W + e] = svec[k * 32 * W + lane * W + e];
    double d_rw = 0.0, d_rzo = 0.0;
    for (int64_t base = row0; base < row1; base += kRowChunk) {
        const int64_t end = min(row1, base + kRowChunk);
        const int nr = (int)(end - base);
        for (int e = threadIdx.x; e < nr; e += blockDim.x) sr[e] = a.r[base + e];
        __syncthreads();
        const int cnt = nr > w ? (nr - w + kNW - 1) / kNW : 0;   // this warp's rows: w + kNW t, t < cnt
        T part[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) part[t] = T(0);
#pragma unroll
        for (int t = 0; t < 32; t += 2) {
            if (t < cnt) {
                RowSlice<T, PL, TC> c0, c1;
                c0.load(a.C + (base + w + (int64_t)kNW * t) * a.s_pad, lane);
                const bool two = t + 1 < cnt;
                if (two) c1.load(a.C + (base + w + (int64_t)kNW * (t + 1)) * a.s_pad, lane);
                T d0 = T(0), d1 = T(0);
#pragma unroll
                for (int k = 0; k < PL; ++k) d0 += c0.v[k] * ys[k];
                part[t] = d0;
                if (two) {
#pragma unroll
                    for (int k = 0; k < PL; ++k) d1 += c1.v[k] * ys[k];
                    part[t + 1] = d1;
                }
            }
        }
        const T dot = reduce_scatter32<T>(part, lane);
        if (lane < cnt) {
            const int il = w + kNW * lane;
            sw[il] = (sr[il] - dot) / a.lam_t;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nr; e += blockDim.x) {
            const T ri = sr[e], wi = sw[e];
            const T zo = a.z[base + e];
            d_rw += (double)ri * (double)wi;
            d_rzo += (double)ri * (double)zo;
            a.z[base + e] = wi;
        }
        __syncthreads();
    }
    *rw = d_rw;
    *rzo = d_rzo;
}

// part[b][c] = sum over warps of swarp[w][c]
template <typename T, typename TC>
__device__ inline void combine_warps(const L2Args<T, TC>& a, const T* swarp, int b) {
    __syncthreads();
    for (int64_t c = threadIdx.x; c < a.s_pad; c += blockDim.x) {
        T v = T(0);
#pragma unroll
        for (int w = 0; w < kNW; ++w) v += swarp[w * a.s_pad + c];
        a.part[(int64_t)b * a.s_pad + c] = v;
    }
}

// out[c] = M[c,:] . svec for c in [c0, c1) (warp per row)
template <typename T, int PL, typename TS = T>
__device__ inline void rows_dot(const TS* M, int64_t s_pad, int64_t c0, int64_t c1, const T* svec,
                                T* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t c = c0 + w; c < c1; c += kNW) {
        RowSlice<T, PL, TS> m;
        m.load(M + c * s_pad, lane);
        T t = msp::warp_sum(m.dot_smem(svec, lane));
        if (lane == 0) out[c] = t;
    }
}

// out[c] = sum_k part[k][c] (+ add_scale * addend[c]) for c in [c0, c1), k < G.
// Fixed order: thread t sums k = t, t + blockDim, ...; then a warp tree; then
// warps in index order. Returns sum_c out[c] * dvec[c] (dvec in shared memory,
// may be null) and sum_c out[c]^2 through *sq (may be null). Columns are
// processed 8 at a time so all loads of a chunk are in flight together.
// With `pre` (stride pre_stride, G entries), its sum is formed alongside, its
// loads in flight with the first chunk's, in the order of sum_parts (same
// value), into *pre_out for every thread; red2 then holds 9 x 32 doubles.
template <typename T>
__device__ inline void reduce_cols(const T* part, int G, int64_t sp, int64_t c0, int64_t c1,
                                   const T* addend, T add_scale, T* out, const T* dvec,
                                   double* dot_out, double* sq_out, double* red2 /*8*32*/,
                                   const double* pre = nullptr, int pre_stride = 0,
                                   double* pre_out = nullptr) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double dot = 0.0, sq = 0.0;
    bool first = true;
    for (int64_t cb = c0; first || cb < c1; cb += 8) {
        const int nc = (int)max((int64_t)0, min((int64_t)8, c1 - cb));
        const bool with_pre = first && pre != nullptr;
        first = false;
        T v[8];
        double pv = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = T(0);
        for (int k = threadIdx.x; k < G; k += blockDim.x) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < nc) v[c] += __ldcg(&part[(int64_t)k * sp + cb + c]);
            if (with_pre) pv += __ldcg(&pre[(int64_t)k * pre_stride]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = msp::warp_sum(v[c]);
        if (with_pre) pv = msp::warp_sum(pv);
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) red2[c * 32 + w] = (double)v[c];
            if (with_pre) red2[8 * 32 + w] = pv;
        }
        __syncthreads();
        if (with_pre) {
            double t = 0.0;
            for (int k = 0; k < nw; ++k) t += red2[8 * 32 + k];
            *pre_out = t;
        }
        if (threadIdx.x < nc) {
            const int c = threadIdx.x;
            double acc = 0.0;
            for (int k = 0; k < nw; ++k) acc += red2[c * 32 + k];
            T r = (T)acc;
            if (addend) r += add_scale * __ldcg(&addend[cb + c]);
            out[cb + c] = r;
            if (dvec) dot += (double)dvec[cb + c] * (double)r;
            sq += (double)r * (double)r;
        }
    }
    __syncthreads();
    if (dot_out) *dot_out = dot;   // per-thread partials; caller block-sums them
    if (sq_out) *sq_out = sq;
}

template <typename T>
__device__ inline void load_full(const T* g, T* s, int64_t m) {
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) s[c] = __ldcg(&g[c]);
}

template <typename T, typename TC, int PL>
__global__ void __launch_bounds__(kThreads, 1) k_level2(L2Args<T, TC> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t sp = a.s_pad;
    T* sd = reinterpret_cast<T*>(smem_raw);       // d (search direction)
    T* sres = sd + sp;                            // level-2 residual
    T* sy = sres + sp;                            // level-2 iterate
    T* stmp = sy + sp;                            // scratch full vector
    T* swarp = stmp + sp;                         // kNW x sp
    T* srow = swarp + kNW * sp;                   // 2 x kRowChunk (row pass staging)
    __shared__ double red[32];
    __shared__ double red64[64];
    __shared__ double red2[9 * 32];
    __shared__ double s_rw, s_rzo;

    CtlBlock* ctl = a.ctl;
    // the control words in one round trip
    const int c_done = ctl->done, c_err = ctl->error;
    const double alpha = ctl->alpha;
    const double rz_outer = ctl->rz;
    const double tol2 = ctl->tol2;
    if (c_done | c_err) return;
    const int G = gridDim.x, b = blockIdx.x;
    const int64_t row0 = a.n * b / G, row1 = a.n * (b + 1) / G;
    const int64_t c0 = sp * b / G, c1 = sp * (b + 1) / G;
    unsigned int* bw = &ctl->bar_word;
    int* err = &ctl->error;

    // ---- level-1 update and g = C^T r partials
    double rr = 0.0;
    if (a.mode == MODE_ITER && a.qpart) {
        // q_i = sum over the packed A pass's slot partials + lam p_i, fixed
        // summation order. Rounds of four 32-row groups: every thread sums
        // its slot group for the four rows, the loads of all four rows in
        // flight together (eight slots per row at a time), warp g finishes
        // group g (its p_i, r_i, x_i loaded before the slot partials), and
        // warp 0 adds the squares of the new r_i row by row in group order.
        constexpr int kGroups = 4;
        T* sq = swarp;  // kGroups x 8 x 32 scratch (swarp holds 8 s_pad >= 1024 values; free here)
        T* rnew = reinterpret_cast<T*>(red2);   // kGroups x 32 new r_i (red2 is free here)
        const int rl = threadIdx.x & 31, grp = threadIdx.x >> 5;
        for (int64_t base = row0; base < row1; base += 32 * kGroups) {
            const int64_t i_own = base + 32 * grp + rl;      // the row this thread finishes (grp < kGroups)
            const bool own = grp < kGroups && i_own < row1;
            T p_own = T(0), r_own = T(0), x_own = T(0);
            if (own) {
                p_own = a.p[i_own];
                r_own = a.r[i_own];
                x_own = a.x[i_own];
            }
            T v[kGroups];
#pragma unroll
            for (int g = 0; g < kGroups; ++g) v[g] = T(0);
            int sl = grp;
            for (; sl + 7 * kNW < a.q_slots; sl += 8 * kNW) {
                T t8[kGroups][8];
#pragma unroll
                for (int g = 0; g < kGroups; ++g) {
                    const int64_t i = base + 32 * g + rl;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        t8[g][u] = (i < row1) ? __ldcg(&a.qpart[(int64_t)(sl + u * kNW) * a.q_ld + i]) : T(0);
                }
#pragma unroll
                for (int g = 0; g < kGroups; ++g)
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[g] += t8[g][u];
            }
            for (; sl < a.q_slots; sl += kNW) {
#pragma unroll
                for (int g = 0; g < kGroups; ++g) {
                    const int64_t i = base + 32 * g + rl;
                    if (i < row1) v[g] += __ldcg(&a.qpart[(int64_t)sl * a.q_ld + i]);
                }
            }
#pragma unroll
            for (int g = 0; g < kGroups; ++g) sq[(g * kNW + grp) * 32 + rl] = v[g];
            __syncthreads();
            if (grp < kGroups) {
                T ri = T(0);
                if (own) {
                    T qi = T(0);
#pragma unroll
                    for (int g = 0; g < kNW; ++g) qi += sq[(grp * kNW + g) * 32 + rl];
                    qi += a.lam * p_own;
                    ri = r_own;
                    a.x[i_own] = x_own + (T)alpha * p_own;
                    ri -= (T)alpha * qi;
                    a.r[i_own] = ri;
                }
                rnew[grp * 32 + rl] = ri;
            }
            __syncthreads();
            if (grp == 0) {
                for (int g = 0; g < kGroups; ++g) {
                    if (base + 32 * g + rl < row1) {
                        const T ri = rnew[g * 32 + rl];
                        rr += (double)ri * (double)ri;
                    }
                }
            }
            __syncthreads();
        }
        rr = block_sum(rr, red);
        if (threadIdx.x == 0) a.dpart[b * 4 + 0] = rr;
    } else if (a.mode != MODE_APPLY) {
        for (int64_t i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
            T ri = a.r[i];
            if (a.mode == MODE_ITER) {
                a.x[i] += (T)alpha * a.p[i];
                ri -= (T)alpha * a.q[i];
                a.r[i] = ri;
            }
            rr += (double)ri * (double)ri;
        }
        rr = block_sum(rr, red);
        if (threadIdx.x == 0) a.dpart[b * 4 + 0] = rr;
    }
    __syncthreads();
    row_pass<T, TC, PL>(a, 0, row0, row1, nullptr, swarp, srow, nullptr, nullptr);
    combine_warps(a, swarp, b);
    if (!msp::grid_barrier(bw, err)) return;

    // ---- g reduced over this block's columns, with |r|^2 (the convergence
    // test) summed alongside; |g|^2 only where the level-2 iteration's
    // tolerance needs it
    const bool inner = a.max_inner > 0;
    double gg = 0.0;
    reduce_cols<T>(a.part, G, sp, c0, c1, nullptr, T(0), a.gvec, nullptr, nullptr, inner ? &gg : nullptr, red2,
                   a.mode != MODE_APPLY ? a.dpart + 0 : nullptr, 4, &rr);
    if (a.mode != MODE_APPLY) {
        if (!isfinite(rr)) {
            if (b == 0 && threadIdx.x == 0) ctl->error = MSP_ENONFINITE;
            return;
        }
        double t2 = tol2;
        if (a.mode == MODE_INIT) t2 = a.tol_rel2 * rr;
        if (rr <= t2) {
            if (b == 0 && threadIdx.x == 0) {
                ctl->rr = rr;
                if (a.mode == MODE_INIT) { ctl->bb = rr; ctl->tol2 = t2; }
                if (a.mode == MODE_ITER) ctl->iters += 1;
                ctl->done = 1;
            }
            return;
        }
    }
    if (inner) {
        gg = block_sum(gg, red);
        if (threadIdx.x == 0) a.dpart[b * 4 + 1] = gg;
    }
    if (!msp::grid_barrier(bw, err)) return;
    if (inner) gg = sum_parts(a.dpart + 1, 4, G, red);
    load_full(a.gvec, sres, sp);
    for (int64_t c = threadIdx.x; c < sp; c += blockDim.x) sy[c] = T(0);
    __syncthreads();

    // ---- z = M2^{-1} res = B^T (B res)
    auto precond = [&](double* rz_out) -> bool {
        rows_dot<T, PL>(a.B, sp, c0, c1, sres, a.tvec);
        if (!msp::grid_barrier(bw, err)) return false;
        load_full(a.tvec, stmp, sp);
        __syncthreads();
        rows_dot<T, PL>(a.Bt, sp, c0, c1, stmp, a.zvec);
        __syncthreads();
        // z^T res only where the level-2 iteration uses it (rz_out given;
        // the same in every block)
        if (rz_out) {
            double part = 0.0;
            for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x)
                part += (double)sres[c] * (double)a.zvec[c];
            part = block_sum(part, red);
            if (threadIdx.x == 0) a.dpart[b * 4 + 2] = part;
        }
        if (!msp::grid_barrier(bw, err)) return false;
        if (rz_out) *rz_out = sum_parts(a.dpart + 2, 4, G, red);
        return true;
    };

    // direct level 2 (max_inner == 0) has no level-2 iteration: z^T res unused
    double rz_in = 0.0;
    if (!precond(inner ? &rz_in : nullptr)) return;
    // direct level 2: M2 is the level-2 operator itself (Phi = I), so
    // y = M2^{-1} C^T r with no correction steps
    load_full(a.zvec, inner ? sd : sy, sp);
    __syncthreads();
    double rres = gg;
    const double tin2 = a.inner_tol2 * gg;
    int k = 0;
    while (k < a.max_inner && rres > tin2) {
        // P1: partial u = C^T (C d) over this block's rows; wd = W d (columns)
        row_pass<T, TC, PL>(a, 1, row0, row1, sd, swarp, srow, nullptr, nullptr);
        combine_warps(a, swarp, b);
        rows_dot<T, PL, TC>(a.W, sp, c0, c1, sd, a.wdvec);
        if (!msp::grid_barrier(bw, err)) return;
        // P2: u over this block's columns; d.u partial
        double du = 0.0;
        reduce_cols<T>(a.part, G, sp, c0, c1, a.wdvec, a.lam_t, a.uvec, sd, &du, nullptr, red2);
        du = block_sum(du, red);
        if (threadIdx.x == 0) a.dpart[b * 4 + 3] = du;
        if (!msp::grid_barrier(bw, err)) return;
        // P3: step
        du = sum_parts(a.dpart + 3, 4, G, red);
        if (!(du > 0.0)) break;   // breakdown (same decision in every block)
        const T ain = (T)(rz_in / du);
        double loc = 0.0;
        for (int64_t c = threadIdx.x; c < sp; c += blockDim.x) {
            T u = __ldcg(&a.uvec[c]);
            sy[c] += ain * sd[c];
            T rv = sres[c] - ain * u;
            sres[c] = rv;
            loc += (double)rv * (double)rv;
        }
        rres = block_sum(loc, red);
        ++k;
        if (rres <= tin2) break;
        double rz_new = 0.0;
        if (!precond(&rz_new)) return;
        const T beta = (T)(rz_new / rz_in);
        rz_in = rz_new;
        for (int64_t c = threadIdx.x; c < sp; c += blockDim.x) sd[c] = __ldcg(&a.zvec[c]) + beta * sd[c];
        __syncthreads();
    }

    // ---- w = (r - C y) / lam~ into z; dots for the level-1 beta
    __syncthreads();
    double rw = 0.0, rzo = 0.0;
    if constexpr (PL <= 32 && (sizeof(T) == 4 || PL <= 16)) row_pass_w<T, TC, PL>(a, row0, row1, sy, srow, &rw, &rzo);
    else row_pass<T, TC, PL>(a, 2, row0, row1, sy, swarp, srow, &rw, &rzo);
    block_sum2(rw, rzo, red64);
    if (threadIdx.x == 0) {
        a.dpart[b * 4 + 0] = rw;
        a.dpart[b * 4 + 1] = rzo;
    }
    if (a.mode == MODE_APPLY) {
        if (b == 0 && threadIdx.x == 0) atomicAdd(&ctl->inner_iters, k);
        return;
    }
    if (!msp::grid_barrier(bw, err)) return;
    // this thread's first row of z and p, in flight with the dot partials
    const int64_t i_first = row0 + threadIdx.x;
    T z_first = T(0), p_first = T(0);
    if (i_first < row1) {
        z_first = a.z[i_first];
        p_first = a.p[i_first];
    }
    sum_parts2(a.dpart + 0, 4, G, red64, rw, rzo);
    T beta = T(0);
    if (a.mode == MODE_ITER) beta = (T)((rw - rzo) / rz_outer);
    for (int64_t i = i_first; i < row1; i += blockDim.x) {
        const T zi = (i == i_first) ? z_first : a.z[i];
        const T pi = (i == i_first) ? p_first : a.p[i];
        a.p[i] = zi + beta * (a.mode == MODE_ITER ? pi : T(0));
    }
    if (b == 0 && threadIdx.x == 0) {
        ctl->rz = rw;
        ctl->beta = (double)beta;
        ctl->rr = rr;
        ctl->inner_iters += k;
        if (a.mode == MODE_ITER) ctl->iters += 1;
        if (a.mode == MODE_INIT) { ctl->bb = rr; ctl->tol2 = a.tol_rel2 * rr; }
        if (!(rw > 0.0) && isfinite(rw)) ctl->error = MSP_ENOTPD;
        if (!isfinite(rw)) ctl->error = MSP_ENONFINITE;
    }
    (void)s_rw;
    (void)s_rzo;
}

template <typename T, typename TC, int PL>
msp_status launch_level2_pl(msp_ctx* ctx, L2Args<T, TC>& a, int G) {
    auto kern = k_level2<T, TC, PL>;
    size_t smem = ((size_t)(4 + kNW) * a.s_pad + 2 * kRowChunk) * sizeof(T);
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    // co-residency is required by the grid barrier: never exceed what fits
    int per_sm = 0;
    MSP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1)
        return msp_set_error(ctx, MSP_EINVAL, "level-2 kernel does not fit on an SM");
    G = std::min(G, per_sm * ctx->num_sms);
    void* args[] = {&a};
    ++ctx->launches;
    MSP_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(kThreads), args,
                                                  smem, ctx->stream));
    return MSP_OK;
}

template <typename T, typename TC>
msp_status launch_level2(msp_ctx* ctx, L2Args<T, TC>& a, int G) {
    // one instantiation per padded sketch size (multiples of 128 up to 1024,
    // then 1536 and 2048)
    switch (a.s_pad) {
        case 128: return launch_level2_pl<T, TC, 4>(ctx, a, G);
        case 256: return launch_level2_pl<T, TC, 8>(ctx, a, G);
        case 384: return launch_level2_pl<T, TC, 12>(ctx, a, G);
        case 512: return launch_level2_pl<T, TC, 16>(ctx, a, G);
        case 640: return launch_level2_pl<T, TC, 20>(ctx, a, G);
        case 768: return launch_level2_pl<T, TC, 24>(ctx, a, G);
        case 896: return launch_level2_pl<T, TC, 28>(ctx, a, G);
        case 1024: return launch_level2_pl<T, TC, 32>(ctx, a, G);
        case 1536:
            if constexpr (sizeof(T) == 4) return launch_level2_pl<T, TC, 48>(ctx, a, G);
            break;
        case 2048:
            if constexpr (sizeof(T) == 4) return launch_level2_pl<T, TC, 64>(ctx, a, G);
            break;
        default: break;
    }
    return msp_set_error(ctx, MSP_EINVAL, "level-2: unsupported padded sketch size %lld",
                         (long long)a.s_pad);
}

struct Workspace {
    void* part;
    void* vecs;
    double* dpart;
    void* level1;   // x r q p z (n_pad each)
    double* gpart;  // A-pass partials
    float* qpart;   // packed A pass: nt x n_pad slot partials (or null)
    int64_t n_pad;
};

template <typename T>
msp_status get_workspace(msp_ctx* ctx, int64_t n, int64_t sp, int G, int Gg, bool packed,
                         Workspace* ws) {
    size_t ts = sizeof(T);
    const int64_t n_pad = round_up(n, 128);
    const int64_t nt = n_pad / 128;
    size_t b_part = round_up((int64_t)G * sp * ts, 256);
    size_t b_vecs = round_up(5 * sp * ts, 256);
    size_t b_dpart = round_up((int64_t)G * 4 * 8, 256);
    size_t b_l1 = round_up(5 * n_pad * ts, 256);
    size_t b_gp = round_up((int64_t)Gg * 8, 256);
    size_t b_qp = packed ? round_up(nt * n_pad * 4, 256) : 0;
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, b_part + b_vecs + b_dpart + b_l1 + b_gp + b_qp, &scr));
    char* c = (char*)scr;
    ws->part = c; c += b_part;
    ws->vecs = c; c += b_vecs;
    ws->dpart = (double*)c; c += b_dpart;
    ws->level1 = c; c += b_l1;
    ws->gpart = (double*)c; c += b_gp;
    ws->qpart = packed ? (float*)c : nullptr;
    ws->n_pad = n_pad;
    return MSP_OK;
}

template <typename T, typename TC>
void fill_l2(L2Args<T, TC>& a, const msp_factor_s* f, int64_t n, const Workspace& ws, CtlBlock* ctl) {
    const int64_t sp = f->s_pad;
    a.n = n;
    a.s_pad = sp;
    // BF16 preconditioner data: the factor's rounded copies of C and W
    a.C = (const TC*)(f->data == MSP_BF16 ? f->Cb : f->sk->C);
    a.W = (const TC*)(f->data == MSP_BF16 ? f->Wb : f->W);
    a.B = (const T*)f->B;
    a.Bt = (const T*)f->Bt;
    a.lam_t = (T)f->lam_tilde;
    a.ctl = ctl;
    a.part = (T*)ws.part;
    T* v = (T*)ws.vecs;
    a.gvec = v;
    a.uvec = v + sp;
    a.tvec = v + 2 * sp;
    a.zvec = v + 3 * sp;
    a.wdvec = v + 4 * sp;
    a.dpart = ws.dpart;
}

// Upper bound on the level-2 grid (2 blocks per SM); launch_level2_pl lowers
// it to what the occupancy calculator guarantees co-resident. The workspace is
// sized for the upper bound.
int level2_grid(msp_ctx* ctx) { return 2 * ctx->num_sms; }
int gemv_grid(msp_ctx* ctx) { return ctx->num_sms * 8; }

// ------------------------------------------------ level-1 graph replay
//
// One level-1 iteration is two launches whose arguments do not change from
// one iteration to the next (the A pass and the cooperative level-2 kernel;
// the scalars travel through the control block). It is captured once into a
// CUDA graph and replayed, which removes the per-launch host work and most
// of the gap between the two kernels. The executable is cached in the
// context under a key of everything the launches were built from (argument
// structs, buffers, grid sizes); any change rebuilds it.

constexpr int kL1Timed = 2;     // event-record nodes of a timed iteration graph

// Captures iter(true) (launches on ctx->stream, redirected to the capture
// stream) as the context's level-1 graph for `key`. With `timed`, iter puts
// an event-record node before the A pass and one between the A pass and the
// level-2 kernel (ctx->events[0..1]), found again here by their events so
// that each replay can point them at fresh events. Leaves ctx->l1_exec null
// where capture is not possible; the caller then launches on the stream.
template <typename F>
msp_status ensure_l1_graph(msp_ctx* ctx, const void* key, size_t klen, bool timed, F&& iter) {
    if (ctx->l1_exec && ctx->l1_key_len == klen && std::memcmp(ctx->l1_key, key, klen) == 0)
        return MSP_OK;
    msp_l1_graph_release(ctx);
    if (klen > sizeof(ctx->l1_key)) return MSP_OK;
    if (!ctx->cap_stream &&
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->cap_stream = nullptr;
        return MSP_OK;
    }
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return MSP_OK;
    }
    const cudaStream_t saved = ctx->stream;
    const int64_t l0 = ctx->launches;
    ctx->stream = ctx->cap_stream;
    const msp_status st = iter(true);
    ctx->stream = saved;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    const int kernels = (int)(ctx->launches - l0);
    ctx->launches = l0;
    bool ok = st == MSP_OK && ce == cudaSuccess && graph != nullptr;
    cudaGraphNode_t evn[kL1Timed] = {};
    if (ok && timed) {
        size_t nn = 0;
        ok = cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0 && nn <= 64;
        cudaGraphNode_t nodes[64];
        if (ok) ok = cudaGraphGetNodes(graph, nodes, &nn) == cudaSuccess;
        for (size_t i = 0; ok && i < nn; ++i) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess) { ok = false; break; }
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) { ok = false; break; }
            for (int k = 0; k < kL1Timed; ++k)
                if (ev == ctx->events[k]) evn[k] = nodes[i];
        }
        for (int k = 0; ok && k < kL1Timed; ++k) ok = evn[k] != nullptr;
    }
    if (ok && cudaGraphInstantiate(&ctx->l1_exec, graph, 0) != cudaSuccess) {
        ctx->l1_exec = nullptr;
        ok = false;
    }
    if (!ok) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return MSP_OK;
    }
    ctx->l1_graph = graph;
    std::memcpy(ctx->l1_key, key, klen);
    ctx->l1_key_len = klen;
    for (int k = 0; k < kL1Timed; ++k) ctx->l1_ev_nodes[k] = evn[k];
    ctx->l1_kernels = kernels;
    return MSP_OK;
}

// Replays one level-1 iteration. Timed: the graph's two event-record nodes
// get fresh events b (before the A pass) and e (after it); the A pass is
// the entry (b, e), and the level-2 kernel of the iteration before, whose
// end the new b marks, the entry (e_prev, b): two events per iteration.
// *l2_open holds e of the last replay until then (-1: none); the spare
// events past the pool stand in once it is used up. Already queued replays
// keep their events.
msp_status replay_l1(msp_ctx* ctx, Profiler& pr, int* l2_open) {
    if (pr.on) {
        cudaEvent_t eb = ctx->events[ctx->n_events - 2], ee = ctx->events[ctx->n_events - 1];
        int ib = -1, ie = -1;
        const bool fresh = pr.take(&eb, &ib) && pr.take(&ee, &ie);
        if (!fresh) {
            eb = ctx->events[ctx->n_events - 2];
            ee = ctx->events[ctx->n_events - 1];
        }
        MSP_CUDA_TRY(ctx, cudaGraphExecEventRecordNodeSetEvent(ctx->l1_exec, ctx->l1_ev_nodes[0], eb));
        MSP_CUDA_TRY(ctx, cudaGraphExecEventRecordNodeSetEvent(ctx->l1_exec, ctx->l1_ev_nodes[1], ee));
        if (fresh) {
            if (*l2_open >= 0) pr.add(1, *l2_open, ib);
            pr.add(0, ib, ie);
        }
        *l2_open = fresh ? ie : -1;
    }
    MSP_CUDA_TRY(ctx, cudaGraphLaunch(ctx->l1_exec, ctx->stream));
    ctx->launches += ctx->l1_kernels;
    ++ctx->l1_graph_iters;
    return MSP_OK;
}

// Ends the timing chain after the last replay of a check interval: an event
// on the stream closes the open level-2 entry.
msp_status close_l1_chain(msp_ctx* ctx, Profiler& pr, int* l2_open) {
    if (!pr.on || *l2_open < 0) return MSP_OK;
    cudaEvent_t ev;
    int idx;
    if (pr.take(&ev, &idx)) {
        MSP_CUDA_TRY(ctx, cudaEventRecord(ev, ctx->stream));
        pr.add(1, *l2_open, idx);
    }
    *l2_open = -1;
    return MSP_OK;
}

template <typename T, typename TC = T>
msp_status krylov_solve_t(msp_ctx* ctx, const msp_factor_s* f, const void* A, msp_dtype dt,
                          int64_t n, int64_t lda, double lambda, const T* rhs, T* sol,
                          double tol_rel, int max_outer, const msp_opts* o, int* iters,
                          int* inner_iters, ProfSlot* prof, const float* packed) {
    const int G = level2_grid(ctx), Gg = gemv_grid(ctx);
    const bool use_packed = (packed != nullptr) && (sizeof(T) == 4);
    Profiler pr;
    pr.ctx = ctx;
    pr.on = (prof != nullptr) && o->profile;
    if (pr.on) MSP_TRY(msp_profiler_reserve(ctx, 4096));
    Workspace ws;
    MSP_TRY(get_workspace<T>(ctx, n, f->s_pad, G, Gg, use_packed, &ws));
    const int64_t np = ws.n_pad;
    T* x = (T*)ws.level1;
    T* r = x + np;
    T* q = r + np;
    T* p = q + np;
    T* z = p + np;
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(ctl, 0, sizeof(CtlBlock), ctx->stream));
    // all five level-1 vectors, pads included (p must be zero past n)
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, 5 * np * sizeof(T), ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(r, rhs, n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));

    // zeroed bytes (padding included): the struct is part of the graph key
    L2Args<T, TC> a;
    std::memset(&a, 0, sizeof a);
    fill_l2(a, f, n, ws, ctl);
    a.tol_rel2 = tol_rel * tol_rel;
    a.inner_tol2 = o->inner_tol * o->inner_tol;
    a.max_inner = o->max_inner;
    a.x = x; a.r = r; a.q = q; a.p = p; a.z = z;
    a.qpart = use_packed ? ws.qpart : nullptr;
    a.q_slots = (int)(np / 128);
    a.q_ld = np;
    a.lam = (T)lambda;
    a.mode = MODE_INIT;
    MSP_TRY(launch_level2(ctx, a, G));
    a.mode = MODE_ITER;

    const bool vec = (lda % (16 / dtype_size(dt)) == 0) &&
                     ((uintptr_t)A % 16 == 0) && (n % (16 / dtype_size(dt)) == 0);
    // one level-1 iteration: the A pass q = (A + lam I) p, then the level-2
    // kernel (the step, SolveM1, the new direction); `cap`: inside a graph
    // capture, where event-record nodes take the profiler's place
    auto mark = [&](bool cap, int k) -> msp_status {
        if (!pr.on) return MSP_OK;
        if (cap) {
            // event-record nodes before the A pass and between the launches
            if (k < kL1Timed)
                MSP_CUDA_TRY(ctx, cudaEventRecordWithFlags(ctx->events[k], ctx->stream, cudaEventRecordExternal));
            return MSP_OK;
        }
        return (k & 1) ? pr.end() : pr.begin(k >> 1);
    };
    auto iteration = [&](bool cap) -> msp_status {
        MSP_TRY(mark(cap, 0));
        if (use_packed) {
            MSP_TRY(msp_symv_packed(ctx, packed, n, (float)lambda, (const float*)p, ws.qpart,
                                    ws.gpart, ctx->num_sms));
        } else {
            if (dt == MSP_F32) {
                if (vec) k_gemv<float, T, true><<<Gg, 256, 0, ctx->stream>>>((const float*)A, lda, n, lambda, p, q, ws.gpart, ctl);
                else k_gemv<float, T, false><<<Gg, 256, 0, ctx->stream>>>((const float*)A, lda, n, lambda, p, q, ws.gpart, ctl);
            } else {
                if (vec) k_gemv<double, T, true><<<Gg, 256, 0, ctx->stream>>>((const double*)A, lda, n, lambda, p, q, ws.gpart, ctl);
                else k_gemv<double, T, false><<<Gg, 256, 0, ctx->stream>>>((const double*)A, lda, n, lambda, p, q, ws.gpart, ctl);
            }
            MSP_CHECK_LAUNCH(ctx);
        }
        MSP_TRY(mark(cap, 1));
        MSP_TRY(mark(cap, 2));
        MSP_TRY(launch_level2(ctx, a, G));
        MSP_TRY(mark(cap, 3));
        return MSP_OK;
    };
    bool graphed = false;
    if (ctx->l1_graphs) {
        struct Key {
            int tag, dt, use_packed, vec, G, Gg, timed, pad;
            const void* A;
            int64_t lda;
            const float* packed;
            double lambda;
            const void* qpart;
            const void* gpart;
            L2Args<T, TC> a;
        } key;
        static_assert(sizeof(Key) <= sizeof(ctx->l1_key), "level-1 graph key too large");
        std::memset(&key, 0, sizeof key);
        key.tag = (int)(10 * sizeof(T) + sizeof(TC));
        key.dt = (int)dt;
        key.use_packed = use_packed;
        key.vec = vec;
        key.G = G;
        key.Gg = Gg;
        key.timed = pr.on;
        key.A = A;
        key.lda = lda;
        key.packed = packed;
        key.lambda = lambda;
        key.qpart = ws.qpart;
        key.gpart = ws.gpart;
        std::memcpy(&key.a, &a, sizeof a);
        MSP_TRY(ensure_l1_graph(ctx, &key, sizeof key, pr.on, iteration));
        graphed = ctx->l1_exec != nullptr;
    }
    int* hf = (int*)ctx->host_flags;
    const int check = std::max(1, o->check_every);
    // profiler entries of iterations known to have run to completion with
    // work (every iteration before a check that found no flag): read while
    // the next interval runs, not after it
    int settled = 0, l2_open = -1;
    for (int it = 0; it < max_outer;) {
        const int nrun = std::min(check, max_outer - it);
        for (int i = 0; i < nrun; ++i) {
            if (graphed) MSP_TRY(replay_l1(ctx, pr, &l2_open));
            else MSP_TRY(iteration(false));
        }
        if (graphed) MSP_TRY(close_l1_chain(ctx, pr, &l2_open));
        it += nrun;
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hf, &ctl->done, 5 * sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        MSP_TRY(pr.harvest(prof, 2, settled));
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        if (hf[0] || hf[1]) break;
        settled = pr.used;
    }
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hf, &ctl->done, 5 * sizeof(int), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(sol, x, n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    // the iterations that did work: ctl->iters counts them, and every launch
    // queued after the flag returned at once
    if (pr.on) MSP_TRY(pr.finish(prof, 2, 2 * hf[2]));
    // hf: done, error, iters, inner_iters, pad
    if (iters) *iters = hf[2];
    if (inner_iters) *inner_iters = hf[3];
    if (hf[1]) {
        const int e = hf[1];
        return msp_set_error(ctx, (msp_status)e, "level-1 iteration stopped with device status %d%s",
                             e, e == MSP_ETIMEOUT ? " (grid barrier timed out)" : "");
    }
    if (!hf[0]) return msp_set_error(ctx, MSP_ENOCONV, "no convergence in %d level-1 iterations",
                                     hf[2]);
    return MSP_OK;
}

}  // namespace

void msp_l1_graph_release(msp_ctx* ctx) {
    if (ctx->l1_exec) cudaGraphExecDestroy(ctx->l1_exec);
    if (ctx->l1_graph) cudaGraphDestroy(ctx->l1_graph);
    ctx->l1_exec = nullptr;
    ctx->l1_graph = nullptr;
    ctx->l1_key_len = 0;
    for (cudaGraphNode_t& nd : ctx->l1_ev_nodes) nd = nullptr;
    ctx->l1_kernels = 0;
}

extern "C" msp_status msp_set_level1_graphs(msp_ctx* ctx, int on) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    ctx->l1_graphs = on != 0;
    if (!ctx->l1_graphs) msp_l1_graph_release(ctx);
    return MSP_OK;
}

// The grid-barrier limit of this unit's kernels (the level-1 and level-2
// iterations) on the current device; 0 restores the default.
msp_status msp_grid_wait_limit_krylov(msp_ctx* ctx, unsigned long long ns) {
    const unsigned long long v = ns ? ns : msp::kWaitLimitNs;
    MSP_CUDA_TRY(ctx, cudaMemcpyToSymbol(msp::g_grid_wait_limit_ns, &v, sizeof v));
    return MSP_OK;
}

msp_status msp_krylov_solve(msp_ctx* ctx, const msp_factor_s* f, const void* A, msp_dtype dt,
                            int64_t n, int64_t lda, double lambda, const void* rhs, void* sol,
                            double tol_rel, int max_outer, const msp_opts* o, int* iters,
                            int* inner_iters, ProfSlot* prof, const float* packed) {
    if (f->dtype == MSP_F32 && f->data == MSP_BF16)
        return krylov_solve_t<float, __nv_bfloat16>(ctx, f, A, dt, n, lda, lambda, (const float*)rhs, (float*)sol,
                                                    tol_rel, max_outer, o, iters, inner_iters, prof, packed);
    if (f->dtype == MSP_F32)
        return krylov_solve_t<float>(ctx, f, A, dt, n, lda, lambda, (const float*)rhs, (float*)sol,
                                     tol_rel, max_outer, o, iters, inner_iters, prof, packed);
    return krylov_solve_t<double>(ctx, f, A, dt, n, lda, lambda, (const double*)rhs, (double*)sol,
                                  tol_rel, max_outer, o, iters, inner_iters, prof, nullptr);
}

// ---------------------------------------------------------------- profiler

// `pairs` event pairs plus four spare events at the end (the sinks of a
// timed level-1 graph once the pairs are used up)
msp_status msp_profiler_reserve(msp_ctx* ctx, int pairs) {
    const int want = 2 * pairs + 4;
    if (ctx->n_events >= want) return MSP_OK;
    for (int i = 0; i < ctx->n_events; ++i) cudaEventDestroy(ctx->events[i]);
    delete[] ctx->events;
    ctx->events = new cudaEvent_t[want];
    ctx->n_events = 0;
    for (int i = 0; i < want; ++i) {
        MSP_CUDA_TRY(ctx, cudaEventCreate(&ctx->events[i]));
        ctx->n_events = i + 1;
    }
    return MSP_OK;
}

msp_status Profiler::begin(int slot) {
    open = false;
    if (!on || used >= 4096 || next_ev + 2 > ctx->n_events - 4) return MSP_OK;
    slot_of[used] = slot;
    ev_b[used] = next_ev++;
    open = true;
    MSP_CUDA_TRY(ctx, cudaEventRecord(ctx->events[ev_b[used]], ctx->stream));
    return MSP_OK;
}

msp_status Profiler::end() {
    // closes the entry of the last begin() that went through
    if (!open) return MSP_OK;
    open = false;
    ev_e[used] = next_ev++;
    MSP_CUDA_TRY(ctx, cudaEventRecord(ctx->events[ev_e[used]], ctx->stream));
    ++used;
    return MSP_OK;
}

bool Profiler::take(cudaEvent_t* ev, int* idx) {
    if (!on || next_ev + 1 > ctx->n_events - 4) return false;
    *idx = next_ev++;
    *ev = ctx->events[*idx];
    return true;
}

void Profiler::add(int slot, int b, int e) {
    if (!on || used >= 4096) return;
    slot_of[used] = slot;
    ev_b[used] = b;
    ev_e[used] = e;
    ++used;
}

msp_status Profiler::harvest(ProfSlot* slots, int nslots, int upto) {
    if (!on) return MSP_OK;
    for (int i = harvested; i < upto && i < used; ++i) {
        float ms = 0.f;
        MSP_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->events[ev_b[i]], ctx->events[ev_e[i]]));
        if (slot_of[i] < nslots) {
            slots[slot_of[i]].ms += ms;
            slots[slot_of[i]].launches += 1;
        }
        harvested = i + 1;
    }
    return MSP_OK;
}

msp_status Profiler::finish(ProfSlot* slots, int nslots, int keep) {
    if (!on) return MSP_OK;
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    MSP_TRY(harvest(slots, nslots, (keep >= 0 && keep < used) ? keep : used));
    used = 0;
    harvested = 0;
    next_ev = 0;
    return MSP_OK;
}

msp_status msp_solve_m1_impl(msp_ctx* ctx, const msp_factor_s* f, const void* r, void* w,
                             const msp_opts* o, int* inner_iters) {
    const int64_t n = f->sk->n;
    const int G = level2_grid(ctx), Gg = gemv_grid(ctx);
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(ctl, 0, sizeof(CtlBlock), ctx->stream));
    int* hf = (int*)ctx->host_flags;
    if (f->dtype == MSP_F32 && f->data == MSP_BF16) {
        Workspace ws;
        MSP_TRY(get_workspace<float>(ctx, n, f->s_pad, G, Gg, false, &ws));
        L2Args<float, __nv_bfloat16> a{};
        fill_l2(a, f, n, ws, ctl);
        a.inner_tol2 = o->inner_tol * o->inner_tol;
        a.max_inner = o->max_inner;
        a.r = (float*)r;
        a.z = (float*)w;
        a.mode = MODE_APPLY;
        MSP_TRY(launch_level2(ctx, a, G));
    } else if (f->dtype == MSP_F32) {
        Workspace ws;
        MSP_TRY(get_workspace<float>(ctx, n, f->s_pad, G, Gg, false, &ws));
        L2Args<float> a{};
        fill_l2(a, f, n, ws, ctl);
        a.inner_tol2 = o->inner_tol * o->inner_tol;
        a.max_inner = o->max_inner;
        a.r = (float*)r;
        a.z = (float*)w;
        a.mode = MODE_APPLY;
        MSP_TRY(launch_level2(ctx, a, G));
    } else {
        Workspace ws;
        MSP_TRY(get_workspace<double>(ctx, n, f->s_pad, G, Gg, false, &ws));
        L2Args<double> a{};
        fill_l2(a, f, n, ws, ctl);
        a.inner_tol2 = o->inner_tol * o->inner_tol;
        a.max_inner = o->max_inner;
        a.r = (double*)r;
        a.z = (double*)w;
        a.mode = MODE_APPLY;
        MSP_TRY(launch_level2(ctx, a, G));
    }
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hf, &ctl->done, 5 * sizeof(int), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (inner_iters) *inner_iters = hf[3];
    if (hf[1]) return msp_set_error(ctx, (msp_status)hf[1], "SolveM1: device status %d", hf[1]);
    return MSP_OK;
}

namespace {

// Error-free transformations (Knuth's TwoSum; the FMA form of Dekker's
// TwoProduct): a + b = s + e and a b = p + e exactly in FP64.
__device__ inline void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ inline void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = fma(a, b, -p);
}
// (hi, lo) += (p, q), a double-double sum (hi, lo) renormalised
__device__ inline void dd_add(double& hi, double& lo, double p, double q) {
    double s, e;
    two_sum(hi, p, s, e);
    e += lo + q;
    hi = s + e;
    lo = e - (hi - s);
}

// x = xh + xl with xh = fl32(x), xl = fl32(x - xh) (x - xh exact in FP64):
// |x - xh - xl| <= 2^-48 |x|.
__global__ void k_split_x(const double* __restrict__ x, int64_t n, float* __restrict__ xh, float* __restrict__ xl) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[j];
        const float h = (float)v;
        xh[j] = h;
        xl[j] = (float)(v - (double)h);
    }
}

// (hi, lo) += p + t (|t| small): TwoSum (Knuth) of hi and p, the error, lo
// and t added, then renormalised by Fast2Sum (Dekker) so that |lo| stays
// within half an ulp of hi; each call adds at most about 2^-47 |hi| of error.
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float p, float t) {
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    e = __fadd_rn(e, __fadd_rn(lo, t));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// out = b - (A + lam I) x for an FP32 A in float-float arithmetic on the FP32
// pipe (the FP64 pipe of this part, two FMAs per clock per SM, held the FP64
// version to a third of the HBM rate). Per element: a xh exactly as p + e
// (TwoProd by FMA), a xl + e rounded (at most about 2^-47 |a x|), both added
// to a per-lane float-float pair (ff_acc). Four pairs per lane (one per
// float4 component), n / 128 elements each; the pairs are added in FP64 in a
// fixed order. Error at most about (n / 128 + 2) 2^-47 sum_j |a_ij x_j|
// (2^-40 at n = 16384), with the split of x: far below the backward errors
// the refinement resolves (1e-10 ~ 2^-33). |out|^2 into *norm2 as k_matvec64.
// Requires lda, n multiples of 4 and 16-byte aligned A.
__global__ void __launch_bounds__(256, 2) k_matvec64_ff(const float* __restrict__ A, int64_t lda, int64_t n,
                                                    double lam, const float* __restrict__ xh,
                                                    const float* __restrict__ xl, const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ out,
                                                    double* __restrict__ part, unsigned int* counter,
                                                    double* norm2) {
    __shared__ double red[32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double nn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const float* row = A + i * lda;
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        int64_t j = (int64_t)lane * 4;
        for (; j + 128 < n; j += 256) {
            const float4 a0 = __ldcs(reinterpret_cast<const float4*>(row + j));
            const float4 a1 = __ldcs(reinterpret_cast<const float4*>(row + j + 128));
            const float4 h0 = __ldg(reinterpret_cast<const float4*>(xh + j));
            const float4 h1 = __ldg(reinterpret_cast<const float4*>(xh + j + 128));
            const float4 l0 = __ldg(reinterpret_cast<const float4*>(xl + j));
            const float4 l1 = __ldg(reinterpret_cast<const float4*>(xl + j + 128));
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
            const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float p = __fmul_rn(av[k], hv[k]);
                const float e = __fmaf_rn(av[k], hv[k], -p);
                ff_acc(hi[k & 3], lo[k & 3], p, __fmaf_rn(av[k], lv[k], e));
            }
        }
        for (; j < n; j += 128) {
            const float4 a0 = __ldcs(reinterpret_cast<const float4*>(row + j));
            const float4 h0 = __ldg(reinterpret_cast<const float4*>(xh + j));
            const float4 l0 = __ldg(reinterpret_cast<const float4*>(xl + j));
            const float av[4] = {a0.x, a0.y, a0.z, a0.w};
            const float hv[4] = {h0.x, h0.y, h0.z, h0.w};
            const float lv[4] = {l0.x, l0.y, l0.z, l0.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float p = __fmul_rn(av[k], hv[k]);
                const float e = __fmaf_rn(av[k], hv[k], -p);
                ff_acc(hi[k], lo[k], p, __fmaf_rn(av[k], lv[k], e));
            }
        }
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += (double)hi[k] + (double)lo[k];
        acc = msp::warp_sum(acc);
        if (lane == 0) {
            double v = acc + lam * x[i];
            if (b) v = b[i] - v;
            out[i] = v;
            nn += v * v;
        }
    }
    double tot = block_sum(nn, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double all = sum_parts(part, 1, gridDim.x, red);
    if (threadIdx.x == 0) {
        *counter = 0;
        if (norm2) *norm2 = all;
    }
}

// out = b - (A + lam I) x with double-double accumulation: every product
// and sum error-free transformed, rounded to FP64 once per row. Its error is
// a few u |r_i| + u^2 sum_j |A_ij x_j| instead of u sum_j |A_ij x_j|, so the
// residual of an ill-conditioned system stays resolved below the FP64
// accumulation floor. |out|^2 into *norm2 as k_matvec64.
template <typename TA>
__global__ void __launch_bounds__(256) k_matvec64_dd(const TA* __restrict__ A, int64_t lda, int64_t n, double lam,
                                                    const double* __restrict__ x, const double* __restrict__ b,
                                                    double* __restrict__ out, double* __restrict__ part,
                                                    unsigned int* counter, double* norm2) {
    __shared__ double red[32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double nn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const TA* row = A + i * lda;
        double hi = 0.0, lo = 0.0;
        for (int64_t j = lane; j < n; j += 32) {
            double p, e;
            two_prod(wide64(__ldcs(&row[j])), x[j], p, e);
            dd_add(hi, lo, p, e);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ph = __shfl_xor_sync(0xffffffffu, hi, o);
            const double pl = __shfl_xor_sync(0xffffffffu, lo, o);
            dd_add(hi, lo, ph, pl);
        }
        if (lane == 0) {
            double p, e;
            two_prod(lam, x[i], p, e);
            dd_add(hi, lo, p, e);
            double v = hi + lo;
            if (b) {
                double rh = b[i], rl = 0.0;
                dd_add(rh, rl, -hi, -lo);
                v = rh + rl;
            }
            out[i] = v;
            nn += v * v;
        }
    }
    double tot = block_sum(nn, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double all = sum_parts(part, 1, gridDim.x, red);
    if (threadIdx.x == 0) {
        *counter = 0;
        if (norm2) *norm2 = all;
    }
}

}  // namespace

msp_status msp_matvec64(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda,
                        double lambda, const double* x, const double* b, double* out,
                        double* norm2_out_dev, bool compensated) {
    const int Gg = gemv_grid(ctx);
    void* scr = nullptr;
    const size_t b_part = round_up((int64_t)Gg * 8, 256), b_x = round_up(n * 4, 256);
    MSP_TRY(msp_scratch(ctx, b_part + 2 * b_x + 256, &scr));
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    if (dt == MSP_BF16) {
        // BF16 A (the matvec of a BF16-stored matrix, e.g. to measure its
        // rounding against an FP32 or FP64 copy)
        if (compensated)
            k_matvec64_dd<__nv_bfloat16><<<Gg, 256, 0, ctx->stream>>>((const __nv_bfloat16*)A, lda, n, lambda, x, b,
                                                                      out, (double*)scr, &ctl->last_block_counter,
                                                                      norm2_out_dev);
        else
            k_matvec64<__nv_bfloat16, false><<<Gg, 256, 0, ctx->stream>>>((const __nv_bfloat16*)A, lda, n, lambda, x,
                                                                          b, out, (double*)scr,
                                                                          &ctl->last_block_counter, norm2_out_dev);
        MSP_CHECK_LAUNCH(ctx);
        return MSP_OK;
    }
    if (compensated) {
        if (dt == MSP_F32)
            k_matvec64_dd<float><<<Gg, 256, 0, ctx->stream>>>((const float*)A, lda, n, lambda, x, b, out,
                                                              (double*)scr, &ctl->last_block_counter,
                                                              norm2_out_dev);
        else
            k_matvec64_dd<double><<<Gg, 256, 0, ctx->stream>>>((const double*)A, lda, n, lambda, x, b, out,
                                                               (double*)scr, &ctl->last_block_counter,
                                                               norm2_out_dev);
        MSP_CHECK_LAUNCH(ctx);
        return MSP_OK;
    }
    const bool vec = (dt == MSP_F32) && (lda % 4 == 0) && (n % 4 == 0) &&
                     ((uintptr_t)A % 16 == 0) && ((uintptr_t)x % 16 == 0);
    if (dt == MSP_F32) {
        if (vec) {
            float* xh = (float*)((char*)scr + b_part);
            float* xl = (float*)((char*)scr + b_part + b_x);
            k_split_x<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms), 256, 0, ctx->stream>>>(
                x, n, xh, xl);
            MSP_CHECK_LAUNCH(ctx);
            k_matvec64_ff<<<Gg, 256, 0, ctx->stream>>>((const float*)A, lda, n, lambda, xh, xl, x, b, out,
                                                       (double*)scr, &ctl->last_block_counter, norm2_out_dev);
        } else
            k_matvec64<float, false><<<Gg, 256, 0, ctx->stream>>>((const float*)A, lda, n, lambda, x, b,
                                                                  out, (double*)scr,
                                                                  &ctl->last_block_counter, norm2_out_dev);
    } else {
        k_matvec64<double, false><<<Gg, 256, 0, ctx->stream>>>((const double*)A, lda, n, lambda, x, b,
                                                               out, (double*)scr,
                                                               &ctl->last_block_counter, norm2_out_dev);
    }
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}
// ------------------------------------------------------------ vector ops

namespace {

// |v|^2 of an FP64 vector, one block, fixed order.
__global__ void k_norm2(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i] * v[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double scale,
                      double* __restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * y[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = scale * acc;
}

// dst = (T)(src / sqrt(*nrm2)) (0 if the norm is 0)
template <typename T>
__global__ void k_scale_cast(const double* __restrict__ src, const double* __restrict__ nrm2,
                             int64_t n, T* __restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
    dst[i] = (T)(src[i] * s);
}

// x (+)= sqrt(*nrm2) * (double)d
template <typename T>
__global__ void k_axpy_back(double* __restrict__ x, const T* __restrict__ d,
                            const double* __restrict__ nrm2, int64_t n, int accumulate) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = sqrt(*nrm2) * (double)d[i];
    x[i] = accumulate ? x[i] + v : v;
}

}  // namespace

msp_status msp_norm2(msp_ctx* ctx, const double* v, int64_t n, double* out_dev) {
    k_norm2<<<1, 1024, 0, ctx->stream>>>(v, n, out_dev);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

extern "C" msp_status msp_dot(msp_ctx* ctx, const double* x, const double* y, int64_t n, double scale,
                              double* out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!x || !y || !out || n < 1) return msp_set_error(ctx, MSP_EINVAL, "dot: bad argument");
    msp::DeviceGuard g(ctx->device);
    k_dot<<<1, 1024, 0, ctx->stream>>>(x, y, n, scale, out);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_scale_cast(msp_ctx* ctx, const double* src, const double* nrm2, int64_t n,
                          msp_dtype dt, void* dst) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (dt == MSP_F32) k_scale_cast<float><<<g, 256, 0, ctx->stream>>>(src, nrm2, n, (float*)dst);
    else k_scale_cast<double><<<g, 256, 0, ctx->stream>>>(src, nrm2, n, (double*)dst);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_axpy_back(msp_ctx* ctx, double* x, const void* d, msp_dtype dt, const double* nrm2,
                         int64_t n, int accumulate) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (dt == MSP_F32) k_axpy_back<float><<<g, 256, 0, ctx->stream>>>(x, (const float*)d, nrm2, n, accumulate);
    else k_axpy_back<double><<<g, 256, 0, ctx->stream>>>(x, (const double*)d, nrm2, n, accumulate);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}
