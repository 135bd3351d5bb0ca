// Three-level MSP for (A^T A + lambda I) x = c with A in R^{m x n} of full
// column rank (Section 5): Algorithm 3 (set-up and the level-1 iteration),
// Algorithm 4 (SolveM1, level 2) and Algorithm 5 (SolveM2, level 3).
//
// Every operator of every level is a pass over the rows of one or two
// row-major FP32 matrices that share the row index (A, m x n, and
// A~ = A S^T, m x s):
//     t_r = X_r . a + beta z_r        (a row dot)
//     out = sum_r t_r Y_r             (a row combination)
// k_rowpass does both in one sweep: each CTA owns a contiguous range of rows,
// its 8 warps take one row each for the dots, then all threads fold those 8
// rows into per-CTA partial sums of Y^T t (the rows come back from L2); a
// column sum finishes the partials in a fixed order. So:
//     level 1  (A^T A + lam I) p            X = Y = A
//     SolveM1  g = A~^T (A r)               X = A,  Y = A~
//              v = A^T (A~ y), u = A~ y     X = A~, Y = A   (u kept)
//              A~^T (A v + lam~ u)          X = A,  Y = A~  (z = u)
//              w = (r - A^T (A~ y)) / lam~  X = A~, Y = A
// SolveM2's two level-3 solves apply W = A~^T A~ as its formed FP64 Gram
// (s x s, cheaper than a pass over A~ and the same operator), both in one
// two-block launch (k_level3_pcg).
// The inner levels run a fixed number of PCG steps (t2, t3) with all scalars
// on the device, so one application of SolveM1 is a fixed launch sequence;
// it is captured once into a CUDA graph and replayed per level-1 iteration.
// The level-3 preconditioners M3a^{-1}, M3b^{-1} are dense FP64 s x s
// inverses of the sketched Grams (FP64 Cholesky), applied by a dense mat-vec.
#include "bulk.cuh"
#include "msp_internal.cuh"

#include <cooperative_groups.h>

#include <cmath>
#include <cstring>
#include <new>

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 8;          // rows per CTA step: one per warp
constexpr int kVecThreads = 1024; // single-block vector kernels
constexpr int kMaxN = 8192;       // columns of A (register partials, vector kernels)

struct Pcg {
    double rz, pq, alpha, rr, beta, rzn, rzo, bb;
    double tol2;    // level 1: tol^2 |b|^2 (a breakdown counts only above it)
};

template <typename Acc>
__device__ __forceinline__ Acc fma_acc(float x, Acc a, Acc t) {
    return fma((Acc)x, a, t);
}

template <typename Acc>
__device__ __forceinline__ Acc warp_sum_t(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename Acc, int NV, bool kSame>
__global__ void __launch_bounds__(kThreads, 2) k_rowpass(
    const float* __restrict__ X, int64_t ldx, int nx4, const float* __restrict__ Y, int64_t ldy,
    int ny4, int64_t m, int64_t rows_per_cta, const Acc* __restrict__ a, const Acc* __restrict__ z,
    Acc beta, Acc* __restrict__ tout, Acc* __restrict__ part, int64_t ldp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* sa = reinterpret_cast<Acc*>(smem_raw);
    __shared__ Acc st[kRows];
    for (int i = threadIdx.x; i < nx4 * 4; i += kThreads) sa[i] = a[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Acc acc[NV][4];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = Acc(0);
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(m, r0 + rows_per_cta);
    const float* Ys = kSame ? X : Y;
    const int64_t ldys = kSame ? ldx : ldy;
    __syncthreads();
    for (int64_t g = r0; g < r1; g += kRows) {
        const int64_t r = g + warp;
        Acc t = Acc(0);
        if (r < r1) {
            const float4* xr = reinterpret_cast<const float4*>(X + r * ldx);
#pragma unroll 8
            for (int c = lane; c < nx4; c += 32) {
                const float4 v = xr[c];
                const Acc* ap = sa + 4 * c;
                t = fma_acc(v.x, ap[0], t);
                t = fma_acc(v.y, ap[1], t);
                t = fma_acc(v.z, ap[2], t);
                t = fma_acc(v.w, ap[3], t);
            }
        }
        t = warp_sum_t(t);
        if (lane == 0) {
            Acc tv = Acc(0);
            if (r < r1) {
                tv = t + (z ? beta * z[r] : Acc(0));
                if (tout) tout[r] = tv;
            }
            st[warp] = tv;
        }
        __syncthreads();
        const int nr = (int)min((int64_t)kRows, r1 - g);
#pragma unroll
        for (int rr = 0; rr < kRows; ++rr) {
            if (rr < nr) {
                const Acc tr = st[rr];
                const float4* yr = reinterpret_cast<const float4*>(Ys + (g + rr) * ldys);
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const int c = threadIdx.x + k * kThreads;
                    if (c < ny4) {
                        const float4 v = yr[c];
                        acc[k][0] = fma_acc(v.x, tr, acc[k][0]);
                        acc[k][1] = fma_acc(v.y, tr, acc[k][1]);
                        acc[k][2] = fma_acc(v.z, tr, acc[k][2]);
                        acc[k][3] = fma_acc(v.w, tr, acc[k][3]);
                    }
                }
            }
        }
        __syncthreads();
    }
    Acc* pp = part + (int64_t)blockIdx.x * ldp;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int c = threadIdx.x + k * kThreads;
        if (c < ny4) {
            pp[4 * c + 0] = acc[k][0];
            pp[4 * c + 1] = acc[k][1];
            pp[4 * c + 2] = acc[k][2];
            pp[4 * c + 3] = acc[k][3];
        }
    }
}

// The same pass with X = Y, the rows staged in shared memory: a producer warp
// streams groups of R contiguous-row copies (cp.async.bulk, one per row) into
// a ring of kRing stages guarded by mbarriers; the 8 worker warps take the row
// dots from shared memory (R < 8: 8/R warps per row, column slices combined in
// a fixed order), then fold the same rows into the per-CTA partial sums. HBM
// sees each row once and nothing is re-read through L2. One CTA per SM.
// Every wait is bounded: a timeout sets *err, the workers leave together
// (a shared flag read after a barrier), and the producer waits for its
// copies in flight before the block exits.
constexpr int kRing = 3;
constexpr int kWorkerThreads = 256;
constexpr int kWW = kWorkerThreads / 32;   // worker warps
constexpr size_t kRingHdr = 128;       // mbarriers and the abort flag
constexpr size_t kRingSaOff = 1024;    // after 64 t values and up to 32 partial dots of 8 bytes
constexpr uint32_t kRingStageMax = 64 * 1024;

__host__ __device__ constexpr size_t ring_a_bytes(int nx4, size_t acc) { return ((size_t)nx4 * 4 * acc + 127) / 128 * 128; }

struct RingShape {
    int rows;            // R, rows per stage
    int wpr;             // warps per row in the dots (R < 8), else 1
    uint32_t row_bytes;  // nx4 * 16
    uint32_t stage_bytes;
};

template <typename Acc, int NV, bool kSame>
__global__ void __launch_bounds__(kWorkerThreads + 32, 1) k_rowpass_ring(
    const float* __restrict__ X, int64_t ldx, int nx4, const float* __restrict__ Y, int64_t ldy, int ny4,
    int64_t m, int64_t rows_per_cta, RingShape sh,
    const Acc* __restrict__ a, const Acc* __restrict__ z, Acc beta, Acc* __restrict__ tout,
    Acc* __restrict__ part, int64_t ldp, int* err) {
    extern __shared__ __align__(128) unsigned char ring_smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(ring_smem);
    uint64_t* empty = full + kRing;
    int* abort_flag = reinterpret_cast<int*>(empty + kRing);
    Acc* st = reinterpret_cast<Acc*>(ring_smem + kRingHdr);             // up to 64 t values
    Acc* sp = st + 64;                                                 // kWW partial dots
    Acc* sa = reinterpret_cast<Acc*>(ring_smem + kRingSaOff);
    unsigned char* ring = ring_smem + kRingSaOff + ring_a_bytes(nx4, sizeof(Acc));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(m, r0 + rows_per_cta);
    const int ngroups = (int)((r1 - r0 + sh.rows - 1) / sh.rows);
    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            msp::mbar_init(&full[s], 1);
            msp::mbar_init(&empty[s], 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < nx4 * 4; i += blockDim.x) sa[i] = a[i];
    __syncthreads();

    if (warp == kWW) {
        // ---- producer
        if (lane == 0) {
            uint32_t k = 0;
            for (int gi = 0; gi < ngroups; ++gi, ++k) {
                const int s = (int)(k % kRing);
                if (k >= (uint32_t)kRing && !msp::mbar_wait_timed(&empty[s], ((k / kRing) & 1u) ^ 1u, err)) break;
                const int64_t g0 = r0 + (int64_t)gi * sh.rows;
                const int nr = (int)min((int64_t)sh.rows, r1 - g0);
                unsigned char* dst = ring + (size_t)s * sh.stage_bytes;
                const uint32_t yb = kSame ? 0u : (uint32_t)ny4 * 16u;
                msp::mbar_arrive_expect_tx(&full[s], (uint32_t)nr * (sh.row_bytes + yb));
                for (int r = 0; r < nr; ++r)
                    msp::bulk_g2s(dst + (size_t)r * sh.row_bytes, X + (g0 + r) * ldx, sh.row_bytes, &full[s]);
                if (!kSame && yb > 0)
                    for (int r = 0; r < nr; ++r)
                        msp::bulk_g2s(dst + (size_t)sh.rows * sh.row_bytes + (size_t)r * yb, Y + (g0 + r) * ldy, yb,
                                      &full[s]);
            }
            // every issued copy lands before the block exits
            const uint32_t kb = k > (uint32_t)kRing ? k - kRing : 0u;
            for (uint32_t q = kb; q < k; ++q)
                if (!msp::mbar_wait_timed(&full[q % kRing], (q / kRing) & 1u, err)) break;
        }
        return;
    }

    // ---- workers
    Acc acc[NV][4];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = Acc(0);
    for (int gi = 0; gi < ngroups; ++gi) {
        const int s = gi % kRing;
        const uint32_t par = (uint32_t)(gi / kRing) & 1u;
        // a timed-out wait is seen by every worker at the barrier after the
        // dots (that warp's dots read stale shared memory, in bounds)
        if (!msp::mbar_wait_timed(&full[s], par, err) && lane == 0) atomicExch(abort_flag, 1);
        const int64_t g0 = r0 + (int64_t)gi * sh.rows;
        const int nr = (int)min((int64_t)sh.rows, r1 - g0);
        const float4* rows4 = reinterpret_cast<const float4*>(ring + (size_t)s * sh.stage_bytes);
        // row dots
        if (sh.wpr > 1) {
            const int row = warp / sh.wpr, part_i = warp % sh.wpr;
            const int per = (nx4 + sh.wpr - 1) / sh.wpr;
            const int c0 = part_i * per, c1 = min(nx4, c0 + per);
            Acc tp = Acc(0);
            if (row < nr) {
                const float4* xr = rows4 + (size_t)row * nx4;
#pragma unroll 4
                for (int c = c0 + lane; c < c1; c += 32) {
                    const float4 v = xr[c];
                    tp = fma_acc(v.x, sa[4 * c + 0], tp);
                    tp = fma_acc(v.y, sa[4 * c + 1], tp);
                    tp = fma_acc(v.z, sa[4 * c + 2], tp);
                    tp = fma_acc(v.w, sa[4 * c + 3], tp);
                }
            }
            tp = warp_sum_t(tp);
            if (lane == 0) sp[warp] = tp;
            msp::bar_workers<kWorkerThreads>();
            if (tid < nr) {
                Acc tv = Acc(0);
                for (int q = 0; q < sh.wpr; ++q) tv += sp[tid * sh.wpr + q];
                const int64_t r = g0 + tid;
                tv += z ? beta * z[r] : Acc(0);
                if (tout) tout[r] = tv;
                st[tid] = tv;
            }
        } else {
            for (int row = warp; row < nr; row += kWW) {
                const float4* xr = rows4 + (size_t)row * nx4;
                Acc tp = Acc(0);
#pragma unroll 4
                for (int c = lane; c < nx4; c += 32) {
                    const float4 v = xr[c];
                    tp = fma_acc(v.x, sa[4 * c + 0], tp);
                    tp = fma_acc(v.y, sa[4 * c + 1], tp);
                    tp = fma_acc(v.z, sa[4 * c + 2], tp);
                    tp = fma_acc(v.w, sa[4 * c + 3], tp);
                }
                tp = warp_sum_t(tp);
                if (lane == 0) {
                    const int64_t r = g0 + row;
                    tp += z ? beta * z[r] : Acc(0);
                    if (tout) tout[r] = tp;
                    st[row] = tp;
                }
            }
        }
        msp::bar_workers<kWorkerThreads>();
        if (*(volatile int*)abort_flag) break;
        // fold the stage's rows (of X itself, or the staged rows of Y)
        const float4* ybase = kSame ? rows4 : rows4 + (size_t)sh.rows * nx4;
        const int nf4 = kSame ? nx4 : ny4;
        for (int row = 0; row < nr; ++row) {
            const Acc tr = st[row];
            const float4* yr = ybase + (size_t)row * nf4;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const int c = tid + q * kWorkerThreads;
                if (c < nf4) {
                    const float4 v = yr[c];
                    acc[q][0] = fma_acc(v.x, tr, acc[q][0]);
                    acc[q][1] = fma_acc(v.y, tr, acc[q][1]);
                    acc[q][2] = fma_acc(v.z, tr, acc[q][2]);
                    acc[q][3] = fma_acc(v.w, tr, acc[q][3]);
                }
            }
        }
        msp::bar_workers<kWorkerThreads>();
        if (tid == 0) msp::mbar_arrive(&empty[s]);
    }
    Acc* pp = part + (int64_t)blockIdx.x * ldp;
    const int nf4 = kSame ? nx4 : ny4;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int c = tid + q * kWorkerThreads;
        if (c < nf4) {
            pp[4 * c + 0] = acc[q][0];
            pp[4 * c + 1] = acc[q][1];
            pp[4 * c + 2] = acc[q][2];
            pp[4 * c + 3] = acc[q][3];
        }
    }
}

// out[j] = alpha sum_g part[g][j] + beta w[j] + v[j] (w, v optional), the
// partials summed in FP64 in a fixed order. Block 32 x 8: 32 columns, the
// G partial rows split over 8 thread rows, combined in a fixed order.
template <typename Acc>
__global__ void k_colsum(const Acc* __restrict__ part, int64_t ldp, int G, int ny, double alpha,
                         const Acc* __restrict__ w, double beta, const Acc* __restrict__ v,
                         Acc* __restrict__ out) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + tx;
    double s = 0.0;
    if (j < ny)
        for (int g = ty; g < G; g += 8) s += (double)part[(int64_t)g * ldp + j];
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && j < ny) {
        double tot = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) tot += red[q][tx];
        double o = alpha * tot;
        if (w) o += beta * (double)w[j];
        if (v) o += (double)v[j];
        out[j] = (Acc)o;
    }
}

// ------------------------------------------------- single-block vector steps

__device__ double block_sum(double v, double* red) {
    v = warp_sum_t(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Compensated FP32 dot products (the FP64 pipe of this part is about 2 DFMA
// per clock per SM, too slow for per-element FP64 on one SM): each product
// is split exactly by FMA (TwoProd) and accumulated with TwoSum into a
// float pair; warps combine pairs the same way and the block adds the 32
// warp sums in FP64, in a fixed order.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void ff_add_prod(FF& acc, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo += e + pe;
}

__device__ double block_sum_ff(FF v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, v.hi, o);
        const float l = __shfl_xor_sync(0xffffffffu, v.lo, o);
        float s, e;
        two_sum(v.hi, h, s, e);
        v.hi = s;
        v.lo += l + e;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = (double)v.hi + (double)v.lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// x = 0, r = b, bb = b.b
__global__ void k_pcg_init(int len, const float* __restrict__ b, float* __restrict__ x,
                           float* __restrict__ r, Pcg* sc) {
    __shared__ double red[33];
    FF a{0.f, 0.f};
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float v = b[i];
        x[i] = 0.f;
        r[i] = v;
        ff_add_prod(a, v, v);
    }
    const double s = block_sum_ff(a, red);
    if (threadIdx.x == 0) {
        sc->bb = s;
        sc->rr = s;
    }
}

// rz = r.z, p = z, zo = z
__global__ void k_pcg_start(int len, const float* __restrict__ r, const float* __restrict__ z,
                            float* __restrict__ p, float* __restrict__ zo, Pcg* sc) {
    __shared__ double red[33];
    FF a{0.f, 0.f};
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float v = z[i];
        p[i] = v;
        zo[i] = v;
        ff_add_prod(a, r[i], v);
    }
    const double s = block_sum_ff(a, red);
    if (threadIdx.x == 0) sc->rz = s;
}

// pq = p.q; alpha = rz / pq (0 when the step is undefined); x += alpha p;
// r -= alpha q; rr = r.r
__global__ void k_pcg_step(int len, const float* __restrict__ p, const float* __restrict__ q,
                           float* __restrict__ x, float* __restrict__ r, Pcg* sc, int* err) {
    __shared__ double red[33];
    FF a{0.f, 0.f};
    for (int i = threadIdx.x; i < len; i += blockDim.x) ff_add_prod(a, p[i], q[i]);
    const double pq = block_sum_ff(a, red);
    const double rz = sc->rz;
    double alpha = 0.0;
    if (pq > 0.0 && isfinite(pq) && isfinite(rz)) alpha = rz / pq;
    else if (err && threadIdx.x == 0 && rz != 0.0 && sc->rr > sc->tol2)
        atomicCAS(err, 0, isfinite(pq) ? (int)MSP_ENOTPD : (int)MSP_ENONFINITE);
    const float af = (float)alpha;
    FF a2{0.f, 0.f};
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        x[i] = fmaf(af, p[i], x[i]);
        const float rv = fmaf(-af, q[i], r[i]);
        r[i] = rv;
        ff_add_prod(a2, rv, rv);
    }
    const double rr = block_sum_ff(a2, red);
    if (threadIdx.x == 0) {
        sc->pq = pq;
        sc->alpha = alpha;
        sc->rr = rr;
    }
}

// rzn = r.z; flexible: beta = (rzn - r.zo) / rz, else rzn / rz; p = z + beta p;
// zo = z; rz = rzn
__global__ void k_pcg_dir(int len, const float* __restrict__ r, const float* __restrict__ z,
                          float* __restrict__ zo, float* __restrict__ p, Pcg* sc, int flexible) {
    __shared__ double red[33];
    FF a1{0.f, 0.f}, a2{0.f, 0.f};
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float rv = r[i];
        ff_add_prod(a1, rv, z[i]);
        ff_add_prod(a2, rv, zo[i]);
    }
    const double rzn = block_sum_ff(a1, red);
    const double rzo = flexible ? block_sum_ff(a2, red) : 0.0;
    const double rz = sc->rz;
    double beta = 0.0;
    if (rz != 0.0 && isfinite(rz)) beta = (rzn - rzo) / rz;
    if (!isfinite(beta)) beta = 0.0;
    const float bf = (float)beta;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float zv = z[i];
        p[i] = fmaf(bf, p[i], zv);
        zo[i] = zv;
    }
    if (threadIdx.x == 0) {
        sc->rzn = rzn;
        sc->rzo = rzo;
        sc->beta = beta;
        sc->rz = rzn;
    }
}

// out = M v for a dense s_pad x s_pad FP64 M (row-major), one warp per row
__global__ void k_dense_mv(const double* __restrict__ M, const float* __restrict__ v, int sp,
                           float* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= sp) return;
    const double2* mr = reinterpret_cast<const double2*>(M + (int64_t)row * sp);
    const float2* vv = reinterpret_cast<const float2*>(v);
    double s = 0.0;
    for (int c = lane; c < sp / 2; c += 32) {
        const double2 a = mr[c];
        const float2 b = vv[c];
        s = fma(a.x, (double)b.x, s);
        s = fma(a.y, (double)b.y, s);
    }
    s = warp_sum_t(s);
    if (lane == 0) out[row] = (float)s;
}

// Algorithm 5 steps 2-3 in one launch: block 0 runs t3 PCG steps on
// W u = r preconditioned by M3a^{-1}, block 1 on (W + lam~ I) v = r with
// M3b^{-1}; W = A~^T A~ is the formed FP64 Gram (the same operator as
// A~^T (A~ .), applied as an s x s product). Thread i < s_pad owns component
// i; every dense product is split over 1024 / s_pad threads per component
// (j ranges, combined in a fixed order) and reads columns of the symmetric
// matrices (coalesced across threads). FP64 throughout; s_pad <= 1024.
__global__ void __launch_bounds__(1024) k_level3_pcg(const double* __restrict__ W, const double* __restrict__ Ma,
                                                    const double* __restrict__ Mb, double lam_t, int sp, int t3,
                                                    const float* __restrict__ b, float* __restrict__ u,
                                                    float* __restrict__ v) {
    __shared__ double red[33];
    __shared__ double vec[1024], pbuf[1024];
    const int tid = threadIdx.x;
    const int parts = max(1, 1024 / sp);
    const int per = (sp + parts - 1) / parts;
    const int ci = tid % sp, part = tid / sp;
    const bool own = tid < sp;
    const double* M = blockIdx.x == 0 ? Ma : Mb;
    const double shift = blockIdx.x == 0 ? 0.0 : lam_t;
    float* out = blockIdx.x == 0 ? u : v;
    // y = Mat vec for the owner threads (vec staged in shared memory by the caller)
    auto mv = [&](const double* Mat) {
        double s = 0.0;
        if (part < parts) {
            const int j0 = part * per, j1 = min(sp, j0 + per);
#pragma unroll 8
            for (int j = j0; j < j1; ++j) s = fma(Mat[(int64_t)j * sp + ci], vec[j], s);
        }
        pbuf[tid] = s;
        __syncthreads();
        double y = 0.0;
        if (own)
            for (int q = 0; q < parts; ++q) y += pbuf[ci + q * sp];
        return y;
    };
    double x = 0.0, r = own ? (double)b[tid] : 0.0;
    vec[tid] = r;
    __syncthreads();
    double z = mv(M);
    double rz = block_sum(own ? r * z : 0.0, red);
    double p = z;
    for (int k = 0; k < t3; ++k) {
        __syncthreads();
        vec[tid] = own ? p : 0.0;
        __syncthreads();
        const double q = mv(W) + shift * p;
        const double pq = block_sum(own ? p * q : 0.0, red);
        const double alpha = (pq > 0.0 && rz != 0.0) ? rz / pq : 0.0;
        x = fma(alpha, p, x);
        r = fma(-alpha, q, r);
        if (k + 1 < t3) {
            __syncthreads();
            vec[tid] = own ? r : 0.0;
            __syncthreads();
            z = mv(M);
            const double rzn = block_sum(own ? r * z : 0.0, red);
            const double beta = rz != 0.0 ? rzn / rz : 0.0;
            p = fma(beta, p, z);
            rz = rzn;
        }
    }
    if (own) out[tid] = (float)x;
}

// The same two level-3 solves on two thread-block clusters of kCl CTAs
// (cluster 0: W u = r with M3a^{-1}; cluster 1: (W + lam~ I) v = r with
// M3b^{-1}). CTA `rank` owns components [rank s_pad / kCl, (rank + 1) s_pad /
// kCl); each warp forms whole rows of the symmetric matrices (lanes over
// columns, coalesced), so the FP64 products run on 2 kCl SMs instead of two.
// Vector slices and dot partials are broadcast to every CTA of the cluster
// through distributed shared memory; cluster barriers order the steps (no
// spin-waits). The dot partials are summed in rank order, so every CTA takes
// the same scalars. s_pad <= 1024, s_pad divisible by kCl.
constexpr int kCl = 8;

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(1024)
    k_level3_cluster(const double* __restrict__ W, const double* __restrict__ Ma, const double* __restrict__ Mb,
                     double lam_t, int sp, int t3, const float* __restrict__ b, float* __restrict__ u,
                     float* __restrict__ v) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double vec[1024];          // the full vector of the next product
    __shared__ double part[2][kCl];       // dot partials, one slot per rank
    __shared__ double loc[32];
    const int rank = (int)cl.block_rank();
    const int sys = blockIdx.x / kCl;
    const double* M = sys == 0 ? Ma : Mb;
    const double shift = sys == 0 ? 0.0 : lam_t;
    float* out = sys == 0 ? u : v;
    const int own = sp / kCl, i0 = rank * own;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // owner state: thread c < own keeps component i0 + c
    double x = 0.0, r = 0.0, z = 0.0, p = 0.0;
    // y_c = (Mat vec)_(i0 + c) for the owned rows, into ys (shared)
    __shared__ double ys[1024];
    auto mv = [&](const double* Mat) {
        for (int c = warp; c < own; c += 32) {
            const double* row = Mat + (int64_t)(i0 + c) * sp;
            double s = 0.0;
            for (int j = lane; j < sp; j += 32) s = fma(row[j], vec[j], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) ys[c] = s;
        }
        __syncthreads();
    };
    // every CTA's vec <- the owners' values (slices from all ranks)
    auto broadcast = [&](double val) {
        if (tid < own)
            for (int q = 0; q < kCl; ++q) {
                double* dst = cl.map_shared_rank(vec, q);
                dst[i0 + tid] = val;
            }
        cl.sync();
    };
    // cluster-wide sum of one value per owner thread, fixed order
    auto csum = [&](double val, int slot) {
        double s = tid < own ? val : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) loc[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 32; ++w) t += loc[w];
            for (int q = 0; q < kCl; ++q) cl.map_shared_rank(&part[slot][0], q)[rank] = t;
        }
        cl.sync();
        double tot = 0.0;
        for (int q = 0; q < kCl; ++q) tot += part[slot][q];
        return tot;
    };
    if (tid < own) r = (double)b[i0 + tid];
    broadcast(r);
    mv(M);
    if (tid < own) z = ys[tid];
    double rz = csum(r * z, 0);
    p = z;
    for (int k = 0; k < t3; ++k) {
        broadcast(p);
        mv(W);
        const double q = tid < own ? ys[tid] + shift * p : 0.0;
        const double pq = csum(p * q, 1);
        const double alpha = (pq > 0.0 && rz != 0.0) ? rz / pq : 0.0;
        x = fma(alpha, p, x);
        r = fma(-alpha, q, r);
        if (k + 1 < t3) {
            broadcast(r);
            mv(M);
            if (tid < own) z = ys[tid];
            const double rzn = csum(r * z, 0);
            const double beta = rz != 0.0 ? rzn / rz : 0.0;
            p = fma(beta, p, z);
            rz = rzn;
        }
    }
    if (tid < own) out[i0 + tid] = (float)x;
    cl.sync();   // no CTA leaves while others may still write its shared memory
}

// out = a x + b y
__global__ void k_axpby(int len, float a, const float* __restrict__ x, float b,
                        const float* __restrict__ y, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = a * x[i] + b * y[i];
}

// ------------------------------------------------------ FP64 refinement

__global__ void k_norm2_64(int len, const double* __restrict__ v, double* out) {
    __shared__ double red[33];
    double s = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) s += v[i] * v[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_scale_to_f32(int len, const double* __restrict__ r, double inv, float* __restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) b[i] = (float)(r[i] * inv);
}

__global__ void k_axpy_64(int len, double a, const float* __restrict__ d, double* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) x[i] += a * (double)d[i];
}

__global__ void k_pad_copy_64(int len, int n, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) dst[i] = (i < n) ? src[i] : 0.0;
}

__global__ void k_pad_copy_32(int len, int n, const float* __restrict__ src, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) dst[i] = (i < n) ? src[i] : 0.f;
}

}  // namespace

// ------------------------------------------------------------ the handle

struct msp_general_s {
    cudaStream_t stream = nullptr;
    int device = 0;
    int64_t m = 0, n = 0, n_pad = 0, lda = 0, s = 0, s_pad = 0, phi = 0;
    int gamma = 0, gamma_phi = 0;
    uint64_t seed = 0;
    double lambda = 0, lambda0 = 0, lam_tilde = 0;
    double shift_a = 0, shift_b = 0;
    int retries_a = 0, retries_b = 0;
    const float* A = nullptr;       // user's A, or A_copy
    float* A_copy = nullptr;        // padded copy when the user's rows are not 16-byte aligned
    float* At = nullptr;            // A~ = A S^T, m x s_pad
    double* M3a = nullptr;          // (A^^T A^)^{-1}, s_pad x s_pad FP64
    double* M3b = nullptr;          // (A^^T A^ + lam~ I)^{-1}
    double* G3a = nullptr;          // A^^T A^ (FP64, before the shift), for tests
    double* G3b = nullptr;
    double* Linv = nullptr;         // FP64 scratch for the factorisations
    void* work = nullptr;
    float *x1, *r1, *z1, *zo1, *p1, *q1, *b1;
    float *g2, *y2, *r2, *z2, *zo2, *p2, *q2;
    float *u3, *v3;
    float *tm, *vn, *part;
    double *part64, *x64, *r64, *c64, *d64;
    Pcg* sc = nullptr;              // [0] level 1, [1] level 2
    int* err = nullptr;
    double* host = nullptr;         // pinned: 16 doubles
    int G = 0;
    int64_t rows_per_cta = 0;
    int64_t ldp = 0;                // row stride of the partials: max(n_pad, s_pad)
    // direct modes: W = A~^T A~, M2^{-1} = (W^{-1} - (W + lam~ I)^{-1}) / lam~
    // (level 3 exact); C = A^T A~ and (C^T C + lam~ W)^{-1} (level 2 exact)
    double* W64 = nullptr;
    double* M2inv = nullptr;
    float* Cm = nullptr;            // n64 x s_pad FP32
    double* Binv = nullptr;
    float* zeros = nullptr;         // s_pad zeros
    int64_t n64 = 0;
    // least squares: the inner handle on A~ = Phi A whose solves precondition
    // the level-1 iteration of this handle (A^T A x = A^T b)
    msp_general_s* inner = nullptr;
    float* As = nullptr;            // A~ (owned), s_ls x n_pad
    int64_t s_ls = 0;
    double inner_tol = 1e-2;
    int inner_maxit = 50;
    int check_every = 4;            // level-1 iterations between host checks
    cudaStream_t cap = nullptr;     // private stream the SolveM1 graph is captured on
    cudaGraphExec_t m1_exec = nullptr;
    int m1_t2 = -1, m1_t3 = -1;
    int m1_kernels = 0;
    // one whole level-1 iteration (operator, step, SolveM1, direction)
    cudaGraphExec_t it_exec = nullptr;
    int it_t2 = -1, it_t3 = -1;
    int it_kernels = 0;
};

namespace {

using G_t = msp_general_s;

// rows [0, rows) split into `ctas` contiguous ranges of rows_per_cta
struct RowGrid {
    int64_t rows, rows_per_cta;
    int ctas;
};

RowGrid make_grid(int64_t rows, int num_sms) {
    RowGrid rg;
    rg.rows = rows;
    int G = (int)std::min<int64_t>(2 * num_sms, (rows + kRows - 1) / kRows);
    rg.rows_per_cta = round_up((rows + G - 1) / G, kRows);
    rg.ctas = (int)((rows + rg.rows_per_cta - 1) / rg.rows_per_cta);
    return rg;
}

template <typename Acc, bool kSame>
msp_status launch_rowpass_rg(msp_ctx* ctx, cudaStream_t strm, const RowGrid& rg, const float* X, int64_t ldx,
                             int nx4, const float* Y, int64_t ldy, int ny4, const Acc* a, const Acc* z, Acc beta,
                             Acc* tout, Acc* part, int64_t ldp, int* count) {
    const size_t smem = (size_t)nx4 * 4 * sizeof(Acc);
    const int nv = (ny4 + kThreads - 1) / kThreads;
#define MSP_RP(NVV)                                                                                     \
    case NVV: {                                                                                         \
        auto kern = k_rowpass<Acc, NVV, kSame>;                                                         \
        kern<<<rg.ctas, kThreads, smem, strm>>>(X, ldx, nx4, Y, ldy, ny4, rg.rows, rg.rows_per_cta, a,  \
                                                z, beta, tout, part, ldp);                              \
        break;                                                                                          \
    }
    switch (nv <= 1 ? 1 : nv <= 2 ? 2 : nv <= 4 ? 4 : 8) {
        MSP_RP(1)
        MSP_RP(2)
        MSP_RP(4)
        MSP_RP(8)
    }
#undef MSP_RP
    MSP_CHECK_LAUNCH(ctx);
    if (count) ++*count;
    return MSP_OK;
}

template <typename Acc, bool kSame>
msp_status launch_rowpass_nv(msp_ctx* ctx, cudaStream_t strm, G_t* g, const float* X, int64_t ldx, int nx4,
                             const float* Y, int64_t ldy, int ny4, const Acc* a, const Acc* z, Acc beta, Acc* tout,
                             Acc* part, int64_t ldp, int* count) {
    const RowGrid rg{g->m, g->rows_per_cta, g->G};
    return launch_rowpass_rg<Acc, kSame>(ctx, strm, rg, X, ldx, nx4, Y, ldy, ny4, a, z, beta, tout, part, ldp,
                                         count);
}

template <typename Acc>
msp_status set_rowpass_attrs(msp_ctx* ctx, size_t smem) {
#define MSP_RA(NVV)                                                                                        \
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_rowpass<Acc, NVV, true>,                                     \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));      \
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_rowpass<Acc, NVV, false>,                                    \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MSP_RA(1)
    MSP_RA(2)
    MSP_RA(4)
    MSP_RA(8)
#undef MSP_RA
    return MSP_OK;
}

// Ring shape for rows of nx4 float4 (plus ny4_staged of Y): R rows per stage
// within kRingStageMax and the shared-memory budget; R < 8 takes 8/R warps
// per row in the dots.
// Returns false when not even one row fits (the caller uses k_rowpass).
bool ring_shape(int nx4, int ny4_staged, size_t acc, size_t smem_optin, RingShape* sh, size_t* smem) {
    const uint32_t rb = (uint32_t)nx4 * 16u;
    const uint32_t rby = (uint32_t)ny4_staged * 16u;
    const size_t fixed = kRingSaOff + ring_a_bytes(nx4, acc);
    if (smem_optin <= fixed) return false;
    const size_t per_stage = std::min<size_t>(kRingStageMax, (smem_optin - fixed) / kRing / 128 * 128);
    int R = (int)(per_stage / (rb + rby));
    if (R < 1) return false;
    if (R > 64) R = 64;
    sh->rows = R;
    sh->wpr = R >= kWW ? 1 : kWW / R;     // e.g. R = 3, 8 warps: 2 warps per row, 2 warps idle in the dots
    sh->row_bytes = rb;
    sh->stage_bytes = (uint32_t)(((size_t)R * (rb + rby) + 127) / 128 * 128);
    *smem = fixed + (size_t)kRing * sh->stage_bytes;
    return true;
}

template <typename Acc>
msp_status set_ring_attrs(msp_ctx* ctx) {
    const int lim = (int)ctx->smem_optin;
#define MSP_RG(NVV)                                                                                        \
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_rowpass_ring<Acc, NVV, true>,                               \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, lim));         \
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_rowpass_ring<Acc, NVV, false>,                              \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MSP_RG(1)
    MSP_RG(2)
    MSP_RG(4)
    MSP_RG(8)
#undef MSP_RG
    return MSP_OK;
}

// The pass over rows [0, rows) of X (and Y): the staged ring when a row of
// each fits, else k_rowpass. Y == X (same ld and width) streams the rows
// once. ny4 = 0: row dots only (tout), nothing folded. `max_ctas` bounds the
// grid (rows of the partials buffer); *ctas_used is what the column sum reads.
template <typename Acc>
msp_status launch_pass(msp_ctx* ctx, cudaStream_t strm, int max_ctas, int64_t rows, const float* X, int64_t ldx,
                       int nx4, const float* Y, int64_t ldy, int ny4, const Acc* a, const Acc* z, Acc beta,
                       Acc* tout, Acc* part, int64_t ldp, int* err, int* count, int* ctas_used) {
    const bool same = (Y == X && ldy == ldx && ny4 == nx4);
    RingShape sh;
    size_t smem = 0;
    if (nx4 > 0 && ring_shape(nx4, same ? 0 : ny4, sizeof(Acc), ctx->smem_optin, &sh, &smem)) {
        const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(ctx->num_sms, max_ctas),
                                                                      (rows + sh.rows - 1) / sh.rows));
        const int64_t rpc = (rows + ctas - 1) / ctas;
        const int nv = (std::max(same ? nx4 : ny4, 1) + kWorkerThreads - 1) / kWorkerThreads;
#define MSP_RL(NVV)                                                                                         \
    case NVV:                                                                                               \
        if (same)                                                                                           \
            k_rowpass_ring<Acc, NVV, true><<<ctas, kWorkerThreads + 32, smem, strm>>>(                      \
                X, ldx, nx4, X, ldx, nx4, rows, rpc, sh, a, z, beta, tout, part, ldp, err);                 \
        else                                                                                                \
            k_rowpass_ring<Acc, NVV, false><<<ctas, kWorkerThreads + 32, smem, strm>>>(                     \
                X, ldx, nx4, Y, ldy, ny4, rows, rpc, sh, a, z, beta, tout, part, ldp, err);                 \
        break;
        switch (nv <= 1 ? 1 : nv <= 2 ? 2 : nv <= 4 ? 4 : 8) {
            MSP_RL(1)
            MSP_RL(2)
            MSP_RL(4)
            MSP_RL(8)
        }
#undef MSP_RL
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        *ctas_used = (int)((rows + rpc - 1) / rpc);
        return MSP_OK;
    }
    const RowGrid rg = make_grid(rows, ctx->num_sms);
    *ctas_used = rg.ctas;
    if (same)
        return launch_rowpass_rg<Acc, true>(ctx, strm, rg, X, ldx, nx4, X, ldx, nx4, a, z, beta, tout, part, ldp,
                                            count);
    return launch_rowpass_rg<Acc, false>(ctx, strm, rg, X, ldx, nx4, Y, ldy, ny4, a, z, beta, tout, part, ldp,
                                         count);
}

template <typename Acc>
msp_status launch_same(msp_ctx* ctx, cudaStream_t strm, int max_ctas, int64_t rows, const float* X, int64_t ldx,
                       int nx4, const Acc* a, const Acc* z, Acc beta, Acc* tout, Acc* part, int64_t ldp, int* err,
                       int* count, int* ctas_used) {
    return launch_pass<Acc>(ctx, strm, max_ctas, rows, X, ldx, nx4, X, ldx, nx4, a, z, beta, tout, part, ldp, err,
                            count, ctas_used);
}

// out = alpha (sum of the pass over the rows) + beta w + v
template <typename Acc>
msp_status colsum(msp_ctx* ctx, cudaStream_t strm, G_t* g, const Acc* part, int64_t ldp, int ny, double alpha, const Acc* w,
                  double beta, const Acc* v, Acc* out, int* count, int ctas = 0) {
    k_colsum<Acc><<<(unsigned)((ny + 31) / 32), 256, 0, strm>>>(part, ldp, ctas ? ctas : g->G, ny, alpha, w, beta,
                                                              v, out);
    MSP_CHECK_LAUNCH(ctx);
    if (count) ++*count;
    return MSP_OK;
}

// The levels' operators. `ld` of the partials is the widest vector (n_pad).
struct Ops {
    msp_ctx* ctx;
    G_t* g;
    int* count;
    cudaStream_t strm;
    int64_t ldp() const { return g->ldp; }
    int na4() const { return (int)(g->n_pad / 4); }
    int ns4() const { return (int)(g->s_pad / 4); }

    // q = (A^T A + lam I) p  (level 1)
    msp_status op1(const float* p, float* q) {
        int used = 0;
        MSP_TRY(launch_same<float>(ctx, strm, g->G, g->m, g->A, g->lda, na4(), p, nullptr, 0.f, nullptr, g->part,
                                   ldp(), g->err, count, &used));
        return colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->n_pad, 1.0, p, g->lambda, nullptr, q, count,
                             used);
    }
    // out = A~^T (A r)
    msp_status sketch_rhs(const float* r, float* out) {
        int used = 0;
        MSP_TRY(launch_pass<float>(ctx, strm, g->G, g->m, g->A, g->lda, na4(), g->At, g->s_pad, ns4(), r, nullptr, 0.f,
                                   nullptr, g->part, ldp(), g->err, count, &used));
        return colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->s_pad, 1.0, nullptr, 0.0, nullptr, out, count,
                             used);
    }
    // q = (A~^T A A^T A~ + lam~ A~^T A~) y  (level 2)
    msp_status op2(const float* y, float* q) {
        int used = 0;
        MSP_TRY(launch_pass<float>(ctx, strm, g->G, g->m, g->At, g->s_pad, ns4(), g->A, g->lda, na4(), y, nullptr, 0.f,
                                   g->tm, g->part, ldp(), g->err, count, &used));
        MSP_TRY(colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->n_pad, 1.0, nullptr, 0.0, nullptr, g->vn, count,
                              used));
        MSP_TRY(launch_pass<float>(ctx, strm, g->G, g->m, g->A, g->lda, na4(), g->At, g->s_pad, ns4(), g->vn, g->tm,
                                   (float)g->lam_tilde, nullptr, g->part, ldp(), g->err, count, &used));
        return colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->s_pad, 1.0, nullptr, 0.0, nullptr, q, count, used);
    }
    // w = (r - A^T (A~ y)) / lam~  (Algorithm 4 step 3)
    msp_status finish_m1(const float* y, const float* r, float* w) {
        int used = 0;
        MSP_TRY(launch_pass<float>(ctx, strm, g->G, g->m, g->At, g->s_pad, ns4(), g->A, g->lda, na4(), y, nullptr, 0.f,
                                   nullptr, g->part, ldp(), g->err, count, &used));
        const double il = 1.0 / g->lam_tilde;
        return colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->n_pad, -il, r, il, nullptr, w, count, used);
    }
    // Algorithm 4 with the level-2 system solved exactly through the formed
    // C = A^T A~: w = (r - C (C^T C + lam~ W)^{-1} C^T r) / lam~
    msp_status solve_m1_direct(const float* r, float* w) {
        const RowGrid rg = make_grid(g->n_pad, ctx->num_sms);
        const int ns4 = (int)(g->s_pad / 4);
        // h = C^T r: row combination with t_j = r_j (zero row dots)
        int used = 0;
        MSP_TRY(launch_same<float>(ctx, strm, rg.ctas, g->n_pad, g->Cm, g->s_pad, ns4, g->zeros, r, 1.f, nullptr,
                                   g->part, ldp(), g->err, count, &used));
        MSP_TRY(colsum<float>(ctx, strm, g, g->part, ldp(), (int)g->s_pad, 1.0, nullptr, 0.0, nullptr, g->g2, count,
                              used));
        MSP_TRY(dense(g->Binv, g->g2, g->y2));
        // t = C y (row dots only), w = (r - t) / lam~
        MSP_TRY(launch_pass<float>(ctx, strm, rg.ctas, g->n_pad, g->Cm, g->s_pad, ns4, g->Cm, g->s_pad, 0, g->y2,
                                   nullptr, 0.f, g->vn, g->part, ldp(), g->err, count, &used));
        const int np = (int)g->n_pad;
        const float il = (float)(1.0 / g->lam_tilde);
        k_axpby<<<(unsigned)((np + 255) / 256), 256, 0, strm>>>(np, il, r, -il, g->vn, w);
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        return MSP_OK;
    }
    msp_status dense(const double* M, const float* v, float* out) {
        const int sp = (int)g->s_pad;
        k_dense_mv<<<(unsigned)((sp + 7) / 8), 256, 0, strm>>>(M, v, sp, out);
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        return MSP_OK;
    }
    msp_status vec(int which, int len, const float* a0, const float* a1, float* a2, float* a3, Pcg* sc,
                   int flexible = 0) {
        switch (which) {
            case 0: k_pcg_init<<<1, kVecThreads, 0, strm>>>(len, a0, a2, a3, sc); break;
            case 1: k_pcg_start<<<1, kVecThreads, 0, strm>>>(len, a0, a1, a2, a3, sc); break;
            // the fixed-step inner levels only freeze a step with p.q <= 0
            case 2: k_pcg_step<<<1, kVecThreads, 0, strm>>>(len, a0, a1, a2, a3, sc, sc == g->sc ? g->err : nullptr); break;
            default: k_pcg_dir<<<1, kVecThreads, 0, strm>>>(len, a0, a1, a2, a3, sc, flexible); break;
        }
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        return MSP_OK;
    }

    // Algorithm 5: z = (u - v) / lam~ (t3 = 0: the exact M2^{-1} r); both
    // level-3 solves run in one launch on the formed W
    msp_status solve_m2(const float* r, float* z, int t3) {
        if (t3 == 0) return dense(g->M2inv, r, z);
        const int sp = (int)g->s_pad;
        if (sp % kCl == 0)
            k_level3_cluster<<<2 * kCl, 1024, 0, strm>>>(g->W64, g->M3a, g->M3b, g->lam_tilde, sp, t3, r, g->u3,
                                                         g->v3);
        else
            k_level3_pcg<<<2, 1024, 0, strm>>>(g->W64, g->M3a, g->M3b, g->lam_tilde, sp, t3, r, g->u3, g->v3);
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        const float il = (float)(1.0 / g->lam_tilde);
        k_axpby<<<(unsigned)((sp + 255) / 256), 256, 0, strm>>>(sp, il, g->u3, -il, g->v3, z);
        MSP_CHECK_LAUNCH(ctx);
        if (count) ++*count;
        return MSP_OK;
    }
    // Algorithm 4: t2 flexible PCG steps on the level-2 system, SolveM2 as
    // the preconditioner, then w = (r - A^T A~ y) / lam~
    msp_status solve_m1(const float* r, float* w, int t2, int t3) {
        if (t2 == 0) return solve_m1_direct(r, w);
        const int sp = (int)g->s_pad;
        Pcg* sc = g->sc + 1;
        MSP_TRY(sketch_rhs(r, g->g2));
        MSP_TRY(vec(0, sp, g->g2, nullptr, g->y2, g->r2, sc));
        MSP_TRY(solve_m2(g->r2, g->z2, t3));
        MSP_TRY(vec(1, sp, g->r2, g->z2, g->p2, g->zo2, sc));
        for (int k = 0; k < t2; ++k) {
            MSP_TRY(op2(g->p2, g->q2));
            MSP_TRY(vec(2, sp, g->p2, g->q2, g->y2, g->r2, sc));
            if (k + 1 < t2) {
                MSP_TRY(solve_m2(g->r2, g->z2, t3));
                MSP_TRY(vec(3, sp, g->r2, g->z2, g->zo2, g->p2, sc, 1));
            }
        }
        return finish_m1(g->y2, r, w);
    }
};

void destroy_general(G_t* g) {
    if (!g) return;
    if (g->m1_exec) cudaGraphExecDestroy(g->m1_exec);
    if (g->it_exec) cudaGraphExecDestroy(g->it_exec);
    cudaStream_t s = g->stream;
    for (void* p : {(void*)g->A_copy, (void*)g->At, (void*)g->M3a, (void*)g->M3b, (void*)g->G3a, (void*)g->G3b,
                    (void*)g->Linv, g->work, (void*)g->W64, (void*)g->M2inv, (void*)g->Cm, (void*)g->Binv,
                    (void*)g->zeros})
        if (p) cudaFreeAsync(p, s);
    if (g->host) cudaFreeHost(g->host);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->inner) destroy_general(g->inner);
    if (g->As) cudaFreeAsync(g->As, s);
    delete g;
}

__global__ void k_diag_add64(const double* __restrict__ W, double d, int64_t s, int64_t sp, double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sp * sp) return;
    const int64_t a = e / sp, b = e % sp;
    out[e] = W[e] + ((a == b && a < s) ? d : 0.0);
}

// out = (X - Y) / d on the leading s x s block, identity on the pad
__global__ void k_diff_scale64(const double* __restrict__ X, const double* __restrict__ Y, double inv_d, int64_t s,
                               int64_t sp, double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sp * sp) return;
    const int64_t a = e / sp, b = e % sp;
    out[e] = (a < s && b < s) ? (X[e] - Y[e]) * inv_d : (a == b ? 1.0 : 0.0);
}

// B = G + lam~ W on the leading block (G's pad is already identity)
__global__ void k_add_scaled64(double* __restrict__ G, double lt, const double* __restrict__ W, int64_t s, int64_t sp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sp * sp) return;
    const int64_t a = e / sp, b = e % sp;
    if (a < s && b < s) G[e] += lt * W[e];
}

msp_status ensure_w64(msp_ctx* ctx, G_t* g) {
    if (g->W64) return MSP_OK;
    const int64_t sp = g->s_pad;
    MSP_TRY(msp_alloc(ctx, (void**)&g->W64, (size_t)sp * sp * 8));
    return msp_gram64(ctx, g->At, g->m, sp, g->s, sp, 0.0, g->W64);
}

// level 3 exact: M2^{-1} = (W^{-1} - (W + lam~ I)^{-1}) / lam~ (Section 5)
msp_status ensure_direct3(msp_ctx* ctx, G_t* g) {
    if (g->M2inv) return MSP_OK;
    MSP_TRY(ensure_w64(ctx, g));
    const int64_t sp = g->s_pad, mat = sp * sp;
    double* tmp = nullptr;
    MSP_TRY(msp_alloc(ctx, (void**)&tmp, (size_t)mat * 3 * 8));
    double *Wi = tmp, *Wb = tmp + mat, *Wbi = tmp + 2 * mat;
    double sh = 0.0;
    int rt = 0;
    const unsigned nb = (unsigned)((mat + 255) / 256);
    msp_status st = msp_spd_inverse(ctx, g->W64, g->s, sp, g->Linv, Wi, &sh, &rt);
    if (st == MSP_OK) {
        k_diag_add64<<<nb, 256, 0, ctx->stream>>>(g->W64, g->lam_tilde, g->s, sp, Wb);
        st = cudaGetLastError() == cudaSuccess ? MSP_OK : msp_set_error(ctx, MSP_ECUDA, "general: launch failed");
        ++ctx->launches;
    }
    if (st == MSP_OK) st = msp_spd_inverse(ctx, Wb, g->s, sp, g->Linv, Wbi, &sh, &rt);
    if (st == MSP_OK) st = msp_alloc(ctx, (void**)&g->M2inv, (size_t)mat * 8);
    if (st == MSP_OK) {
        k_diff_scale64<<<nb, 256, 0, ctx->stream>>>(Wi, Wbi, 1.0 / g->lam_tilde, g->s, sp, g->M2inv);
        st = cudaGetLastError() == cudaSuccess ? MSP_OK : msp_set_error(ctx, MSP_ECUDA, "general: launch failed");
        ++ctx->launches;
    }
    cudaFreeAsync(tmp, ctx->stream);
    if (st != MSP_OK && g->M2inv) {
        cudaFreeAsync(g->M2inv, ctx->stream);
        g->M2inv = nullptr;
    }
    return st;
}

// level 2 exact: C = A^T A~ (n64 x s_pad) and (C^T C + lam~ W)^{-1}
msp_status ensure_direct2(msp_ctx* ctx, G_t* g) {
    if (g->Binv) return MSP_OK;
    MSP_TRY(ensure_w64(ctx, g));
    const int64_t sp = g->s_pad, mat = sp * sp;
    g->n64 = round_up(g->n, 64);
    if (!g->Cm) {
        MSP_TRY(msp_alloc(ctx, (void**)&g->Cm, (size_t)g->n64 * sp * 4));
        MSP_TRY(msp_gemm_tn(ctx, g->A, g->lda, g->n, g->At, sp, sp, g->m, g->n64, sp, g->Cm));
    }
    if (!g->zeros) {
        MSP_TRY(msp_alloc(ctx, (void**)&g->zeros, (size_t)sp * 4));
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->zeros, 0, (size_t)sp * 4, ctx->stream));
    }
    double* B = nullptr;
    MSP_TRY(msp_alloc(ctx, (void**)&B, (size_t)mat * 8));
    double sh = 0.0;
    int rt = 0;
    msp_status st = msp_gram64(ctx, g->Cm, g->n64, sp, g->s, sp, 0.0, B);
    if (st == MSP_OK) {
        k_add_scaled64<<<(unsigned)((mat + 255) / 256), 256, 0, ctx->stream>>>(B, g->lam_tilde, g->W64, g->s, sp);
        st = cudaGetLastError() == cudaSuccess ? MSP_OK : msp_set_error(ctx, MSP_ECUDA, "general: launch failed");
        ++ctx->launches;
    }
    if (st == MSP_OK) st = msp_alloc(ctx, (void**)&g->Binv, (size_t)mat * 8);
    if (st == MSP_OK) st = msp_spd_inverse(ctx, B, g->s, sp, g->Linv, g->Binv, &sh, &rt);
    cudaFreeAsync(B, ctx->stream);
    if (st != MSP_OK && g->Binv) {
        cudaFreeAsync(g->Binv, ctx->stream);
        g->Binv = nullptr;
    }
    return st;
}

msp_status ensure_direct(msp_ctx* ctx, G_t* g, int t2, int t3) {
    if (t2 == 0) return ensure_direct2(ctx, g);
    if (t3 == 0) return ensure_direct3(ctx, g);
    return ensure_w64(ctx, g);
}

// SolveM1 for the handle's (t2, t3) as a CUDA graph, rebuilt when they change
msp_status ensure_m1_graph(msp_ctx* ctx, G_t* g, int t2, int t3) {
    if (g->m1_exec && g->m1_t2 == t2 && g->m1_t3 == t3) return MSP_OK;
    if (g->m1_exec) {
        cudaGraphExecDestroy(g->m1_exec);
        g->m1_exec = nullptr;
    }
    int count = 0;
    Ops ops{ctx, g, &count, g->cap};
    MSP_CUDA_TRY(ctx, cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = ctx->launches;
    msp_status st = ops.solve_m1(g->r1, g->z1, t2, t3);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
    ctx->launches = l0;   // counted per replay instead
    if (st != MSP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph) {
        cudaGetLastError();
        return msp_set_error(ctx, MSP_ECUDA, "general: SolveM1 capture failed: %s", cudaGetErrorString(ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&g->m1_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        g->m1_exec = nullptr;
        return msp_set_error(ctx, MSP_ECUDA, "general: graph instantiation failed");
    }
    g->m1_t2 = t2;
    g->m1_t3 = t3;
    g->m1_kernels = count;
    return MSP_OK;
}

msp_status run_m1(msp_ctx* ctx, G_t* g, int t2, int t3) {
    MSP_TRY(ensure_direct(ctx, g, t2, t3));
    MSP_TRY(ensure_m1_graph(ctx, g, t2, t3));
    MSP_CUDA_TRY(ctx, cudaGraphLaunch(g->m1_exec, ctx->stream));
    ctx->launches += g->m1_kernels;
    return MSP_OK;
}

// One level-1 iteration (q = (A^T A + lam I) p, the step, z = SolveM1(r),
// the new direction) as a CUDA graph for the handle's (t2, t3); the lambda
// values are baked in, so msp_general_set_lambda drops it.
msp_status ensure_iter_graph(msp_ctx* ctx, G_t* g, int t2, int t3) {
    if (g->it_exec && g->it_t2 == t2 && g->it_t3 == t3) return MSP_OK;
    if (g->it_exec) {
        cudaGraphExecDestroy(g->it_exec);
        g->it_exec = nullptr;
    }
    MSP_TRY(ensure_direct(ctx, g, t2, t3));
    int count = 0;
    Ops ops{ctx, g, &count, g->cap};
    const int len = (int)g->n_pad;
    MSP_CUDA_TRY(ctx, cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = ctx->launches;
    msp_status st = ops.op1(g->p1, g->q1);
    if (st == MSP_OK) st = ops.vec(2, len, g->p1, g->q1, g->x1, g->r1, g->sc);
    if (st == MSP_OK) st = ops.solve_m1(g->r1, g->z1, t2, t3);
    if (st == MSP_OK) st = ops.vec(3, len, g->r1, g->z1, g->zo1, g->p1, g->sc, 1);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
    ctx->launches = l0;
    if (st != MSP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph) {
        cudaGetLastError();
        return msp_set_error(ctx, MSP_ECUDA, "general: iteration capture failed: %s", cudaGetErrorString(ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&g->it_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        g->it_exec = nullptr;
        return msp_set_error(ctx, MSP_ECUDA, "general: graph instantiation failed");
    }
    g->it_t2 = t2;
    g->it_t3 = t3;
    g->it_kernels = count;
    return MSP_OK;
}

msp_status read_scalars(msp_ctx* ctx, G_t* g, const Pcg* sc, double* rr, double* bb) {
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->host, sc, sizeof(Pcg), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->host + 8, g->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const Pcg* h = reinterpret_cast<const Pcg*>(g->host);
    *rr = h->rr;
    *bb = h->bb;
    int e = 0;
    std::memcpy(&e, g->host + 8, sizeof(int));
    if (e != 0) return msp_set_error(ctx, (msp_status)e, "general: breakdown in an inner iteration (status %d)", e);
    return MSP_OK;
}

// Level 1 (Algorithm 3 step 7): flexible PCG on (A^T A + lam I) x1 = b1 with
// SolveM1, FP32 vectors; stops at |r| <= tol |b1| or after maxit steps.
msp_status level1(msp_ctx* ctx, G_t* g, double tol, int maxit, int t2, int t3, int* iters, bool* conv,
                  int* inner);

// z1 = M^{-1} r1: SolveM1 (the graph), or for a least-squares handle one
// solve with the inner handle on A~ to relative residual inner_tol (constant
// accuracy; the level-1 iteration is flexible)
msp_status precond(msp_ctx* ctx, G_t* g, int t2, int t3, int* inner) {
    if (!g->inner) {
        MSP_TRY(run_m1(ctx, g, t2, t3));
        *inner += t2;
        return MSP_OK;
    }
    G_t* h = g->inner;
    h->check_every = 1;     // constant-accuracy inner solves stop at the first chance
    const size_t bytes = (size_t)g->n_pad * 4;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(h->b1, g->r1, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    int it = 0, in2 = 0;
    bool conv = false;
    MSP_TRY(level1(ctx, h, g->inner_tol, g->inner_maxit, t2, t3, &it, &conv, &in2));
    *inner += it;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->z1, h->x1, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

msp_status level1(msp_ctx* ctx, G_t* g, double tol, int maxit, int t2, int t3, int* iters, bool* conv,
                  int* inner) {
    Ops ops{ctx, g, nullptr, ctx->stream};
    const int len = (int)g->n_pad;
    Pcg* sc = g->sc;
    MSP_TRY(ops.vec(0, len, g->b1, nullptr, g->x1, g->r1, sc));
    double rr = 0, bb = 0;
    MSP_TRY(read_scalars(ctx, g, sc, &rr, &bb));
    *iters = 0;
    *conv = false;
    if (bb == 0.0) {
        *conv = true;
        return MSP_OK;
    }
    g->host[13] = tol * tol * bb;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(&sc->tol2, g->host + 13, 8, cudaMemcpyHostToDevice, ctx->stream));
    MSP_TRY(precond(ctx, g, t2, t3, inner));
    MSP_TRY(ops.vec(1, len, g->r1, g->z1, g->p1, g->zo1, sc));
    if (!g->inner) {
        // whole iterations replayed as one graph, the host check every
        // `check` iterations (a converged PCG only keeps improving)
        MSP_TRY(ensure_iter_graph(ctx, g, t2, t3));
        const int check = std::max(1, g->check_every);
        // replay as many iterations as the observed rate says are still
        // needed (at most `check`), so the check rarely overshoots
        int k = 0, nrun = 1;
        double rr_prev = bb;
        while (k < maxit) {
            nrun = std::max(1, std::min(nrun, maxit - k));
            for (int i = 0; i < nrun; ++i) MSP_CUDA_TRY(ctx, cudaGraphLaunch(g->it_exec, ctx->stream));
            ctx->launches += (int64_t)nrun * g->it_kernels;
            k += nrun;
            *inner += nrun * t2;
            MSP_TRY(read_scalars(ctx, g, sc, &rr, &bb));
            *iters = k;
            if (!std::isfinite(rr)) return msp_set_error(ctx, MSP_ENONFINITE, "general: non-finite residual");
            if (rr <= tol * tol * bb) {
                *conv = true;
                return MSP_OK;
            }
            if (rr > 1e8 * bb) return MSP_OK;
            const double rate = std::pow(rr / rr_prev, 1.0 / nrun);
            const double need = (rate > 0.0 && rate < 1.0) ? std::log(tol * tol * bb / rr) / std::log(rate) : 1.0;
            nrun = (int)std::min<double>(check, std::max(1.0, std::floor(need)));
            rr_prev = rr;
        }
        return MSP_OK;
    }
    for (int k = 1; k <= maxit; ++k) {
        MSP_TRY(ops.op1(g->p1, g->q1));
        MSP_TRY(ops.vec(2, len, g->p1, g->q1, g->x1, g->r1, sc));
        MSP_TRY(read_scalars(ctx, g, sc, &rr, &bb));
        *iters = k;
        if (!std::isfinite(rr)) return msp_set_error(ctx, MSP_ENONFINITE, "general: non-finite residual");
        if (rr <= tol * tol * bb) {
            *conv = true;
            return MSP_OK;
        }
        // a residual 1e4 times the right-hand side: the (inexact) preconditioner
        // has broken the iteration; stop instead of running to the cap
        if (rr > 1e8 * bb) return MSP_OK;
        if (k == maxit) break;
        MSP_TRY(precond(ctx, g, t2, t3, inner));
        MSP_TRY(ops.vec(3, len, g->r1, g->z1, g->zo1, g->p1, sc, 1));
    }
    return MSP_OK;
}

// out = sgn (A^T A + lam I) x64 + v, FP64 accumulation
msp_status apply64(msp_ctx* ctx, G_t* g, double sgn, const double* v, double* out) {
    const int na4 = (int)(g->n_pad / 4);
    int used = 0;
    MSP_TRY(launch_same<double>(ctx, ctx->stream, g->G, g->m, g->A, g->lda, na4, g->x64, nullptr, 0.0, nullptr,
                                g->part64, g->n_pad, g->err, nullptr, &used));
    return colsum<double>(ctx, ctx->stream, g, g->part64, g->n_pad, (int)g->n_pad, sgn, g->x64, sgn * g->lambda, v,
                          out, nullptr, used);
}

// r64 = c64 - (A^T A + lam I) x64
msp_status residual64(msp_ctx* ctx, G_t* g) { return apply64(ctx, g, -1.0, g->c64, g->r64); }

msp_status norm64(msp_ctx* ctx, G_t* g, const double* v, double* out) {
    k_norm2_64<<<1, kVecThreads, 0, ctx->stream>>>((int)g->n_pad, v, g->d64);
    MSP_CHECK_LAUNCH(ctx);
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->host + 10, g->d64, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->host + 11, g->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *out = std::sqrt(g->host[10]);
    int e = 0;
    std::memcpy(&e, g->host + 11, sizeof(int));
    if (e != 0) return msp_set_error(ctx, (msp_status)e, "general: device error %d (a bounded wait timed out)", e);
    return MSP_OK;
}

// The level-1 solve of (A^T A + lam I) x64 = c64 (|c64| = cn > 0): FP32
// alone (MSP_PREC_FP32), or wrapped in FP64 refinement (MSP_PREC_MIXED);
// result MSP_ENOCONV when the tolerance was not reached.
msp_status solve_refined(msp_ctx* ctx, G_t* g, const msp_opts& o, double cn, msp_info* inf_out,
                         msp_status* result_out) {
    const int t2 = o.level2_iters, t3 = o.level3_iters;
    const int np = (int)g->n_pad;
    const unsigned nb = (unsigned)((np + 255) / 256);
    g->check_every = std::max(1, std::min(o.check_every, 64));
    msp_status& result = *result_out;
    msp_info& inf = *inf_out;
    result = MSP_OK;
    if (o.precision == MSP_PREC_FP32) {
        k_scale_to_f32<<<nb, 256, 0, ctx->stream>>>(np, g->c64, 1.0 / cn, g->b1);
        MSP_CHECK_LAUNCH(ctx);
        int it = 0;
        bool conv = false;
        MSP_TRY(level1(ctx, g, o.tol, o.max_outer, t2, t3, &it, &conv, &inf.inner_iters));
        inf.outer_iters = it;
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->x64, 0, (size_t)np * 8, ctx->stream));
        k_axpy_64<<<nb, 256, 0, ctx->stream>>>(np, cn, g->x1, g->x64);
        MSP_CHECK_LAUNCH(ctx);
        MSP_TRY(residual64(ctx, g));
        double rn = 0.0;
        MSP_TRY(norm64(ctx, g, g->r64, &rn));
        inf.rel_resid = rn / cn;
        if (!conv) result = MSP_ENOCONV;
    } else {
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->x64, 0, (size_t)np * 8, ctx->stream));
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->r64, g->c64, (size_t)np * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        double rn = cn;
        bool done = false;
        for (int step = 0; step < o.max_refine; ++step) {
            if (rn <= o.tol * cn) {
                done = true;
                break;
            }
            k_scale_to_f32<<<nb, 256, 0, ctx->stream>>>(np, g->r64, 1.0 / rn, g->b1);
            MSP_CHECK_LAUNCH(ctx);
            int it = 0;
            bool conv = false;
            MSP_TRY(level1(ctx, g, o.refine_tol, o.max_outer, t2, t3, &it, &conv, &inf.inner_iters));
            inf.outer_iters += it;
            ++inf.refine_steps;
            k_axpy_64<<<nb, 256, 0, ctx->stream>>>(np, rn, g->x1, g->x64);
            MSP_CHECK_LAUNCH(ctx);
            MSP_TRY(residual64(ctx, g));
            const double prev = rn;
            MSP_TRY(norm64(ctx, g, g->r64, &rn));
            if (!std::isfinite(rn)) return msp_set_error(ctx, MSP_ENONFINITE, "general: non-finite residual");
            if (rn >= prev && !(rn <= o.tol * cn)) break;   // refinement stalled
        }
        if (!done && rn <= o.tol * cn) done = true;
        inf.rel_resid = rn / cn;
        if (!done) result = MSP_ENOCONV;
    }
    return MSP_OK;
}

msp_status check_vec_args(msp_ctx* ctx, const void* p) {
    if (!p) return msp_set_error(ctx, MSP_EINVAL, "general: NULL vector");
    return MSP_OK;
}

}  // namespace

namespace {

// Everything but the sketch: A (or its aligned copy), the row partition, the
// work vectors for level-1 vectors of n_pad and inner vectors of s_pad
// (0: none), the capture stream. On failure nothing is left allocated.
msp_status create_base(msp_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, double lambda,
                       double lambda0, int64_t s_pad, G_t** out) {
    G_t* g = new (std::nothrow) G_t();
    if (!g) return msp_set_error(ctx, MSP_ENOMEM, "general: host allocation failed");
    g->stream = ctx->stream;
    g->device = ctx->device;
    g->m = m;
    g->n = n;
    g->n_pad = round_up(n, 4);
    g->s_pad = s_pad;
    g->lambda = lambda;
    g->lambda0 = lambda0;
    g->lam_tilde = lambda + lambda0;
    auto fail = [&](msp_status st) {
        cudaStreamSynchronize(ctx->stream);
        destroy_general(g);
        return st;
    };
    if (cudaMallocHost((void**)&g->host, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        g->host = nullptr;
        return fail(msp_set_error(ctx, MSP_ENOMEM, "general: pinned allocation failed"));
    }
    const int64_t np = g->n_pad, sp = g->s_pad;
    // rows must start on 16-byte boundaries for the float4 row passes
    const bool aligned = (lda % 4 == 0) && (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    msp_status st = MSP_OK;
    (void)st;
    if (aligned) {
        g->A = A;
        g->lda = lda;
    } else {
        if ((st = msp_alloc(ctx, (void**)&g->A_copy, (size_t)m * np * 4)) != MSP_OK) return fail(st);
        if (np != n && cudaMemsetAsync(g->A_copy, 0, (size_t)m * np * 4, ctx->stream) != cudaSuccess)
            return fail(msp_set_error(ctx, MSP_ECUDA, "general: memset failed"));
        if (cudaMemcpy2DAsync(g->A_copy, np * 4, A, lda * 4, n * 4, m, cudaMemcpyDeviceToDevice, ctx->stream) !=
            cudaSuccess) {
            cudaGetLastError();
            return fail(msp_set_error(ctx, MSP_ECUDA, "general: copy of A failed"));
        }
        g->A = g->A_copy;
        g->lda = np;
    }
    // rows per CTA step: 2 CTAs per SM
    g->G = (int)std::min<int64_t>(2 * ctx->num_sms, (m + kRows - 1) / kRows);
    g->rows_per_cta = round_up((m + g->G - 1) / g->G, kRows);
    g->G = (int)((m + g->rows_per_cta - 1) / g->rows_per_cta);
    g->ldp = std::max<int64_t>(g->n_pad, g->s_pad);
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g->cap = nullptr;
        return fail(msp_set_error(ctx, MSP_ECUDA, "general: stream creation failed"));
    }

    // ---- work vectors
    {
        size_t off = 0;
        auto take = [&](size_t b) { const size_t o = off; off += (size_t)round_up((int64_t)b, 256); return o; };
        size_t o1[7], o2[7], o3[2];
        for (auto& o : o1) o = take((size_t)np * 4);
        for (auto& o : o2) o = take((size_t)sp * 4);
        for (auto& o : o3) o = take((size_t)sp * 4);
        const size_t o_tm = take((size_t)m * 4), o_vn = take((size_t)np * 4);
        const size_t o_part = take((size_t)g->G * g->ldp * 4);
        const size_t o_p64 = take((size_t)g->G * np * 8);
        const size_t o_x64 = take((size_t)np * 8), o_r64 = take((size_t)np * 8), o_c64 = take((size_t)np * 8);
        const size_t o_d64 = take(64);
        const size_t o_sc = take(sizeof(Pcg) * 3), o_err = take(16);
        if ((st = msp_alloc(ctx, &g->work, off)) != MSP_OK) return fail(st);
        if (cudaMemsetAsync(g->work, 0, off, ctx->stream) != cudaSuccess)
            return fail(msp_set_error(ctx, MSP_ECUDA, "general: memset failed"));
        char* w = (char*)g->work;
        float** v1[7] = {&g->x1, &g->r1, &g->z1, &g->zo1, &g->p1, &g->q1, &g->b1};
        float** v2[7] = {&g->g2, &g->y2, &g->r2, &g->z2, &g->zo2, &g->p2, &g->q2};
        for (int q = 0; q < 7; ++q) {
            *v1[q] = (float*)(w + o1[q]);
            *v2[q] = (float*)(w + o2[q]);
        }
        g->u3 = (float*)(w + o3[0]);
        g->v3 = (float*)(w + o3[1]);
        g->tm = (float*)(w + o_tm);
        g->vn = (float*)(w + o_vn);
        g->part = (float*)(w + o_part);
        g->part64 = (double*)(w + o_p64);
        g->x64 = (double*)(w + o_x64);
        g->r64 = (double*)(w + o_r64);
        g->c64 = (double*)(w + o_c64);
        g->d64 = (double*)(w + o_d64);
        g->sc = (Pcg*)(w + o_sc);
        g->err = (int*)(w + o_err);
    }
    if ((st = set_ring_attrs<float>(ctx)) != MSP_OK || (st = set_ring_attrs<double>(ctx)) != MSP_OK ||
        (st = set_rowpass_attrs<float>(ctx, (size_t)std::max(np, sp) * 4)) != MSP_OK ||
        (st = set_rowpass_attrs<double>(ctx, (size_t)np * 8)) != MSP_OK)
        return fail(st);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(msp_set_error(ctx, MSP_ECUDA, "general: set-up failed"));
    }
    *out = g;
    return MSP_OK;
}


// Algorithm 3 steps 3-6 on a base handle: S, A~ = A S^T, A^ = Phi A~,
// M3a = A^^T A^, M3b = M3a + lam~ I and their FP64 inverses.
msp_status setup_sketch(msp_ctx* ctx, G_t* g) {
    const int64_t m = g->m, n = g->n, s = g->s, sp = g->s_pad, phi = g->phi;
    const int gamma = g->gamma, gamma_phi = g->gamma_phi;
    const uint64_t seed = g->seed;
    msp_status st = MSP_OK;
    auto fail = [&](msp_status e) { return e; };
    // ---- Algorithm 3 steps 3-4: S, A~ = A S^T, A^ = Phi A~
    {
        int32_t *idx = nullptr, *ptr = nullptr, *ent = nullptr, *pptr = nullptr, *pent = nullptr;
        int8_t *sgn = nullptr;
        float* Ah = nullptr;
        void* tmp = nullptr;
        const size_t b_idx = (size_t)std::max<int64_t>(n * gamma, m * gamma_phi) * 4;
        const size_t b_sgn = (size_t)std::max<int64_t>(n * gamma, m * gamma_phi);
        const size_t b_ptr = (size_t)(std::max<int64_t>(sp, phi) + 1) * 4;
        size_t off = 0;
        auto take = [&](size_t b) { const size_t o = off; off += (size_t)round_up((int64_t)b, 256); return o; };
        const size_t o_idx = take(b_idx), o_sgn = take(b_sgn), o_ptr = take(b_ptr), o_ent = take(b_idx);
        const size_t o_ah = take((size_t)phi * sp * 4);
        if ((st = msp_alloc(ctx, &tmp, off)) != MSP_OK) return fail(st);
        char* tb = (char*)tmp;
        idx = (int32_t*)(tb + o_idx);
        sgn = (int8_t*)(tb + o_sgn);
        ptr = (int32_t*)(tb + o_ptr);
        ent = (int32_t*)(tb + o_ent);
        pptr = ptr;
        pent = ent;
        Ah = (float*)(tb + o_ah);
        auto tfail = [&](msp_status e) {
            cudaStreamSynchronize(ctx->stream);
            cudaFreeAsync(tmp, ctx->stream);
            return fail(e);
        };
        if ((st = msp_alloc(ctx, (void**)&g->At, (size_t)m * sp * 4)) != MSP_OK) return tfail(st);
        if ((st = msp_pattern_launch(ctx, n, s, gamma, seed, 0, idx, sgn, nullptr)) != MSP_OK ||
            (st = msp_build_csr(ctx, n, sp, gamma, idx, sgn, ptr, ent)) != MSP_OK ||
            (st = msp_sketch_apply_rows(ctx, g->A, MSP_F32, m, n, g->lda, sp, ptr, ent, gamma, g->At)) != MSP_OK)
            return tfail(st);
        // Phi (phi x m) on the level-2 streams; its rows gather rows of A~
        if ((st = msp_pattern_launch(ctx, m, phi, gamma_phi, seed, 2, idx, sgn, nullptr)) != MSP_OK ||
            (st = msp_build_csr(ctx, m, phi, gamma_phi, idx, sgn, pptr, pent)) != MSP_OK ||
            (st = msp_gather_rows(ctx, MSP_F32, phi, sp, pptr, pent, g->At, sp, 1.0 / std::sqrt((double)gamma_phi),
                                  Ah, sp)) != MSP_OK)
            return tfail(st);
        // ---- steps 5-6: M3a = A^^T A^, M3b = M3a + lam~ I and their inverses
        const size_t mat = (size_t)sp * sp;
        if ((st = msp_alloc(ctx, (void**)&g->M3a, mat * 8)) != MSP_OK ||
            (st = msp_alloc(ctx, (void**)&g->M3b, mat * 8)) != MSP_OK ||
            (st = msp_alloc(ctx, (void**)&g->G3a, mat * 8)) != MSP_OK ||
            (st = msp_alloc(ctx, (void**)&g->G3b, mat * 8)) != MSP_OK ||
            (st = msp_alloc(ctx, (void**)&g->Linv, mat * 8)) != MSP_OK)
            return tfail(st);
        if ((st = msp_gram_inverse(ctx, Ah, phi, s, sp, 0.0, g->G3a, g->Linv, g->M3a, &g->shift_a,
                                   &g->retries_a)) != MSP_OK ||
            (st = msp_gram_inverse(ctx, Ah, phi, s, sp, g->lam_tilde, g->G3b, g->Linv, g->M3b, &g->shift_b,
                                   &g->retries_b)) != MSP_OK)
            return tfail(st);
        cudaFreeAsync(tmp, ctx->stream);
    }
    return MSP_OK;
}

}  // namespace

extern "C" {

msp_status msp_general_create(msp_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, double lambda,
                              double lambda0, int64_t s, int gamma, int64_t phi, int gamma_phi, uint64_t seed,
                              msp_general_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !out) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    *out = nullptr;
    if (n < 16 || n > kMaxN || m < n || m >= (1ll << 30) || lda < n || !(lambda >= 0.0) || !(lambda0 >= 0.0) ||
        !(lambda + lambda0 > 0.0) || s < 16 || s > MSP_MAX_S || s > n || gamma < 1 || gamma > MSP_MAX_GAMMA ||
        gamma > s || phi < s || phi > m || gamma_phi < 1 || gamma_phi > MSP_MAX_GAMMA || gamma_phi > phi)
        return msp_set_error(ctx, MSP_EINVAL,
                             "general: need 16 <= n <= %d, n <= m < 2^30, lda >= n, lambda, lambda0 >= 0 with "
                             "lambda + lambda0 > 0, 16 <= s <= min(n, %d), 1 <= gamma <= min(s, %d), "
                             "s <= phi <= m, 1 <= gamma_phi <= min(phi, %d)",
                             kMaxN, MSP_MAX_S, MSP_MAX_GAMMA, MSP_MAX_GAMMA);
    msp::DeviceGuard guard(ctx->device);
    G_t* g = nullptr;
    MSP_TRY(create_base(ctx, A, m, n, lda, lambda, lambda0, round_up(s, MSP_S_ALIGN), &g));
    g->s = s;
    g->phi = phi;
    g->gamma = gamma;
    g->gamma_phi = gamma_phi;
    g->seed = seed;
    msp_status st = setup_sketch(ctx, g);
    if (st == MSP_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        st = msp_set_error(ctx, MSP_ECUDA, "general: set-up failed");
    }
    if (st != MSP_OK) {
        cudaStreamSynchronize(ctx->stream);
        destroy_general(g);
        return st;
    }
    *out = g;
    return MSP_OK;
}

void msp_general_destroy(msp_general_t* g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    destroy_general(g);
    cudaSetDevice(prev);
}

msp_status msp_general_info(const msp_general_t* g, int64_t* s_pad, double* lambda_tilde, double* shift_a,
                            double* shift_b) {
    if (!g) return msp_set_error(nullptr, MSP_EINVAL, "general: handle is NULL");
    if (s_pad) *s_pad = g->s_pad;
    if (lambda_tilde) *lambda_tilde = g->lam_tilde;
    if (shift_a) *shift_a = g->shift_a;
    if (shift_b) *shift_b = g->shift_b;
    return MSP_OK;
}

msp_status msp_general_get(msp_ctx* ctx, const msp_general_t* g, float* At, int64_t ld_at, double* M3a,
                           double* M3b) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    msp::DeviceGuard guard(ctx->device);
    const int64_t sp = g->s_pad;
    if (At) {
        if (ld_at < g->s) return msp_set_error(ctx, MSP_EINVAL, "general_get: ld_at < s");
        MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(At, ld_at * 4, g->At, sp * 4, g->s * 4, g->m, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
    }
    if (M3a)
        MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(M3a, g->s * 8, g->G3a, sp * 8, g->s * 8, g->s, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
    if (M3b)
        MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(M3b, g->s * 8, g->G3b, sp * 8, g->s * 8, g->s, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
    return MSP_OK;
}

msp_status msp_general_solve_m2(msp_ctx* ctx, msp_general_t* g, const float* r, float* z, int t3) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    MSP_TRY(check_vec_args(ctx, r));
    MSP_TRY(check_vec_args(ctx, z));
    if (t3 < 0 || t3 > 1000) return msp_set_error(ctx, MSP_EINVAL, "general: need 0 <= t3 <= 1000");
    msp::DeviceGuard guard(ctx->device);
    MSP_TRY(t3 == 0 ? ensure_direct3(ctx, g) : ensure_w64(ctx, g));
    const int sp = (int)g->s_pad;
    k_pad_copy_32<<<(unsigned)((sp + 255) / 256), 256, 0, ctx->stream>>>(sp, (int)g->s, r, g->r2);
    MSP_CHECK_LAUNCH(ctx);
    Ops ops{ctx, g, nullptr, ctx->stream};
    MSP_TRY(ops.solve_m2(g->r2, g->z2, t3));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(z, g->z2, (size_t)g->s * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

msp_status msp_general_solve_m1(msp_ctx* ctx, msp_general_t* g, const float* r, float* w, int t2, int t3) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    MSP_TRY(check_vec_args(ctx, r));
    MSP_TRY(check_vec_args(ctx, w));
    if (t2 < 0 || t2 > 1000 || t3 < 0 || t3 > 1000)
        return msp_set_error(ctx, MSP_EINVAL, "general: need 0 <= t2, t3 <= 1000");
    msp::DeviceGuard guard(ctx->device);
    const int np = (int)g->n_pad;
    k_pad_copy_32<<<(unsigned)((np + 255) / 256), 256, 0, ctx->stream>>>(np, (int)g->n, r, g->r1);
    MSP_CHECK_LAUNCH(ctx);
    MSP_TRY(run_m1(ctx, g, t2, t3));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(w, g->z1, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

msp_status msp_general_op(msp_ctx* ctx, msp_general_t* g, const float* p, float* q) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    MSP_TRY(check_vec_args(ctx, p));
    MSP_TRY(check_vec_args(ctx, q));
    msp::DeviceGuard guard(ctx->device);
    const int np = (int)g->n_pad;
    if (p != g->p1) {
        k_pad_copy_32<<<(unsigned)((np + 255) / 256), 256, 0, ctx->stream>>>(np, (int)g->n, p, g->p1);
        MSP_CHECK_LAUNCH(ctx);
    }
    Ops ops{ctx, g, nullptr, ctx->stream};
    MSP_TRY(ops.op1(g->p1, g->q1));
    if (q != g->q1)
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(q, g->q1, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

msp_status msp_general_matvec64(msp_ctx* ctx, msp_general_t* g, const double* x, double* y) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    MSP_TRY(check_vec_args(ctx, x));
    MSP_TRY(check_vec_args(ctx, y));
    msp::DeviceGuard guard(ctx->device);
    const int np = (int)g->n_pad;
    k_pad_copy_64<<<(unsigned)((np + 255) / 256), 256, 0, ctx->stream>>>(np, (int)g->n, x, g->x64);
    MSP_CHECK_LAUNCH(ctx);
    MSP_TRY(apply64(ctx, g, 1.0, nullptr, g->r64));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(y, g->r64, (size_t)g->n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

msp_status msp_general_solve(msp_ctx* ctx, msp_general_t* g, const double* c, double* x, const msp_opts* opts,
                             msp_info* info) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    MSP_TRY(check_vec_args(ctx, c));
    MSP_TRY(check_vec_args(ctx, x));
    msp_opts o;
    if (opts) o = *opts;
    else msp_default_opts(&o);
    if (!(o.tol > 0.0) || o.max_outer < 1 || o.level2_iters < 0 || o.level2_iters > 1000 || o.level3_iters < 0 ||
        o.level3_iters > 1000 || (o.precision != MSP_PREC_MIXED && o.precision != MSP_PREC_FP32) ||
        o.criterion != MSP_STOP_RESIDUAL || (o.precision == MSP_PREC_MIXED && !(o.refine_tol > 0.0)))
        return msp_set_error(ctx, MSP_EINVAL,
                             "general: need tol > 0, max_outer >= 1, 0 <= level2_iters, level3_iters <= 1000, "
                             "precision MIXED or FP32, the residual criterion");
    msp::DeviceGuard guard(ctx->device);
    msp_info inf;
    std::memset(&inf, 0, sizeof inf);
    inf.lambda_tilde = g->lam_tilde;
    inf.shift = g->shift_a;
    inf.shift_retries = g->retries_a + g->retries_b;
    const int np = (int)g->n_pad;
    const unsigned nb = (unsigned)((np + 255) / 256);
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->err, 0, sizeof(int), ctx->stream));
    k_pad_copy_64<<<nb, 256, 0, ctx->stream>>>(np, (int)g->n, c, g->c64);
    MSP_CHECK_LAUNCH(ctx);
    double cn = 0.0;
    MSP_TRY(norm64(ctx, g, g->c64, &cn));
    msp_status result = MSP_OK;
    if (cn == 0.0) MSP_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, (size_t)g->n * 8, ctx->stream));
    else MSP_TRY(solve_refined(ctx, g, o, cn, &inf, &result));
    if (cn != 0.0)
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(x, g->x64, (size_t)g->n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    inf.status = result;
    if (info) *info = inf;
    if (result == MSP_ENOCONV)
        return msp_set_error(ctx, MSP_ENOCONV, "general: relative residual %.3g above tol %.3g", inf.rel_resid,
                             o.tol);
    return result;
}

msp_status msp_general_set_lambda(msp_ctx* ctx, msp_general_t* g, double lambda, double lambda0) {
    if (!ctx || !g) return msp_set_error(ctx, MSP_EINVAL, "general: NULL argument");
    if (g->inner || g->s_pad == 0 || !(lambda >= 0.0) || !(lambda0 >= 0.0) || !(lambda + lambda0 > 0.0))
        return msp_set_error(ctx, MSP_EINVAL,
                             "general_set_lambda: need a general handle, lambda, lambda0 >= 0, lambda + lambda0 > 0");
    msp::DeviceGuard guard(ctx->device);
    if (lambda != g->lambda && g->it_exec) {
        // the captured level-1 iteration has lambda in its operator
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        cudaGraphExecDestroy(g->it_exec);
        g->it_exec = nullptr;
        g->it_t2 = g->it_t3 = -1;
    }
    g->lambda = lambda;
    g->lambda0 = lambda0;
    const double lt = lambda + lambda0;
    if (lt == g->lam_tilde) return MSP_OK;
    g->lam_tilde = lt;
    // lam~-dependent state: M3b (level 3), the exact-level inverses (rebuilt
    // when next used) and the captured SolveM1 (its kernels take lam~)
    const int64_t sp = g->s_pad, mat = sp * sp;
    k_diag_add64<<<(unsigned)((mat + 255) / 256), 256, 0, ctx->stream>>>(g->G3a, lt, g->s, sp, g->G3b);
    MSP_CHECK_LAUNCH(ctx);
    MSP_TRY(msp_spd_inverse(ctx, g->G3b, g->s, sp, g->Linv, g->M3b, &g->shift_b, &g->retries_b));
    if (g->M2inv) {
        cudaFreeAsync(g->M2inv, ctx->stream);
        g->M2inv = nullptr;
    }
    if (g->Binv) {
        cudaFreeAsync(g->Binv, ctx->stream);
        g->Binv = nullptr;
    }
    if (g->m1_exec || g->it_exec) {
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        if (g->m1_exec) cudaGraphExecDestroy(g->m1_exec);
        if (g->it_exec) cudaGraphExecDestroy(g->it_exec);
        g->m1_exec = g->it_exec = nullptr;
        g->m1_t2 = g->m1_t3 = g->it_t2 = g->it_t3 = -1;
    }
    return MSP_OK;
}

// ------------------------------------------------------- least squares

msp_status msp_lsq_create(msp_ctx* ctx, const float* A, int64_t n_rows, int64_t d, int64_t lda, int64_t s_ls,
                          int gamma_ls, double lambda0, int64_t s, int gamma, int64_t phi, int gamma_phi,
                          uint64_t seed, msp_lsq_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !out) return msp_set_error(ctx, MSP_EINVAL, "lsq: NULL argument");
    *out = nullptr;
    if (d < 16 || d > kMaxN || s_ls < d || n_rows < s_ls || n_rows >= (1ll << 30) || lda < d || gamma_ls < 1 ||
        gamma_ls > MSP_MAX_GAMMA || gamma_ls > s_ls || !(lambda0 > 0.0))
        return msp_set_error(ctx, MSP_EINVAL,
                             "lsq: need 16 <= d <= %d, d <= s_ls <= n_rows < 2^30, lda >= d, "
                             "1 <= gamma_ls <= min(s_ls, %d), lambda0 > 0",
                             kMaxN, MSP_MAX_GAMMA);
    msp::DeviceGuard guard(ctx->device);
    G_t* g = nullptr;
    MSP_TRY(create_base(ctx, A, n_rows, d, lda, 0.0, 0.0, 0, &g));
    auto fail = [&](msp_status st) {
        cudaStreamSynchronize(ctx->stream);
        destroy_general(g);
        return st;
    };
    const int64_t np = g->n_pad;
    msp_status st = MSP_OK;
    if ((st = msp_alloc(ctx, (void**)&g->As, (size_t)s_ls * np * 4)) != MSP_OK) return fail(st);
    if (cudaMemsetAsync(g->As, 0, (size_t)s_ls * np * 4, ctx->stream) != cudaSuccess)
        return fail(msp_set_error(ctx, MSP_ECUDA, "lsq: memset failed"));
    // A~ = Phi A: Phi a sparse embedding of the n_rows rows (streams 4, 5)
    {
        void* tmp = nullptr;
        size_t off = 0;
        auto take = [&](size_t b) { const size_t o = off; off += (size_t)round_up((int64_t)b, 256); return o; };
        const size_t o_idx = take((size_t)n_rows * gamma_ls * 4), o_sgn = take((size_t)n_rows * gamma_ls);
        const size_t o_ptr = take((size_t)(s_ls + 1) * 4), o_ent = take((size_t)n_rows * gamma_ls * 4);
        if ((st = msp_alloc(ctx, &tmp, off)) != MSP_OK) return fail(st);
        char* tb = (char*)tmp;
        int32_t* idx = (int32_t*)(tb + o_idx);
        int8_t* sgn = (int8_t*)(tb + o_sgn);
        int32_t* ptr = (int32_t*)(tb + o_ptr);
        int32_t* ent = (int32_t*)(tb + o_ent);
        if ((st = msp_pattern_launch(ctx, n_rows, s_ls, gamma_ls, seed, 4, idx, sgn, nullptr)) != MSP_OK ||
            (st = msp_build_csr(ctx, n_rows, s_ls, gamma_ls, idx, sgn, ptr, ent)) != MSP_OK ||
            (st = msp_gather_rows(ctx, MSP_F32, s_ls, d, ptr, ent, g->A, g->lda, 1.0 / std::sqrt((double)gamma_ls),
                                  g->As, np)) != MSP_OK) {
            cudaStreamSynchronize(ctx->stream);
            cudaFreeAsync(tmp, ctx->stream);
            return fail(st);
        }
        cudaFreeAsync(tmp, ctx->stream);
    }
    // Theorem 3.1's solver on A~ (lambda = 0, lambda~ = lambda0)
    msp_general_t* inner = nullptr;
    if ((st = msp_general_create(ctx, g->As, s_ls, d, np, 0.0, lambda0, s, gamma, phi, gamma_phi, seed, &inner)) !=
        MSP_OK)
        return fail(st);
    g->inner = inner;
    g->s_ls = s_ls;
    *out = g;
    return MSP_OK;
}

void msp_lsq_destroy(msp_lsq_t* h) { msp_general_destroy(h); }

msp_status msp_lsq_solve(msp_ctx* ctx, msp_lsq_t* g, const double* b, double* x, const msp_opts* opts,
                         msp_info* info, double* resid_norm) {
    if (!ctx || !g || !g->inner) return msp_set_error(ctx, MSP_EINVAL, "lsq: NULL argument or not a lsq handle");
    MSP_TRY(check_vec_args(ctx, b));
    MSP_TRY(check_vec_args(ctx, x));
    msp_opts o;
    if (opts) o = *opts;
    else msp_default_opts(&o);
    if (!(o.tol > 0.0) || o.max_outer < 1 || o.level2_iters < 0 || o.level2_iters > 1000 || o.level3_iters < 0 ||
        o.level3_iters > 1000 || (o.precision != MSP_PREC_MIXED && o.precision != MSP_PREC_FP32) ||
        o.criterion != MSP_STOP_RESIDUAL || (o.precision == MSP_PREC_MIXED && !(o.refine_tol > 0.0)) ||
        !(o.inner_tol > 0.0) || o.max_inner < 1)
        return msp_set_error(ctx, MSP_EINVAL,
                             "lsq: need tol, refine_tol, inner_tol > 0, max_outer, max_inner >= 1, "
                             "0 <= level2_iters, level3_iters <= 1000, precision MIXED or FP32, the residual "
                             "criterion");
    msp::DeviceGuard guard(ctx->device);
    g->inner_tol = o.inner_tol;
    g->inner_maxit = o.max_inner;
    msp_info inf;
    std::memset(&inf, 0, sizeof inf);
    inf.lambda_tilde = g->inner->lam_tilde;
    const int np = (int)g->n_pad, na4 = np / 4;
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->err, 0, sizeof(int), ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->inner->err, 0, sizeof(int), ctx->stream));
    // c64 = A^T b in FP64 (row dots with a = 0 give t = b)
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->x64, 0, (size_t)np * 8, ctx->stream));
    int used = 0;
    MSP_TRY(launch_same<double>(ctx, ctx->stream, g->G, g->m, g->A, g->lda, na4, g->x64, b, 1.0, nullptr, g->part64,
                                g->n_pad, g->err, nullptr, &used));
    MSP_TRY(colsum<double>(ctx, ctx->stream, g, g->part64, g->n_pad, np, 1.0, nullptr, 0.0, nullptr, g->c64,
                           nullptr, used));
    double cn = 0.0;
    MSP_TRY(norm64(ctx, g, g->c64, &cn));
    msp_status result = MSP_OK;
    if (cn == 0.0) {
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(g->x64, 0, (size_t)np * 8, ctx->stream));
    } else {
        MSP_TRY(solve_refined(ctx, g, o, cn, &inf, &result));
    }
    // |A x - b| in FP64: row dots t = A x - b only
    MSP_TRY(launch_pass<double>(ctx, ctx->stream, g->G, g->m, g->A, g->lda, na4, g->A, g->lda, 0, g->x64, b, -1.0,
                                g->part64, g->part64, g->n_pad, g->err, nullptr, &used));
    k_norm2_64<<<1, kVecThreads, 0, ctx->stream>>>((int)g->m, g->part64, g->d64);
    MSP_CHECK_LAUNCH(ctx);
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(g->host + 12, g->d64, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(x, g->x64, (size_t)g->n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (resid_norm) *resid_norm = std::sqrt(g->host[12]);
    inf.status = result;
    if (info) *info = inf;
    if (result == MSP_ENOCONV)
        return msp_set_error(ctx, MSP_ENOCONV, "lsq: normal-equation residual %.3g above tol %.3g", inf.rel_resid,
                             o.tol);
    return result;
}

}  // extern "C"
