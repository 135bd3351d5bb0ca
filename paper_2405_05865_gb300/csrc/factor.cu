// Level-2 preconditioner of Algorithm 1, step 4, on sm_103a:
//   M2 = C~^T C~ + lambda~ W   (s x s, assembled in FP64),
//   M2 + nu I = L L^T          (FP64 Cholesky; nu = 0, then the stabilising
//                               shift retries described in msp.h),
//   L^{-1}                     (FP64), stored in the working precision as
//                               B = L^{-1} and B^T so that the level-2
//                               iteration applies M2^{-1} v = B^T (B v).
// The factorisation recursion halves the matrix:
//   [A11 . ; A21 A22]:  (L11, X11) = f(A11);  L21 = A21 X11^T;
//   A22 -= L21 L21^T;   (L22, X22) = f(A22);  X21 = -X22 (L21 X11),
// with a one-block Cholesky + inverse at the leaves (at most 32 x 32) and an
// FP64 GEMM kernel for the rest; L21 X11 runs on a side stream beside the
// factorisation of A22.
#include "bulk.cuh"
#include "msp_internal.cuh"

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// ----------------------------------------------------------- Gram (SIMT)

// M2[a][b] = sum_k Ct[k][a] Ct[k][b] + lam_t * W[a][b], FP64 output; pad rows
// (a >= s or b >= s) get the identity. One 64 x 64 tile of the upper
// triangle per block (mirrored), 256 threads each 4 x 4 outputs, K chunks of
// 16 from shared memory. Each chunk is summed in TA, then added into an
// (hi, lo) pair with Knuth's TwoSum (compensated summation), so the
// accumulated rounding error does not grow with K (K = n when Phi = I).
template <typename TA>
__device__ inline void two_sum_add(TA& hi, TA& lo, TA v) {
    TA s = hi + v;
    TA bp = s - hi;
    TA err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

constexpr int kGramSlices = 4;   // split-K slices of the Gram (combined in FP64)

// Partial Gram of one K slice: P[slice][a][b] = sum_{k in slice} Ct[k][a] Ct[k][b]
// for the upper-triangular 64 x 64 tile pairs (mirrored), FP64 output (hi + lo).
// blockIdx.x = tile pair, blockIdx.y = K slice.
template <typename TA>
__global__ void __launch_bounds__(256, 4) k_gram(const TA* __restrict__ Ct, int64_t K, int64_t ld,
                                                int64_t s_pad, double* __restrict__ P) {
    __shared__ __align__(16) TA As[16][64];
    __shared__ __align__(16) TA Bs[16][64];
    const int nt = (int)(s_pad / 64);
    int ta = 0, rem = blockIdx.x;
    while (rem >= nt - ta) { rem -= nt - ta; ++ta; }
    const int tb = ta + rem;
    const int a0 = ta * 64, b0 = tb * 64;
    const int64_t kper = ((K + kGramSlices - 1) / kGramSlices + 15) / 16 * 16;
    const int64_t kbeg = (int64_t)blockIdx.y * kper;
    const int64_t kend = min(K, kbeg + kper);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    TA hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { hi[i][j] = TA(0); lo[i][j] = TA(0); }
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e >> 6, cc = e & 63;
            bool in = (k0 + kk) < kend;
            As[kk][cc] = in ? Ct[(k0 + kk) * ld + a0 + cc] : TA(0);
            Bs[kk][cc] = in ? Ct[(k0 + kk) * ld + b0 + cc] : TA(0);
        }
        __syncthreads();
        TA acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = TA(0);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            TA av[4], bv[4];
            if constexpr (sizeof(TA) == 4) {
                const float4 va = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
                const float4 vb = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                av[0] = va.x; av[1] = va.y; av[2] = va.z; av[3] = va.w;
                bv[0] = vb.x; bv[1] = vb.y; bv[2] = vb.z; bv[3] = vb.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_add(hi[i][j], lo[i][j], acc[i][j]);
        __syncthreads();
    }
    double* Ps = P + (int64_t)blockIdx.y * s_pad * s_pad;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
            const double v = (double)hi[i][j] + (double)lo[i][j];
            Ps[a * s_pad + b] = v;
            Ps[b * s_pad + a] = v;
        }
}

// M2 = sum_slices P + lam_t W (FP64, fixed order), or + lam_t I when W is
// NULL; pad rows/cols get identity.
// The same partial Grams (FP32 input) with 128 x 128 tiles: 512 threads,
// each 8 rows (ty*4 + i and 64 + ty*4 + i) x 4 columns (tx*4 + j), K chunks
// of 16 double-buffered in shared memory by 16-byte async copies. Per output
// the arithmetic is k_gram's -- the same K slices, chunks of 16 summed in
// FP32 from zero in increasing k, TwoSum into (hi, lo) -- so P is the same
// to the bit; a thread's 32 outputs per shared-memory read of 12 values (4
// for k_gram's 16) keep the FP32 pipe, not shared memory, the limit.
__global__ void __launch_bounds__(512, 1) k_gram128(const float* __restrict__ Ct, int64_t K, int64_t ld,
                                                    int64_t s_pad, double* __restrict__ P) {
    __shared__ __align__(16) float As[2][16][128];
    __shared__ __align__(16) float Bs[2][16][128];
    const int nt = (int)(s_pad / 128);
    int ta = 0, rem = blockIdx.x;
    while (rem >= nt - ta) { rem -= nt - ta; ++ta; }
    const int tb = ta + rem;
    const int a0 = ta * 128, b0 = tb * 128;
    const int64_t kper = ((K + kGramSlices - 1) / kGramSlices + 15) / 16 * 16;
    const int64_t kbeg = (int64_t)blockIdx.y * kper;
    const int64_t kend = min(K, kbeg + kper);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // loader: thread t copies float4 (t & 31) of row t >> 5 of the chunk, of A and of B
    const int lk = (int)(threadIdx.x >> 5), lc = (int)(threadIdx.x & 31) * 4;
    auto issue = [&](int64_t k0, int st) {
        const int64_t k = k0 + lk;
        const bool in = k < kend;
        msp::cp_async16(&As[st][lk][lc], in ? Ct + k * ld + a0 + lc : Ct, in);
        msp::cp_async16(&Bs[st][lk][lc], in ? Ct + k * ld + b0 + lc : Ct, in);
    };
    float hi[8][4], lo[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { hi[i][j] = 0.f; lo[i][j] = 0.f; }
    if (kbeg < kend) issue(kbeg, 0);
    msp::cp_async_commit();
    int st = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
        if (k0 + 16 < kend) issue(k0 + 16, st ^ 1);
        msp::cp_async_commit();
        msp::cp_async_wait<1>();
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 x0 = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
            const float4 x1 = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
            const float4 y = *reinterpret_cast<const float4*>(&Bs[st][kk][tx * 4]);
            const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const float bv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_add(hi[i][j], lo[i][j], acc[i][j]);
        __syncthreads();
        st ^= 1;
    }
    double* Ps = P + (int64_t)blockIdx.y * s_pad * s_pad;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t a = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4)), b = b0 + tx * 4 + j;
            const double v = (double)hi[i][j] + (double)lo[i][j];
            Ps[a * s_pad + b] = v;
            Ps[b * s_pad + a] = v;
        }
}

// Split-K partial Grams of FP32 Ct into P (kGramSlices x s_pad x s_pad).
msp_status launch_gram_f32(msp_ctx* ctx, const float* Ct, int64_t K, int64_t ld, int64_t sp, double* P) {
    if (sp % 128 == 0 && ld % 4 == 0 && ((uintptr_t)Ct & 15) == 0) {
        const int nt = (int)(sp / 128);
        dim3 grid((unsigned)(nt * (nt + 1) / 2), kGramSlices);
        k_gram128<<<grid, 512, 0, ctx->stream>>>(Ct, K, ld, sp, P);
    } else {
        const int nt = (int)(sp / 64);
        dim3 grid((unsigned)(nt * (nt + 1) / 2), kGramSlices);
        k_gram<float><<<grid, 256, 0, ctx->stream>>>(Ct, K, ld, sp, P);
    }
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

template <typename TA>
__global__ void k_gram_finish(const double* __restrict__ P, const TA* __restrict__ W, double lam_t,
                              int64_t s, int64_t s_pad, double* __restrict__ M2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    const int64_t a = e / s_pad, b = e % s_pad;
    double v;
    if (a < s && b < s) {
        v = 0.0;
#pragma unroll
        for (int sl = 0; sl < kGramSlices; ++sl) v += P[(int64_t)sl * s_pad * s_pad + e];
        v += W ? lam_t * (double)W[e] : (a == b ? lam_t : 0.0);
    } else {
        v = (a == b) ? 1.0 : 0.0;
    }
    M2[e] = v;
}

// W <- (W + W^T)/2 in place (working precision) and W64 = (double)W.
template <typename T>
__global__ void k_symmetrize(T* __restrict__ W, double* __restrict__ W64, int64_t s_pad) {
    int64_t a = blockIdx.y * 32 + threadIdx.y, b = blockIdx.x * 32 + threadIdx.x;
    if (a >= s_pad || b >= s_pad || b > a) return;
    T v = (W[a * s_pad + b] + W[b * s_pad + a]) * T(0.5);
    W[a * s_pad + b] = v;
    W[b * s_pad + a] = v;
    W64[a * s_pad + b] = (double)v;
    W64[b * s_pad + a] = (double)v;
}

// ----------------------------------------------------------- FP64 GEMM

// Cm = alpha * op(A) op(B) + beta * Cm, row-major; op(A) is m x k, op(B) k x n.
// TS x TS output tile (TS = 16 or 32), 256 threads, K chunks of 16. The
// triangular structure of the operands limits the K range of each tile:
//   tri_a = 1: op(A) lower triangular (A[i][k] = 0 for k > i)
//   tri_b = 1: op(B) upper triangular (B[k][j] = 0 for k > j)
//   tri_b = 2: op(B) lower triangular (B[k][j] = 0 for k < j)
//   lower_out: only tiles touching the lower triangle (i >= j) are computed.
template <bool TA_, bool TB_, int TS>
__global__ void __launch_bounds__(256) k_dgemm(int64_t m, int64_t n, int64_t k, double alpha,
                                              const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb,
                                              double beta, double* __restrict__ Cm, int64_t ldc,
                                              int tri_a, int tri_b, int lower_out) {
    constexpr int PT = TS / 16;              // outputs per thread per dimension
    __shared__ double As[16][TS + 1];        // As[kk][i] = op(A)[i][k0+kk]
    __shared__ double Bs[16][TS + 1];        // Bs[kk][j] = op(B)[k0+kk][j]
    const int64_t i0 = (int64_t)blockIdx.y * TS, j0 = (int64_t)blockIdx.x * TS;
    if (lower_out && j0 > i0 + TS - 1) return;
    int64_t kbeg = 0, kend = k;
    if (tri_a == 1) kend = min(kend, i0 + TS);
    if (tri_b == 1) kend = min(kend, j0 + TS);
    if (tri_b == 2) kbeg = (j0 / 16) * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[PT][PT];
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * TS; e += 256) {
            int kk, ii;
            if (TA_) { ii = e % TS; kk = e / TS; }   // A^T: read A[k][i], contiguous in i
            else { kk = e & 15; ii = e >> 4; }        // A: read A[i][k], contiguous in k
            int64_t gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < m && gk < kend) v = TA_ ? A[gk * lda + gi] : A[gi * lda + gk];
            As[kk][ii] = v;
        }
        for (int e = threadIdx.x; e < 16 * TS; e += 256) {
            int kk, jj;
            if (TB_) { kk = e & 15; jj = e >> 4; }    // B^T: read B[j][k], contiguous in k
            else { jj = e % TS; kk = e / TS; }        // B: read B[k][j], contiguous in j
            int64_t gj = j0 + jj, gk = k0 + kk;
            double v = 0.0;
            if (gj < n && gk < kend) v = TB_ ? B[gj * ldb + gk] : B[gk * ldb + gj];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[PT], bv[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) av[i] = As[kk][ty * PT + i];
#pragma unroll
            for (int j = 0; j < PT; ++j) bv[j] = Bs[kk][tx * PT + j];
#pragma unroll
            for (int i = 0; i < PT; ++i)
#pragma unroll
                for (int j = 0; j < PT; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            int64_t gi = i0 + ty * PT + i, gj = j0 + tx * PT + j;
            if (gi < m && gj < n) {
                double c = beta == 0.0 ? 0.0 : beta * Cm[gi * ldc + gj];
                Cm[gi * ldc + gj] = c + alpha * acc[i][j];
            }
        }
}

// ----------------------------------------------------- float-float kernels
//
// The factor of an FP32 sketch runs in float-float arithmetic on the FP32
// pipe: a value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)
// / 2 once normalised), a product is exact by FMA (TwoProduct, Dekker), a sum
// by TwoSum (Knuth), about 2^-46 relative per operation. FP64 runs at 2
// lanes per clock per SM on this part, the FP32 pipe at 128. Every operation
// below uses the _rn intrinsics, which the compiler never contracts.

__device__ __forceinline__ float2 ff_fast2sum(float a, float b) {   // needs |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 ff_2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// (sh, sl) += a b, sl collecting the low parts until the next ff_norm
__device__ __forceinline__ void ff_fma_acc(float& sh, float& sl, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float2 t = ff_2sum(sh, p);
    sh = t.x;
    sl = __fadd_rn(sl, __fadd_rn(t.y, e));
}

__device__ __forceinline__ float2 ff_norm(float sh, float sl) { return ff_2sum(sh, sl); }

__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_fast2sum(p, e);
}

__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 s = ff_2sum(a.x, b.x);
    return ff_fast2sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 ff_from_double(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

// k_dgemm in float-float: the same tiling, triangular limits and lower_out,
// operands and result stored as float2 (hi, lo). alpha is +-1 and beta 0 or
// 1 (what the recursion uses): Cm = beta Cm +- op(A) op(B). The accumulators
// are renormalised after every K chunk of 16.
template <bool TA_, bool TB_, int TS>
__global__ void __launch_bounds__(256) k_ffgemm(int64_t m, int64_t n, int64_t k, float alpha,
                                               const float2* __restrict__ A, int64_t lda,
                                               const float2* __restrict__ B, int64_t ldb,
                                               int beta, float2* __restrict__ Cm, int64_t ldc,
                                               int tri_a, int tri_b, int lower_out) {
    constexpr int PT = TS / 16;
    __shared__ float2 As[16][TS + 1];
    __shared__ float2 Bs[16][TS + 1];
    const int64_t i0 = (int64_t)blockIdx.y * TS, j0 = (int64_t)blockIdx.x * TS;
    if (lower_out && j0 > i0 + TS - 1) return;
    int64_t kbeg = 0, kend = k;
    if (tri_a == 1) kend = min(kend, i0 + TS);
    if (tri_b == 1) kend = min(kend, j0 + TS);
    if (tri_b == 2) kbeg = (j0 / 16) * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float sh[PT][PT], sl[PT][PT];
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) sh[i][j] = sl[i][j] = 0.f;
    const float2 zero = make_float2(0.f, 0.f);
    // the K chunk's operands, loaded into registers one chunk ahead
    constexpr int LD = 16 * TS / 256;        // elements per thread per operand
    float2 ra[LD], rb[LD];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = threadIdx.x + 256 * u;
            int kk, ii;
            if (TA_) { ii = e % TS; kk = e / TS; }
            else { kk = e & 15; ii = e >> 4; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            ra[u] = (gi < m && gk < kend) ? (TA_ ? A[gk * lda + gi] : A[gi * lda + gk]) : zero;
            int jj;
            if (TB_) { kk = e & 15; jj = e >> 4; }
            else { jj = e % TS; kk = e / TS; }
            const int64_t gj = j0 + jj, gk2 = k0 + kk;
            rb[u] = (gj < n && gk2 < kend) ? (TB_ ? B[gj * ldb + gk2] : B[gk2 * ldb + gj]) : zero;
        }
    };
    if (kbeg < kend) fetch(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = threadIdx.x + 256 * u;
            int kk, ii, jj;
            if (TA_) { ii = e % TS; kk = e / TS; }
            else { kk = e & 15; ii = e >> 4; }
            As[kk][ii] = ra[u];
            if (TB_) { kk = e & 15; jj = e >> 4; }
            else { jj = e % TS; kk = e / TS; }
            Bs[kk][jj] = rb[u];
        }
        __syncthreads();
        if (k0 + 16 < kend) fetch(k0 + 16);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float2 av[PT], bv[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) av[i] = As[kk][ty * PT + i];
#pragma unroll
            for (int j = 0; j < PT; ++j) bv[j] = Bs[kk][tx * PT + j];
#pragma unroll
            for (int i = 0; i < PT; ++i)
#pragma unroll
                for (int j = 0; j < PT; ++j) ff_fma_acc(sh[i][j], sl[i][j], av[i], bv[j]);
        }
#pragma unroll
        for (int i = 0; i < PT; ++i)
#pragma unroll
            for (int j = 0; j < PT; ++j) {
                const float2 t = ff_norm(sh[i][j], sl[i][j]);
                sh[i][j] = t.x;
                sl[i][j] = t.y;
            }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            const int64_t gi = i0 + ty * PT + i, gj = j0 + tx * PT + j;
            if (gi < m && gj < n) {
                float2 r = make_float2(sh[i][j], sl[i][j]);
                if (alpha < 0.f) r = ff_neg(r);
                if (beta) r = ff_add(Cm[gi * ldc + gj], r);
                Cm[gi * ldc + gj] = r;
            }
        }
}

constexpr int kLeafSmem = 2 * 64 * 65 * (int)sizeof(double);
constexpr int kLeafUpd = 256;                 // eight update warps (32 x 8 thread grid)
constexpr int kLeafThreads = kLeafUpd + 32;   // and the pivot warp

// 1/sqrt(d) for a positive normal FP64 d: FP32 reciprocal square root as the
// seed, then two Newton-Raphson steps y <- y (3 - d y^2) / 2 for f(y) =
// 1/y^2 - d (quadratic convergence: ~2^-22 -> 2^-44 -> FP64 rounding). The
// FP64 square root and division cost tens of FP64 instructions each on this
// part, whose FP64 unit takes ~64 cycles per warp instruction.
__device__ inline double rsqrt_newton(double d) {
    if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
    const double hd = 0.5 * d;
    y = y * fma(-hd * y, y, 1.5);
    y = y * fma(-hd * y, y, 1.5);
    return y;
}

// 1/d for a positive normal FP64 d: FP32 reciprocal as the seed, then two
// Newton-Raphson steps r <- r + r (1 - d r) for f(r) = 1/r - d.
__device__ inline double rcp_newton(double d) {
    if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / d;
    double r = (double)(1.0f / (float)d);
    r = fma(r, fma(-d, r, 1.0), r);
    r = fma(r, fma(-d, r, 1.0), r);
    return r;
}

// Cholesky and inverse of an nb x nb (nb <= 64; the recursion passes at most
// 32) FP64 block on one SM:
// M = L L^T (lower triangle of M overwritten with L), X = L^{-1}.
// One elimination sweep in LDL^T form: at step k every row i > k takes
// t_i = a_ik / d_k and updates both its Schur-complement entries,
// a_ij -= t_i a_jk (k < j < i), and its row of X, x_ij -= t_i x_kj (j <= k),
// with X starting as the identity -- the same row operations turn the
// identity into L_u^{-1} for A = L_u D L_u^T. Every update of a step is
// independent (no substitution chains), and the two parts together keep the
// work per step near n^2 / 2. The diagonal is kept apart by a fifth warp,
// which also forms the next pivot d_{k+1} and 1/d_{k+1} while the update
// warps work, so a step costs one barrier. At the end L = L_u D^{1/2}
// (l_ik = a_ik / sqrt(d_k), l_kk = sqrt(d_k)) and L^{-1} = D^{-1/2} L_u^{-1}.
// A pivot that is not positive and finite sets *fail (and is replaced by 1).
__global__ void __launch_bounds__(kLeafThreads) k_chol_leaf(double* __restrict__ M, double* __restrict__ X,
                                                           int64_t ld, int nb, int* __restrict__ fail) {
    extern __shared__ __align__(16) double leaf_smem[];
    double (*a)[65] = reinterpret_cast<double (*)[65]>(leaf_smem);
    double (*x)[65] = reinterpret_cast<double (*)[65]>(leaf_smem + 64 * 65);
    __shared__ double piv[64], rinv[64], rs[64];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool pivot_warp = tid >= kLeafUpd;
    if (tid == 0) bad = 0;
    for (int e = tid; e < nb * nb; e += kLeafThreads) {
        const int i = e / nb, j = e % nb;
        a[i][j] = (j <= i) ? M[i * ld + j] : 0.0;
        x[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // pivot warp: the diagonal of rows lane and lane + 32
    double dg0 = 1.0, dg1 = 1.0;
    if (pivot_warp) {
        if (lane < nb) dg0 = a[lane][lane];
        if (lane + 32 < nb) dg1 = a[lane + 32][lane + 32];
        if (lane == 0) {
            double d = dg0;
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
                d = 1.0;
            }
            piv[0] = d;
            rinv[0] = rcp_newton(d);
        }
    }
    __syncthreads();
    // update threads: row offsets interleaved over the warps, so that the
    // last steps (few rows) still use all eight
    const int tx = tid & 7, ty = tid >> 3;
    const int rr = ((ty & 3) << 3) | (ty >> 2);
    for (int k = 0; k < nb; ++k) {
        const double rk = rinv[k];
        if (!pivot_warp) {
            for (int i = k + 1 + rr; i < nb; i += 32) {
                const double ti = a[i][k] * rk;
                for (int j = tx; j <= k; j += 8) x[i][j] = fma(-ti, x[k][j], x[i][j]);
                for (int j = k + 1 + tx; j < i; j += 8) a[i][j] = fma(-ti, a[j][k], a[i][j]);
            }
        } else if (k + 1 < nb) {
            if (lane > k && lane < nb) {
                const double ti = a[lane][k] * rk;
                dg0 = fma(-ti, a[lane][k], dg0);
            }
            if (lane + 32 > k && lane + 32 < nb) {
                const double ti = a[lane + 32][k] * rk;
                dg1 = fma(-ti, a[lane + 32][k], dg1);
            }
            const int kn = k + 1;
            if (lane == (kn & 31)) {
                double d = kn < 32 ? dg0 : dg1;
                if (!(d > 0.0) || !isfinite(d)) {
                    bad = 1;
                    d = 1.0;
                }
                piv[kn] = d;
                rinv[kn] = rcp_newton(d);
            }
        }
        __syncthreads();
    }
    for (int k = tid; k < nb; k += kLeafThreads) rs[k] = rsqrt_newton(piv[k]);
    __syncthreads();
    for (int e = tid; e < nb * nb; e += kLeafThreads) {
        const int i = e / nb, j = e % nb;
        if (j < i) M[i * ld + j] = a[i][j] * rs[j];
        else if (j == i) M[i * ld + j] = piv[i] * rs[i];
        X[i * ld + j] = (j <= i) ? x[i][j] * rs[i] : 0.0;
    }
    if (tid == 0 && bad) atomicExch(fail, 1);
}

// 1/d in float-float for a positive normal d: the FP32 reciprocal r0, then
// one Newton-Raphson step r = r0 + r0 (1 - d r0) with the residual 1 - d r0
// formed exactly to first order (1 - hi(d r0) is exact: d r0 is within
// 2^-23 of 1), ~2^-46 relative.
__device__ __forceinline__ float2 ff_rcp(float2 d) {
    const float r0 = __frcp_rn(d.x);
    const float p = __fmul_rn(d.x, r0);
    const float pe = __fmaf_rn(d.y, r0, __fmaf_rn(d.x, r0, -p));
    const float res = __fsub_rn(__fsub_rn(1.0f, p), pe);
    return ff_fast2sum(r0, __fmul_rn(r0, res));
}

// d^{-1/2} in float-float for a positive normal d: the FP32 rsqrtf r0, then
// one Newton-Raphson step r = r0 + r0 (1 - d r0^2) / 2 with the residual
// 1 - d r0^2 formed to first order exactly (r0^2 and d r0^2 by TwoProduct;
// d r0^2 is within about 2^-21 of 1), ~2^-43 relative.
__device__ __forceinline__ float2 ff_rsqrt(float2 d) {
    const float r0 = rsqrtf(d.x);
    const float th = __fmul_rn(r0, r0), tl = __fmaf_rn(r0, r0, -th);
    const float p = __fmul_rn(d.x, th);
    const float pe = __fmaf_rn(d.y, th, __fmaf_rn(d.x, tl, __fmaf_rn(d.x, th, -p)));
    const float res = __fsub_rn(__fsub_rn(1.0f, p), pe);
    return ff_fast2sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), res));
}

// k_chol_leaf in float-float (the same elimination and pivot warp; the
// block and its inverse in shared memory as float2; 31 update warps take a
// row each, a lane per element, so that a step of a 32-wide leaf is one
// dependent chain per lane, where the FP64 version is bound by the FP64
// pipe): M = L L^T,
// X = L^{-1}, both float2 with leading dimension ld.
constexpr int kFFUpd = 31 * 32;              // update warps of the float-float leaf
constexpr int kFFThreads = kFFUpd + 32;       // and its pivot warp

__global__ void __launch_bounds__(kFFThreads) k_chol_leaf_ff(float2* __restrict__ M, float2* __restrict__ X,
                                                              int64_t ld, int nb, int* __restrict__ fail) {
    extern __shared__ __align__(16) float2 leaf_smem_ff[];
    float2 (*a)[65] = reinterpret_cast<float2 (*)[65]>(leaf_smem_ff);
    float2 (*x)[65] = reinterpret_cast<float2 (*)[65]>(leaf_smem_ff + 64 * 65);
    __shared__ float2 piv[64], rinv[64], rs[64];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool pivot_warp = tid >= kFFUpd;
    const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
    if (tid == 0) bad = 0;
    for (int e = tid; e < nb * nb; e += kFFThreads) {
        const int i = e / nb, j = e % nb;
        a[i][j] = (j <= i) ? M[i * ld + j] : zero;
        x[i][j] = (i == j) ? one : zero;
    }
    __syncthreads();
    auto pivot_ok = [](float2 d) { return d.x > 0.f && isfinite(d.x); };
    float2 dg0 = one, dg1 = one;
    if (pivot_warp) {
        if (lane < nb) dg0 = a[lane][lane];
        if (lane + 32 < nb) dg1 = a[lane + 32][lane + 32];
        if (lane == 0) {
            float2 d = dg0;
            if (!pivot_ok(d)) {
                bad = 1;
                d = one;
            }
            piv[0] = d;
            rinv[0] = ff_rcp(d);
        }
    }
    __syncthreads();
    const int warp = tid >> 5;
    for (int k = 0; k < nb; ++k) {
        const float2 rk = rinv[k];
        if (!pivot_warp) {
            // one warp per row i = k + 1 + w, + 31, ...: lane j < i updates
            // its element of the row, x[i][j] (j <= k) or a[i][j] (k < j <
            // i), so the step's updates spread evenly over the lanes (no
            // store of the step touches row k or column k)
            for (int i = k + 1 + warp; i < nb; i += kFFUpd / 32) {
                const float2 nti = ff_neg(ff_mul(a[i][k], rk));
                for (int j = lane; j < i; j += 32) {
                    const bool xs = j <= k;
                    const float2 src = xs ? x[k][j] : a[j][k];
                    float2* dst = xs ? &x[i][j] : &a[i][j];
                    const float2 v = *dst;
                    float h = v.x, l = v.y;
                    ff_fma_acc(h, l, nti, src);
                    *dst = ff_norm(h, l);
                }
            }
        } else if (k + 1 < nb) {
            if (lane > k && lane < nb) {
                const float2 nti = ff_neg(ff_mul(a[lane][k], rk));
                float h = dg0.x, l = dg0.y;
                ff_fma_acc(h, l, nti, a[lane][k]);
                dg0 = ff_norm(h, l);
            }
            if (lane + 32 > k && lane + 32 < nb) {
                const float2 nti = ff_neg(ff_mul(a[lane + 32][k], rk));
                float h = dg1.x, l = dg1.y;
                ff_fma_acc(h, l, nti, a[lane + 32][k]);
                dg1 = ff_norm(h, l);
            }
            const int kn = k + 1;
            if (lane == (kn & 31)) {
                float2 d = kn < 32 ? dg0 : dg1;
                if (!pivot_ok(d)) {
                    bad = 1;
                    d = one;
                }
                piv[kn] = d;
                rinv[kn] = ff_rcp(d);
            }
        }
        __syncthreads();
    }
    for (int k = tid; k < nb; k += kFFThreads) rs[k] = ff_rsqrt(piv[k]);
    __syncthreads();
    for (int e = tid; e < nb * nb; e += kFFThreads) {
        const int i = e / nb, j = e % nb;
        if (j < i) M[i * ld + j] = ff_mul(a[i][j], rs[j]);
        else if (j == i) M[i * ld + j] = ff_mul(piv[i], rs[i]);
        X[i * ld + j] = (j <= i) ? ff_mul(x[i][j], rs[i]) : zero;
    }
    if (tid == 0 && bad) atomicExch(fail, 1);
}

__global__ void k_copy_add_diag(const double* __restrict__ src, double* __restrict__ dst,
                                int64_t s_pad, double nu) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    int64_t i = e / s_pad, j = e % s_pad;
    dst[e] = src[e] + ((i == j) ? nu : 0.0);
}

// dst = float-float of (src + nu I) scale (scale a power of two: exact)
__global__ void k_copy_add_diag_ff(const double* __restrict__ src, float2* __restrict__ dst,
                                   int64_t s_pad, double nu, double scale) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    int64_t i = e / s_pad, j = e % s_pad;
    dst[e] = ff_from_double((src[e] + ((i == j) ? nu : 0.0)) * scale);
}

// dst = src scale in FP64 (scale a power of two)
__global__ void k_ff_to_double(const float2* __restrict__ src, double* __restrict__ dst, int64_t count,
                               double scale) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    dst[e] = ff_to_double(src[e]) * scale;
}

// Frobenius norm^2 partials (single block, deterministic order).
// |M|_F^2 in two fixed-order stages: kFroBlocks block partials, then one
// block sums them.
constexpr int kFroBlocks = 128;

__global__ void __launch_bounds__(256) k_fro2_part(const double* __restrict__ M, int64_t m,
                                                  double* __restrict__ part) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        acc += M[e] * M[e];
    acc = msp::warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w];
        part[blockIdx.x] = v;
    }
}

__global__ void k_fro2_final(const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int b = 0; b < kFroBlocks; ++b) v += part[b];
        *out = v;
    }
}

template <typename T>
__global__ void k_cast_tri(const double* __restrict__ X, T* __restrict__ B, T* __restrict__ Bt,
                           int64_t s_pad) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    int64_t i = e / s_pad, j = e % s_pad;
    double v = (j <= i) ? X[e] : 0.0;
    B[e] = (T)v;
    Bt[j * s_pad + i] = (T)v;
}

template <int TS>
void launch_dgemm_ts(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     double* Cm, int64_t ldc, int tri_a, int tri_b, int lower_out) {
    dim3 grid((unsigned)((n + TS - 1) / TS), (unsigned)((m + TS - 1) / TS));
    if (!ta && !tb) k_dgemm<false, false, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else if (!ta && tb) k_dgemm<false, true, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else if (ta && !tb) k_dgemm<true, false, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else k_dgemm<true, true, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
}

msp_status dgemm(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* Cm, int64_t ldc, int tri_a = 0, int tri_b = 0, int lower_out = 0) {
    // FP64 work is pipe-bound on this part: prefer the larger tile only when it
    // still yields two blocks per SM
    const int64_t tiles32 = ((m + 31) / 32) * ((n + 31) / 32);
    if (tiles32 >= 2 * ctx->num_sms)
        launch_dgemm_ts<32>(ctx, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else
        launch_dgemm_ts<16>(ctx, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

template <int TS>
void launch_ffgemm_ts(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                      const float2* A, int64_t lda, const float2* B, int64_t ldb, int beta,
                      float2* Cm, int64_t ldc, int tri_a, int tri_b, int lower_out) {
    dim3 grid((unsigned)((n + TS - 1) / TS), (unsigned)((m + TS - 1) / TS));
    if (!ta && !tb) k_ffgemm<false, false, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else if (!ta && tb) k_ffgemm<false, true, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else if (ta && !tb) k_ffgemm<true, false, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
    else k_ffgemm<true, true, TS><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
}

// The recursion's products on the two storages: FP64, or float-float
// (alpha +-1, beta 0 or 1).
msp_status gemm_s(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* Cm, int64_t ldc, int tri_a, int tri_b, int lower_out) {
    return dgemm(ctx, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc, tri_a, tri_b, lower_out);
}

msp_status gemm_s(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                  const float2* A, int64_t lda, const float2* B, int64_t ldb, double beta,
                  float2* Cm, int64_t ldc, int tri_a, int tri_b, int lower_out) {
    if (!(alpha == 1.0 || alpha == -1.0) || !(beta == 0.0 || beta == 1.0))
        return msp_set_error(ctx, MSP_EINVAL, "factor: float-float product needs alpha = +-1, beta = 0 or 1");
    // the FP32 pipe has room for the larger tile once it fills the SMs
    const int64_t tiles32 = ((m + 31) / 32) * ((n + 31) / 32);
    if (tiles32 >= ctx->num_sms)
        launch_ffgemm_ts<32>(ctx, ta, tb, m, n, k, (float)alpha, A, lda, B, ldb, (int)beta, Cm, ldc, tri_a, tri_b, lower_out);
    else
        launch_ffgemm_ts<16>(ctx, ta, tb, m, n, k, (float)alpha, A, lda, B, ldb, (int)beta, Cm, ldc, tri_a, tri_b, lower_out);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

template <typename Kern>
msp_status leaf_attr(msp_ctx* ctx, Kern kern, std::atomic<bool>* attr_set) {
    // set once per device; batch set-up calls this from several threads
    const int d = ctx->device;
    if (d < 0 || d >= 64 || !attr_set[d].load()) {
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafSmem));
        if (d >= 0 && d < 64) attr_set[d] = true;
    }
    return MSP_OK;
}

msp_status leaf_s(msp_ctx* ctx, double* M, double* X, int64_t ld, int64_t n, int* fail) {
    static std::atomic<bool> attr_set[64];
    MSP_TRY(leaf_attr(ctx, k_chol_leaf, attr_set));
    k_chol_leaf<<<1, kLeafThreads, kLeafSmem, ctx->stream>>>(M, X, ld, (int)n, fail);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status leaf_s(msp_ctx* ctx, float2* M, float2* X, int64_t ld, int64_t n, int* fail) {
    static std::atomic<bool> attr_set[64];
    MSP_TRY(leaf_attr(ctx, k_chol_leaf_ff, attr_set));
    k_chol_leaf_ff<<<1, kFFThreads, kLeafSmem, ctx->stream>>>(M, X, ld, (int)n, fail);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// Recursive Cholesky + inverse of the n x n block at offset `off` of M (ld),
// inverse into X (same offsets); T1/T2 are n x n temporaries (ld). Only X =
// L^{-1} is kept: M is scratch (the Schur complements overwrite its lower
// triangle, the leaves leave their L blocks there, L21 is not stored). Leaves
// of at most 32: a leaf runs on one SM, whose FP64 pipe bounds it (its work
// grows as nb^3), while the products of the recursion spread over all SMs.
template <typename S>
msp_status chol_inv(msp_ctx* ctx, S* M, S* X, S* T1, S* T2, int64_t ld,
                    int64_t off, int64_t n, int* fail, int depth) {
    if (n <= 32) return leaf_s(ctx, M + off * ld + off, X + off * ld + off, ld, n, fail);
    int64_t n1 = std::max<int64_t>(32, (n / 2) / 32 * 32);
    int64_t n2 = n - n1;
    S* A21 = M + (off + n1) * ld + off;
    S* A22 = M + (off + n1) * ld + off + n1;
    S* X11 = X + off * ld + off;
    S* X21 = X + (off + n1) * ld + off;
    S* X22 = X + (off + n1) * ld + off + n1;
    MSP_TRY(chol_inv(ctx, M, X, T1, T2, ld, off, n1, fail, depth + 1));
    // T1 = L21 = A21 X11^T   (n2 x n1; X11^T is upper triangular)
    MSP_TRY(gemm_s(ctx, false, true, n2, n1, n1, 1.0, A21, ld, X11, ld, 0.0, T1, ld, 0, 1, 0));
    // T2 = L21 X11 (X11 lower) needs only T1 and X11, so it runs on the side
    // stream of this depth while A22 is updated and factored on the main
    // stream. Disjoint memory: T1 and T2 hold columns [0, n1) of the
    // temporaries, the second half works in columns [n1, n) of them.
    // The stream and both events of this depth are the context's (created
    // once): recursion at one depth is sequential, and every wait on an
    // event is enqueued before the event is recorded again.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_t1 = nullptr, ev_t2 = nullptr;
    if (ctx->fac_overlap && depth < 8) {
        cudaEvent_t* ev = ctx->fac_ev[depth];
        if ((ctx->fac_side[depth] ||
             cudaStreamCreateWithFlags(&ctx->fac_side[depth], cudaStreamNonBlocking) == cudaSuccess) &&
            (ev[0] || cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess) &&
            (ev[1] || cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess)) {
            side = ctx->fac_side[depth];
            ev_t1 = ev[0];
            ev_t2 = ev[1];
        }
    }
    if (side && (cudaEventRecord(ev_t1, ctx->stream) != cudaSuccess ||
                 cudaStreamWaitEvent(side, ev_t1, 0) != cudaSuccess)) {
        cudaGetLastError();
        side = nullptr;     // fall back to the main stream
    }
    if (!side) cudaGetLastError();
    msp_status st = MSP_OK;
    if (side) {
        cudaStream_t main_stream = ctx->stream;
        ctx->stream = side;
        st = gemm_s(ctx, false, false, n2, n1, n1, 1.0, T1, ld, X11, ld, 0.0, T2, ld, 0, 2, 0);
        ctx->stream = main_stream;
        if (st == MSP_OK && cudaEventRecord(ev_t2, side) != cudaSuccess)
            st = msp_set_error(ctx, MSP_ECUDA, "factor: side stream record failed");
    }
    // A22 -= L21 L21^T (lower triangle is all the recursion reads)
    if (st == MSP_OK)
        st = gemm_s(ctx, false, true, n2, n2, n1, -1.0, T1, ld, T1, ld, 1.0, A22, ld, 0, 0, 1);
    if (st == MSP_OK) st = chol_inv(ctx, M, X, T1 + n1, T2 + n1, ld, off + n1, n2, fail, depth + 1);
    if (st == MSP_OK) {
        if (side) {
            if (cudaStreamWaitEvent(ctx->stream, ev_t2, 0) != cudaSuccess)
                st = msp_set_error(ctx, MSP_ECUDA, "factor: side stream join failed");
        } else {
            st = gemm_s(ctx, false, false, n2, n1, n1, 1.0, T1, ld, X11, ld, 0.0, T2, ld, 0, 2, 0);
        }
    }
    if (side && st != MSP_OK) cudaStreamSynchronize(side);
    MSP_TRY(st);
    // X21 = -X22 T2 (X22 lower)
    MSP_TRY(gemm_s(ctx, false, false, n2, n1, n2, -1.0, X22, ld, T2, ld, 0.0, X21, ld, 1, 0, 0));
    return MSP_OK;
}

// One float-float factor attempt (chol_inv on scratch buffers) replayed
// from a CUDA graph: the recursion issues about 130 launches of a few
// microseconds each, whose host-side cost would otherwise pace the GPU. The
// executable is keyed by the buffers and the size; the side-stream forks of
// the recursion become parallel branches of the graph. Where capture is
// not possible the recursion launches on the stream.
msp_status chol_inv_ff_graphed(msp_ctx* ctx, float2* M, float2* X, float2* T1, float2* T2, int64_t sp,
                               int* fail) {
    struct Key {
        const void *M, *X, *T1, *T2, *fail;
        int64_t sp;
        int overlap, device;
    } key;
    std::memset(&key, 0, sizeof key);
    key.M = M; key.X = X; key.T1 = T1; key.T2 = T2; key.fail = fail;
    key.sp = sp;
    key.overlap = ctx->fac_overlap;
    key.device = ctx->device;
    static_assert(sizeof(Key) <= sizeof(ctx->fac_key), "factor graph key too large");
    const bool hit = ctx->fac_exec && ctx->fac_key_len == sizeof key &&
                     std::memcmp(ctx->fac_key, &key, sizeof key) == 0;
    if (!hit) {
        msp_fac_graph_release(ctx);
        bool ok = ctx->cap_stream != nullptr ||
                  cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) ok = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            const cudaStream_t saved = ctx->stream;
            const int64_t l0 = ctx->launches;
            ctx->stream = ctx->cap_stream;
            const msp_status st = chol_inv(ctx, M, X, T1, T2, sp, 0, sp, fail, 0);
            ctx->stream = saved;
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
            const int kernels = (int)(ctx->launches - l0);
            ctx->launches = l0;
            ok = st == MSP_OK && ce == cudaSuccess && graph != nullptr &&
                 cudaGraphInstantiate(&ctx->fac_exec, graph, 0) == cudaSuccess;
            if (ok) {
                ctx->fac_graph = graph;
                std::memcpy(ctx->fac_key, &key, sizeof key);
                ctx->fac_key_len = sizeof key;
                ctx->fac_kernels = kernels;
            } else {
                ctx->fac_exec = nullptr;
                if (graph) cudaGraphDestroy(graph);
            }
        }
        cudaGetLastError();
        if (!ok) return chol_inv(ctx, M, X, T1, T2, sp, 0, sp, fail, 0);
    }
    MSP_CUDA_TRY(ctx, cudaGraphLaunch(ctx->fac_exec, ctx->stream));
    ctx->launches += ctx->fac_kernels;
    return MSP_OK;
}

// Cholesky inverse of M + nu I (lower L^{-1} into Linv64), s_pad x s_pad
// FP64 M with identity padding. FP32 data: M carries rounding errors of
// about 2^-24 |M|_F (its operands are FP32), which leave it indefinite by
// that much where it has tiny eigenvalues; nu starts there, which saves a
// second factorisation. FP64 data: unshifted first, then s 2^-52 |M|_F.
// Then nu x 100 per retry, at most 4 retries, else MSP_ENOTPD.
msp_status factor_shifted(msp_ctx* ctx, const double* M, int64_t s, int64_t sp, bool fp32_data,
                          double* Linv64, double* shift_out, int* retries_out) {
    // FP32 data: the factorisation in float-float (its backward error, a
    // small multiple of s 2^-46 |M|, stays far below the shift 2^-24 |M|_F
    // the data needs), on M scaled by a power of four to |M|_F in [1, 4) so
    // that no float range limit is near
    const bool ff = fp32_data && ctx->factor_ff;
    void* scr = nullptr;
    size_t mat = (size_t)sp * sp * 8;
    MSP_TRY(msp_scratch(ctx, (ff ? 4 : 3) * mat + 2048, &scr));
    double* Mw = (double*)scr;
    double* T1 = Mw + sp * sp;
    double* T2 = T1 + sp * sp;
    float2* Xff = reinterpret_cast<float2*>(T2 + sp * sp);       // ff only
    int* fail = (int*)(T2 + (ff ? 2 : 1) * sp * sp);
    double* fro = (double*)(fail + 16);
    double* fro_part = fro + 2;
    int* hflag = (int*)ctx->host_flags;
    auto fro_norm = [&](double* out) -> msp_status {
        k_fro2_part<<<kFroBlocks, 256, 0, ctx->stream>>>(M, sp * sp, fro_part);
        MSP_CHECK_LAUNCH(ctx);
        k_fro2_final<<<1, 32, 0, ctx->stream>>>(fro_part, fro);
        MSP_CHECK_LAUNCH(ctx);
        double h = 0.0;
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(&h, fro, 8, cudaMemcpyDeviceToHost, ctx->stream));
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        *out = std::sqrt(h);
        return MSP_OK;
    };
    double nu = 0.0;
    int scale_k = 0;            // M scaled by 4^scale_k, L^{-1} by 2^-scale_k
    if (fp32_data) {
        double fn = 0.0;
        MSP_TRY(fro_norm(&fn));
        nu = std::ldexp(1.0, -24) * fn;
        if (ff && fn > 0.0 && std::isfinite(fn)) scale_k = -(std::ilogb(fn) / 2);
    }
    for (int attempt = 0; attempt <= 4; ++attempt) {
        unsigned blocks = (unsigned)((sp * sp + 255) / 256);
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(fail, 0, sizeof(int), ctx->stream));
        if (ff) {
            k_copy_add_diag_ff<<<blocks, 256, 0, ctx->stream>>>(M, reinterpret_cast<float2*>(Mw), sp, nu,
                                                                std::ldexp(1.0, 2 * scale_k));
            MSP_CHECK_LAUNCH(ctx);
            MSP_CUDA_TRY(ctx, cudaMemsetAsync(Xff, 0, mat, ctx->stream));
            MSP_TRY(chol_inv_ff_graphed(ctx, reinterpret_cast<float2*>(Mw), Xff, reinterpret_cast<float2*>(T1),
                                        reinterpret_cast<float2*>(T2), sp, fail));
        } else {
            k_copy_add_diag<<<blocks, 256, 0, ctx->stream>>>(M, Mw, sp, nu);
            MSP_CHECK_LAUNCH(ctx);
            MSP_CUDA_TRY(ctx, cudaMemsetAsync(Linv64, 0, mat, ctx->stream));
            MSP_TRY(chol_inv(ctx, Mw, Linv64, T1, T2, sp, 0, sp, fail, 0));
        }
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hflag, fail, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        if (hflag[0] == 0) {
            if (ff) {
                k_ff_to_double<<<blocks, 256, 0, ctx->stream>>>(Xff, Linv64, sp * sp, std::ldexp(1.0, scale_k));
                MSP_CHECK_LAUNCH(ctx);
            }
            *shift_out = nu;
            *retries_out = attempt;
            return MSP_OK;
        }
        if (nu == 0.0) {
            double fn = 0.0;
            MSP_TRY(fro_norm(&fn));
            nu = (fp32_data ? std::ldexp(1.0, -24) : (double)s * std::ldexp(1.0, -52)) * fn;
            if (nu == 0.0) break;
        } else {
            nu *= 100.0;
        }
    }
    return msp_set_error(ctx, MSP_ENOTPD,
                         "matrix + shift is not positive definite after 4 retries (last shift %g)",
                         nu / 100.0);
}

}  // namespace

// Build W (symmetrised), M2, its shifted Cholesky inverse, and the working
// copies B, Bt. `Ct` is C~ (phi_rows x s_pad, dtype of the sketch).
msp_status msp_build_factor(msp_ctx* ctx, msp_factor_s* f, const void* Ct, int64_t phi_rows) {
    const int64_t sp = f->s_pad;
    const size_t ts = dtype_size(f->dtype);
    // W symmetrise + FP64 copy
    {
        dim3 blk(32, 32), grid((unsigned)((sp + 31) / 32), (unsigned)((sp + 31) / 32));
        if (f->dtype == MSP_F32)
            k_symmetrize<float><<<grid, blk, 0, ctx->stream>>>((float*)f->W, f->W64, sp);
        else
            k_symmetrize<double><<<grid, blk, 0, ctx->stream>>>((double*)f->W, f->W64, sp);
        MSP_CHECK_LAUNCH(ctx);
    }
    // M2 = Ct^T Ct + lam_t W: on the tensor cores (FP32 data), else split-K
    // partial Grams (upper tiles, mirrored) then the fixed-order FP64
    // combination
    if (f->dtype == MSP_F32 && ctx->gram_tc && msp_gram_tc_ok(sp)) {
        MSP_TRY(msp_gram_tc(ctx, (const float*)Ct, phi_rows, sp, f->s, sp, (const float*)f->W, f->lam_tilde, f->M2));
    } else {
        void* scr = nullptr;
        MSP_TRY(msp_scratch(ctx, (size_t)kGramSlices * sp * sp * 8, &scr));
        double* P = (double*)scr;
        const int nt = (int)(sp / 64);
        dim3 grid((unsigned)(nt * (nt + 1) / 2), kGramSlices);
        const unsigned fb = (unsigned)((sp * sp + 255) / 256);
        if (f->dtype == MSP_F32) {
            MSP_TRY(launch_gram_f32(ctx, (const float*)Ct, phi_rows, sp, sp, P));
            k_gram_finish<float><<<fb, 256, 0, ctx->stream>>>(P, (const float*)f->W, f->lam_tilde,
                                                               f->s, sp, f->M2);
        } else {
            k_gram<double><<<grid, 256, 0, ctx->stream>>>((const double*)Ct, phi_rows, sp, sp, P);
            MSP_CHECK_LAUNCH(ctx);
            k_gram_finish<double><<<fb, 256, 0, ctx->stream>>>(P, (const double*)f->W, f->lam_tilde,
                                                                f->s, sp, f->M2);
        }
        MSP_CHECK_LAUNCH(ctx);
    }
    MSP_TRY(factor_shifted(ctx, f->M2, f->s, sp, f->dtype == MSP_F32, f->Linv64, &f->shift, &f->retries));
    unsigned b2 = (unsigned)((sp * sp + 255) / 256);
    if (f->dtype == MSP_F32)
        k_cast_tri<float><<<b2, 256, 0, ctx->stream>>>(f->Linv64, (float*)f->B, (float*)f->Bt, sp);
    else
        k_cast_tri<double><<<b2, 256, 0, ctx->stream>>>(f->Linv64, (double*)f->B, (double*)f->Bt, sp);
    MSP_CHECK_LAUNCH(ctx);
    (void)ts;
    return MSP_OK;
}

// G64 = X^T X + diag I over the leading s columns of X (rows x ld FP32
// row-major, columns s..s_pad-1 zero): split-K partial Grams with compensated
// FP32 sums, combined in FP64 in a fixed order; pad block identity.
msp_status msp_gram64(msp_ctx* ctx, const float* X, int64_t rows, int64_t ld, int64_t s, int64_t sp,
                      double diag, double* G64) {
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, (size_t)kGramSlices * sp * sp * 8, &scr));
    double* P = (double*)scr;
    MSP_TRY(launch_gram_f32(ctx, X, rows, ld, sp, P));
    k_gram_finish<float><<<(unsigned)((sp * sp + 255) / 256), 256, 0, ctx->stream>>>(P, nullptr, diag, s, sp,
                                                                                      G64);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// Minv = M^{-1} (dense FP64) for an SPD s_pad x s_pad M64: FP64 Cholesky,
// shifted only on failure (the FP64-data rule), then L^{-T} L^{-1}.
msp_status msp_spd_inverse(msp_ctx* ctx, const double* M64, int64_t s, int64_t sp, double* Linv64,
                           double* Minv, double* shift, int* retries) {
    MSP_TRY(factor_shifted(ctx, M64, s, sp, false, Linv64, shift, retries));
    return dgemm(ctx, true, false, sp, sp, sp, 1.0, Linv64, sp, Linv64, sp, 0.0, Minv, sp);
}

// Dense inverse of G + diag I with G = X^T X. G is the Gram of the stored
// FP32 X itself, accumulated with compensated FP32 partial sums combined in
// FP64: PSD to about 2^-48 relative, so the FP64-data shift rule (unshifted
// first) applies. An FP32 copy of the inverse would perturb its products by
// about 2^-24 kappa(G), so the inverse stays FP64. G64 receives G + diag I.
msp_status msp_gram_inverse(msp_ctx* ctx, const float* X, int64_t rows, int64_t s, int64_t sp,
                            double diag, double* G64, double* Linv64, double* Minv,
                            double* shift, int* retries) {
    MSP_TRY(msp_gram64(ctx, X, rows, sp, s, sp, diag, G64));
    return msp_spd_inverse(ctx, G64, s, sp, Linv64, Minv, shift, retries);
}

namespace {

// Partial products P[slice][a][b] = sum_{k in slice} X[k][a] Y[k][b] for one
// 64 x 64 output tile (blockIdx.x over tile pairs, blockIdx.y the K slice),
// FP32 chunks of 16 accumulated with TwoSum into FP64 outputs. Columns of X
// at or beyond ncx (of Y: ncy) read as zero.
__global__ void __launch_bounds__(256, 4) k_gemm_tn(const float* __restrict__ X, int64_t ldx, int64_t ncx,
                                                   const float* __restrict__ Y, int64_t ldy, int64_t ncy,
                                                   int64_t K, int64_t ny_pad, int64_t nx_pad,
                                                   double* __restrict__ P) {
    __shared__ __align__(16) float As[16][64];
    __shared__ __align__(16) float Bs[16][64];
    const int nty = (int)(ny_pad / 64);
    const int ta = blockIdx.x / nty, tb = blockIdx.x % nty;
    const int64_t a0 = (int64_t)ta * 64, b0 = (int64_t)tb * 64;
    const int64_t kper = ((K + kGramSlices - 1) / kGramSlices + 15) / 16 * 16;
    const int64_t kbeg = (int64_t)blockIdx.y * kper;
    const int64_t kend = min(K, kbeg + kper);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { hi[i][j] = 0.f; lo[i][j] = 0.f; }
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e >> 6, cc = e & 63;
            const bool in = (k0 + kk) < kend;
            As[kk][cc] = (in && a0 + cc < ncx) ? X[(k0 + kk) * ldx + a0 + cc] : 0.f;
            Bs[kk][cc] = (in && b0 + cc < ncy) ? Y[(k0 + kk) * ldy + b0 + cc] : 0.f;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 va = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 vb = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[4] = {va.x, va.y, va.z, va.w}, bv[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_add(hi[i][j], lo[i][j], acc[i][j]);
        __syncthreads();
    }
    double* Ps = P + (int64_t)blockIdx.y * nx_pad * ny_pad;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            Ps[(a0 + ty * 4 + i) * ny_pad + b0 + tx * 4 + j] = (double)hi[i][j] + (double)lo[i][j];
}

__global__ void k_sum_slices_f32(const double* __restrict__ P, int64_t len, float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double v = 0.0;
#pragma unroll
    for (int sl = 0; sl < kGramSlices; ++sl) v += P[(int64_t)sl * len + e];
    out[e] = (float)v;
}

}  // namespace

// C = X^T Y (FP32 nx_pad x ny_pad row-major, nx_pad and ny_pad multiples of
// 64) for X: K x ncx (ldx) and Y: K x ncy (ldy), FP32 row-major; entries past
// ncx / ncy are zero. Compensated FP32 chunk sums combined in FP64, rounded
// once to FP32.
msp_status msp_gemm_tn(msp_ctx* ctx, const float* X, int64_t ldx, int64_t ncx, const float* Y, int64_t ldy,
                       int64_t ncy, int64_t K, int64_t nx_pad, int64_t ny_pad, float* C) {
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, (size_t)kGramSlices * nx_pad * ny_pad * 8, &scr));
    double* P = (double*)scr;
    dim3 grid((unsigned)((nx_pad / 64) * (ny_pad / 64)), kGramSlices);
    k_gemm_tn<<<grid, 256, 0, ctx->stream>>>(X, ldx, ncx, Y, ldy, ncy, K, ny_pad, nx_pad, P);
    MSP_CHECK_LAUNCH(ctx);
    const int64_t len = nx_pad * ny_pad;
    k_sum_slices_f32<<<(unsigned)((len + 255) / 256), 256, 0, ctx->stream>>>(P, len, C);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

extern "C" msp_status msp_set_factor_float_float(msp_ctx* ctx, int on) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    ctx->factor_ff = on != 0;
    return MSP_OK;
}

void msp_fac_graph_release(msp_ctx* ctx) {
    if (ctx->fac_exec) cudaGraphExecDestroy(ctx->fac_exec);
    if (ctx->fac_graph) cudaGraphDestroy(ctx->fac_graph);
    ctx->fac_exec = nullptr;
    ctx->fac_graph = nullptr;
    ctx->fac_key_len = 0;
    ctx->fac_kernels = 0;
}
