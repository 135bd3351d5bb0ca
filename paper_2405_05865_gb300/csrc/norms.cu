// A certified lower bound of |A|_2 for symmetric PSD A, used by the
// backward-error stopping rule |r| <= tol ((L + lambda) |x| + |b|):
//   L = max( max_i |A e_i|_2 ,  1^T A 1 / n ),
// both terms at most |A|_2 (a column of A is A e_i; the second is the Rayleigh
// quotient of the all-ones vector). One pass over A.
//
// k_row_stats  one warp per row: the row is summed in chunks of 64 entries
//              per lane in FP32 (sum, sum of |.|, sum of squares), chunk
//              results combined in FP64, with the rounding bound of every
//              FP32 chunk kept beside it (the FP64 pipe of this part is 1/64
//              of the FP32 rate: with chunks of 16 the FP64 conversions and
//              sums alone kept it ~80% busy and held the pass to ~4 TB/s).
// k_norm_lb    one block: max of the row squares and the FP64 sum of the row
//              sums in a fixed order, each lowered by its rounding bound, so
//              the result stays at most |A|_2.
#include "msp_internal.cuh"

namespace {

// FP32 chunk of kChunk terms: |fl(sum) - sum| <= (kChunk - 1) u sum|t|
// (recursive summation, u = 2^-24); the exact sum of squares (positive terms)
// is at least (1 - (kChunk + 3) u) of the computed one, FP32 rounding of FP64
// entries included.
constexpr int kChunk = 64;
constexpr double kU32 = 5.9604644775390625e-8;

// The statistics of one row, by one warp.
template <typename T>
__device__ __forceinline__ void row_stats_one(const T* __restrict__ row, int64_t n, int lane,
                                              double* rowsum, double* rowerr, double* rowsq) {
    double s = 0.0, e = 0.0, q = 0.0;
    int64_t j = 0;
    if constexpr (sizeof(T) == 4) {
        // 16-byte loads, four per lane in flight; a chunk is four such
        // rounds (64 entries per lane)
        static_assert(kChunk == 64, "the vector path sums 4 x 4 float4 per chunk");
        if ((((uintptr_t)row) & 15) == 0) {
            const int64_t n4 = n & ~(int64_t)127;
            while (j < n4) {
                float cs = 0.f, ca = 0.f, cq = 0.f;
                for (int round = 0; round < 4 && j < n4; ++round, j += 4 * 128) {
                    float4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = (j + u * 128 < n4) ? __ldcs(reinterpret_cast<const float4*>(row + j + u * 128) + lane)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float w4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            cs += w4[c];
                            ca += fabsf(w4[c]);
                            cq = fmaf(w4[c], w4[c], cq);
                        }
                    }
                }
                s += (double)cs;
                e += (double)ca;
                q += (double)cq;
            }
            j = n4;
        }
    }
    j += lane;
    while (j < n) {
        float cs = 0.f, ca = 0.f, cq = 0.f;
#pragma unroll 4
        for (int k = 0; k < kChunk && j < n; ++k, j += 32) {
            const float v = (float)__ldcs(row + j);
            cs += v;
            ca += fabsf(v);
            cq = fmaf(v, v, cq);
        }
        s += (double)cs;
        e += (double)ca;
        q += (double)cq;
    }
    s = msp::warp_sum(s);
    e = msp::warp_sum(e);
    q = msp::warp_sum(q);
    if (lane == 0) {
        *rowsum = s;
        // chunk summation ((kChunk - 1) u) plus, for FP64 input, the
        // rounding of each entry to FP32 (u)
        *rowerr = (kChunk + 1) * kU32 * e * (1.0 + 1e-6);
        *rowsq = q;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_stats(const T* __restrict__ A, int64_t n, int64_t lda,
                                                  double* __restrict__ rowsum, double* __restrict__ rowerr,
                                                  double* __restrict__ rowsq) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * 8)
        row_stats_one<T>(A + i * lda, n, lane, rowsum + i, rowerr + i, rowsq + i);
}

__global__ void __launch_bounds__(1024) k_norm_lb(const double* __restrict__ rowsum,
                                                 const double* __restrict__ rowerr,
                                                 const double* __restrict__ rowsq, int64_t n,
                                                 double* out) {
    __shared__ double ssum[32], serr[32], smax[32];
    double s = 0.0, e = 0.0, m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s += rowsum[i];
        e += rowerr[i];
        m = fmax(m, rowsq[i]);
    }
    s = msp::warp_sum(s);
    e = msp::warp_sum(e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ssum[w] = s;
        serr[w] = e;
        smax[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, te = 0.0, tm = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            ts += ssum[k];
            te += serr[k];
            tm = fmax(tm, smax[k]);
        }
        // FP64 combination error (n^2 / kChunk chunk terms) is far below the
        // FP32 chunk bound; 2e-6 covers it with room
        const double col = sqrt(tm * (1.0 - (kChunk + 3) * kU32) * (1.0 - 2e-6));
        const double ones = (ts - te * (1.0 + 2e-6) - 2e-6 * fabs(ts)) / (double)n;
        *out = fmax(col, ones);
    }
}

}  // namespace

msp_status msp_norm_lb_launch(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda,
                              double* work, double* out_dev) {
    const unsigned blocks = (unsigned)((n + 7) / 8);
    if (dt == MSP_F32)
        k_row_stats<float><<<blocks, 256, 0, ctx->stream>>>((const float*)A, n, lda, work, work + n,
                                                           work + 2 * n);
    else
        k_row_stats<double><<<blocks, 256, 0, ctx->stream>>>((const double*)A, n, lda, work, work + n,
                                                            work + 2 * n);
    MSP_CHECK_LAUNCH(ctx);
    k_norm_lb<<<1, 1024, 0, ctx->stream>>>(work, work + n, work + 2 * n, n, out_dev);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_norm_lb_finish(msp_ctx* ctx, double* work, int64_t n, double* out_dev) {
    k_norm_lb<<<1, 1024, 0, ctx->stream>>>(work, work + n, work + 2 * n, n, out_dev);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

extern "C" msp_status msp_norm_lower_bound(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                                           int64_t lda, double* out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !out || n < 1 || lda < n || (dtype != MSP_F32 && dtype != MSP_F64))
        return msp_set_error(ctx, MSP_EINVAL, "norm_lower_bound: bad argument");
    msp::DeviceGuard g(ctx->device);
    void* mem = nullptr;
    MSP_TRY(msp_alloc(ctx, &mem, (size_t)(3 * n + 1) * 8));
    double* work = (double*)mem;
    msp_status st = msp_norm_lb_launch(ctx, A, dtype, n, lda, work, work + 3 * n);
    if (st == MSP_OK) {
        cudaError_t e = cudaMemcpyAsync(out, work + 3 * n, 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = msp_set_error(ctx, MSP_ECUDA, "norm_lower_bound: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(mem, ctx->stream);
    return st;
}
