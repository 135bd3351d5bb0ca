// A certified lower bound of |A|_2 for symmetric PSD A, used by the
// backward-error stopping rule |r| <= tol ((L + lambda) |x| + |b|):
//   L = max( max_i |A e_i|_2 ,  1^T A 1 / n ),
// both terms at most |A|_2 (a column of A is A e_i; the second is the Rayleigh
// quotient of the all-ones vector). One pass over A.
//
// k_row_stats  one warp per row: FP64 sums of a_ij and a_ij^2 over the row
//              (= column, A symmetric), lanes striding the row, fixed-order
//              warp reduction.
// k_norm_lb    one block: the maximum of the row squares and the FP64 sum of
//              the row sums in a fixed order.
#include "msp_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_row_stats(const T* __restrict__ A, int64_t n, int64_t lda,
                                                  double* __restrict__ rowsum, double* __restrict__ rowsq) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const T* row = A + i * lda;
    double s = 0.0, q = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        const double v = (double)__ldcs(row + j);
        s += v;
        q += v * v;
    }
    s = msp::warp_sum(s);
    q = msp::warp_sum(q);
    if (lane == 0) {
        rowsum[i] = s;
        rowsq[i] = q;
    }
}

__global__ void __launch_bounds__(1024) k_norm_lb(const double* __restrict__ rowsum,
                                                 const double* __restrict__ rowsq, int64_t n,
                                                 double* out) {
    __shared__ double ssum[32], smax[32];
    double s = 0.0, m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s += rowsum[i];
        m = fmax(m, rowsq[i]);
    }
    s = msp::warp_sum(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ssum[w] = s;
        smax[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            ts += ssum[k];
            tm = fmax(tm, smax[k]);
        }
        *out = fmax(sqrt(tm), ts / (double)n);
    }
}

}  // namespace

msp_status msp_norm_lb_launch(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda,
                              double* work, double* out_dev) {
    const unsigned blocks = (unsigned)((n + 7) / 8);
    if (dt == MSP_F32)
        k_row_stats<float><<<blocks, 256, 0, ctx->stream>>>((const float*)A, n, lda, work, work + n);
    else
        k_row_stats<double><<<blocks, 256, 0, ctx->stream>>>((const double*)A, n, lda, work, work + n);
    MSP_CHECK_LAUNCH(ctx);
    k_norm_lb<<<1, 1024, 0, ctx->stream>>>(work, work + n, n, out_dev);
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
    MSP_TRY(msp_alloc(ctx, &mem, (size_t)(2 * n + 1) * 8));
    double* work = (double*)mem;
    msp_status st = msp_norm_lb_launch(ctx, A, dtype, n, lda, work, work + 2 * n);
    if (st == MSP_OK) {
        cudaError_t e = cudaMemcpyAsync(out, work + 2 * n, 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = msp_set_error(ctx, MSP_ECUDA, "norm_lower_bound: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(mem, ctx->stream);
    return st;
}
