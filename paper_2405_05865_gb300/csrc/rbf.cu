// RBF kernel matrices and the adjoint of their length scale, on sm_103a.
//
// Coordinates are carried as exact FP32 pairs p = hi + lo, so a coordinate
// difference (hi_i - hi_j) + (lo_i - lo_j) is accurate to a few FP32 ulps of
// the difference itself (not of the coordinates): d_ij^2 keeps ~1e-7 relative
// accuracy even for close pairs.
//
// k_rbf_kernel   K_ij = exp(-|p_i - p_j|^2 / (2 ell^2)) in FP32 (kernel ridge
//                regression systems, Section 3); 64 x 64 output tiles with
//                both point blocks in shared memory.
// k_rbf_grad_ell out = -sum_ij a_i (dK_ij/d ell) x_j with
//                dK_ij/d ell = K_ij d_ij^2 / ell^3 recomputed per pair, so
//                dK is never formed. Each warp owns a row i; the points and
//                x_j (split into an exact FP32 pair x_hi + x_lo) are staged
//                per chunk in shared memory; per-lane sums are compensated
//                (TwoSum) in FP32 and combined in FP64; a_i multiplies the
//                FP64 row total; the last block sums the block totals in a
//                fixed order.
#include "msp_internal.cuh"

#include <cmath>
#include <mutex>

namespace {

constexpr int kRbfChunk = 1024;

struct PtHL {
    float4 hi, lo;
};

__device__ inline PtHL load_point(const double* __restrict__ P, int64_t i, int dim) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < dim; ++d) {
        const double v = P[i * dim + d];
        h[d] = (float)v;
        l[d] = (float)(v - (double)h[d]);
    }
    return {make_float4(h[0], h[1], h[2], h[3]), make_float4(l[0], l[1], l[2], l[3])};
}

__device__ inline float sqdist(const PtHL& a, const PtHL& b) {
    const float dx = (a.hi.x - b.hi.x) + (a.lo.x - b.lo.x);
    const float dy = (a.hi.y - b.hi.y) + (a.lo.y - b.lo.y);
    const float dz = (a.hi.z - b.hi.z) + (a.lo.z - b.lo.z);
    const float dw = (a.hi.w - b.hi.w) + (a.lo.w - b.lo.w);
    return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, dw * dw)));
}

__device__ inline PtHL zero_point() {
    return {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
}

__global__ void __launch_bounds__(256) k_rbf_kernel(const double* __restrict__ P, int64_t n, int dim,
                                                   float inv2l2, float* __restrict__ K, int64_t ldk) {
    __shared__ PtHL pi[64], pj[64];
    const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
    if (threadIdx.x < 64) {
        pi[threadIdx.x] = (i0 + threadIdx.x < n) ? load_point(P, i0 + threadIdx.x, dim) : zero_point();
    } else if (threadIdx.x < 128) {
        const int t = threadIdx.x - 64;
        pj[t] = (j0 + t < n) ? load_point(P, j0 + t, dim) : zero_point();
    }
    __syncthreads();
    const int tj = threadIdx.x & 63;
    for (int ti = threadIdx.x >> 6; ti < 64; ti += 4) {
        const int64_t i = i0 + ti, j = j0 + tj;
        if (i < n && j < n) K[i * ldk + j] = expf(-sqdist(pi[ti], pj[tj]) * inv2l2);
    }
}

__device__ inline void two_sum_acc(float& s, float& c, float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

__global__ void __launch_bounds__(256) k_rbf_grad_ell(const double* __restrict__ P, int64_t n, int dim,
                                                     float inv2l2, const double* __restrict__ a,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ part,
                                                     unsigned int* counter, double* out,
                                                     double scale) {
    __shared__ PtHL pts[kRbfChunk];
    __shared__ float xh[kRbfChunk], xl[kRbfChunk];
    __shared__ double red[8];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 8 + w;
    const PtHL pi = (i < n) ? load_point(P, i, dim) : zero_point();
    float s = 0.f, c = 0.f;
    double row = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kRbfChunk) {
        const int len = (int)min((int64_t)kRbfChunk, n - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < len; t += blockDim.x) {
            pts[t] = load_point(P, j0 + t, dim);
            const double xv = x[j0 + t];
            const float hi = (float)xv;
            xh[t] = hi;
            xl[t] = (float)(xv - (double)hi);
        }
        __syncthreads();
        if (i < n) {
            for (int t = lane; t < len; t += 32) {
                const float d2 = sqdist(pi, pts[t]);
                const float term = expf(-d2 * inv2l2) * d2;       // K_ij d_ij^2
                const float p = term * xh[t];
                const float e = fmaf(term, xh[t], -p);            // exact product error
                two_sum_acc(s, c, p);
                c += fmaf(term, xl[t], e);
            }
        }
        // fold the chunk into FP64 so the FP32 running sum stays short
        row += (double)s + (double)c;
        s = 0.f;
        c = 0.f;
    }
    row = msp::warp_sum(row);
    double contrib = (lane == 0 && i < n) ? a[i] * row : 0.0;
    if (lane == 0) red[w] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < 8; ++k) tot += red[k];
        part[blockIdx.x] = tot;
        __threadfence();
        const unsigned int tk = atomicAdd(counter, 1u);
        am_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    __threadfence();
    double all = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) all += __ldcg(&part[b]);
    *counter = 0;
    *out = -all * scale;
}

// ---------------------------------------------------- no-allocation variant
//
// Scratch of msp_rbf_grad_ell_static: word 0 holds the last-block counter,
// the FP64 block partials start at element 32 (256 bytes in). The grid has
// one block per 8 points, so n is limited to 8 * kStaticMaxBlocks. Every GPU
// that loads the library holds this array (about 512 KiB) until exit.
constexpr int64_t kStaticMaxBlocks = 65536;
constexpr int64_t kStaticMaxN = 8 * kStaticMaxBlocks;
static __device__ __align__(256) double g_rbf_grad_static[32 + kStaticMaxBlocks];

std::mutex g_static_mu;
double* g_static_ptr[64] = {};   // device address of the array, per device

}  // namespace

extern "C" {

msp_status msp_rbf_grad_ell_static(const double* points, int64_t n, int dim, double ell,
                                   const double* a, const double* x, double* out, void* stream) {
    if (!points || !a || !x || !out || n < 1 || dim < 1 || dim > 4 || !(ell > 0.0))
        return msp_set_error(nullptr, MSP_EINVAL,
                             "rbf_grad_ell_static: need n >= 1, 1 <= dim <= 4, ell > 0, non-NULL arrays");
    if (n > kStaticMaxN)
        return msp_set_error(nullptr, MSP_EINVAL,
                             "rbf_grad_ell_static: n = %lld exceeds the static scratch limit n <= %lld",
                             (long long)n, (long long)kStaticMaxN);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return msp_set_error(nullptr, MSP_ECUDA, "rbf_grad_ell_static: no current CUDA device");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (st) {
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess || sdev != dev) {
            cudaGetLastError();
            return msp_set_error(nullptr, MSP_EINVAL,
                                 "rbf_grad_ell_static: the stream does not belong to the current device %d", dev);
        }
    }
    double* scratch = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // name of the array is not a device address
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_rbf_grad_static);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return msp_set_error(nullptr, MSP_ECUDA, "rbf_grad_ell_static: cudaGetSymbolAddress: %s",
                                     cudaGetErrorString(e));
            }
            g_static_ptr[dev] = (double*)p;
        }
        scratch = g_static_ptr[dev];
    }
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    // the counter must start at zero (the array keeps the last call's contents)
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return msp_set_error(nullptr, MSP_ECUDA, "rbf_grad_ell_static: %s", cudaGetErrorString(e));
    }
    const unsigned blocks = (unsigned)((n + 7) / 8);
    k_rbf_grad_ell<<<blocks, 256, 0, st>>>(points, n, dim, (float)(1.0 / (2.0 * ell * ell)), a, x,
                                           scratch + 32, counter, out, 1.0 / (ell * ell * ell));
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return msp_set_error(nullptr, MSP_ECUDA, "rbf_grad_ell_static: launch: %s", cudaGetErrorString(e));
    return MSP_OK;
}

msp_status msp_rbf_kernel(msp_ctx* ctx, const double* points, int64_t n, int dim, double ell,
                          float* K, int64_t ldk) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!points || !K || n < 1 || ldk < n || dim < 1 || dim > 4 || !(ell > 0.0))
        return msp_set_error(ctx, MSP_EINVAL, "rbf_kernel: need n >= 1, 1 <= dim <= 4, ell > 0, ldk >= n");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ctx->device) cudaSetDevice(ctx->device);
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64));
    k_rbf_kernel<<<grid, 256, 0, ctx->stream>>>(points, n, dim, (float)(1.0 / (2.0 * ell * ell)), K, ldk);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_rbf_grad_ell(msp_ctx* ctx, const double* points, int64_t n, int dim, double ell,
                            const double* a, const double* x, double* out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!points || !a || !x || !out || n < 1 || dim < 1 || dim > 4 || !(ell > 0.0))
        return msp_set_error(ctx, MSP_EINVAL, "rbf_grad_ell: need n >= 1, 1 <= dim <= 4, ell > 0");
    msp::DeviceGuard guard(ctx->device);
    const unsigned blocks = (unsigned)((n + 7) / 8);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, (size_t)blocks * 8 + 256, &scr));
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    k_rbf_grad_ell<<<blocks, 256, 0, ctx->stream>>>(points, n, dim, (float)(1.0 / (2.0 * ell * ell)), a,
                                                    x, (double*)scr, &ctl->last_block_counter, out,
                                                    1.0 / (ell * ell * ell));
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

}  // extern "C"
