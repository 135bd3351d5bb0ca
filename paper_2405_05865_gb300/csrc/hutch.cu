// Schatten-1 norm of a PSD matrix by Hutchinson's estimator on sm_103a.
//
// For PSD A, |A|_1 = tr(A) (the p = 1 case of the norm estimators of
// Section 3.2); the estimate is (1/m) sum_j q_j, q_j = g_j^T A g_j, with
// Rademacher probes g_j drawn from the counter-based generator
// (row i of probe j is negative iff the top bit of
//  draw(seed, 7 + 2 (j / 256), i, j mod 256) is set).
//
// A is read once, as the packed upper 128 x 128 tiles (symv.cu layout):
//   q_j = sum_{I <= J} (2 - [I == J]) g_{I,j}^T A_IJ g_{J,j}.
// k_hutch_tile: one block per tile; the tile is staged transposed in shared
// memory, then for each chunk of 64 probes T = A_IJ G_J (128 x 64) is formed
// with an 8 x 4 register tile per thread and contracted with G_I; the
// per-tile partials (FP32, 128-term sums) are written per (tile, probe).
// k_hutch_reduce: q_j = sum_tiles w_tile part[tile][j] in FP64, fixed order.
#include "msp_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kT = 128;        // tile side (packed layout)
constexpr int kPC = 64;        // probes per chunk
constexpr int kAP = kT + 4;    // padded row length of the transposed tile
constexpr int kGP = kPC + 4;   // padded row length of the probe chunks
constexpr size_t kHutchSmem = (size_t)(kT * kAP + 2 * kT * kGP + 16 * kPC) * sizeof(float);

__global__ void k_probes(int64_t n, int64_t n_pad, int m, uint64_t seed, float* __restrict__ G) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pad * m) return;
    const int64_t i = e / m;
    const int j = (int)(e % m);
    float v = 0.f;
    if (i < n) {
        const uint64_t u = msp::draw(seed, (uint32_t)(7 + 2 * (j / 256)), (uint64_t)i, (uint32_t)(j % 256));
        v = (u >> 63) ? -1.f : 1.f;
    }
    G[e] = v;
}

__device__ inline void tile_coords_h(int t, int nt, int& I, int& J) {
    // FP32 estimate (the FP64 pipe is scarce on this part), then exact
    // integer correction
    const float a = 2.0f * nt + 1.0f;
    int i = (int)((a - sqrtf(fmaxf(a * a - 8.0f * t, 0.0f))) * 0.5f);
    if (i < 0) i = 0;
    if (i > nt - 1) i = nt - 1;
    while (i > 0 && (long long)i * nt - (long long)i * (i - 1) / 2 > t) --i;
    while (i + 1 < nt && (long long)(i + 1) * nt - (long long)(i + 1) * i / 2 <= t) ++i;
    I = i;
    J = i + (t - (int)((long long)i * nt - (long long)i * (i - 1) / 2));
}

__global__ void __launch_bounds__(256, 1) k_hutch_tile(const float* __restrict__ packed, int nt,
                                                      const float* __restrict__ G, int m,
                                                      float* __restrict__ part) {
    extern __shared__ __align__(16) float hs[];
    float* At = hs;                          // At[c][r] = A_IJ[r][c], row length kAP
    float* Gj = At + kT * kAP;               // Gj[c][j]: probe chunk rows of block J
    float* Gi = Gj + kT * kGP;               // Gi[r][j]: probe chunk rows of block I
    float* red = Gi + kT * kGP;              // 16 x 64
    const int t = blockIdx.x;
    int I, J;
    tile_coords_h(t, nt, I, J);
    const float* tile = packed + (size_t)t * kT * kT;
    for (int e = threadIdx.x; e < kT * kT / 4; e += blockDim.x) {
        const int r = e / (kT / 4), c4 = (e % (kT / 4)) * 4;
        const float4 v = __ldcs(reinterpret_cast<const float4*>(tile) + e);
        At[(c4 + 0) * kAP + r] = v.x;
        At[(c4 + 1) * kAP + r] = v.y;
        At[(c4 + 2) * kAP + r] = v.z;
        At[(c4 + 3) * kAP + r] = v.w;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // probes tx*4.., rows ty*8..
    for (int pc = 0; pc < m; pc += kPC) {
        __syncthreads();
        for (int e = threadIdx.x; e < kT * kPC / 4; e += blockDim.x) {
            const int r = e / (kPC / 4), j4 = (e % (kPC / 4)) * 4;
            const float4 gj = *reinterpret_cast<const float4*>(G + ((int64_t)J * kT + r) * m + pc + j4);
            const float4 gi = *reinterpret_cast<const float4*>(G + ((int64_t)I * kT + r) * m + pc + j4);
            *reinterpret_cast<float4*>(Gj + r * kGP + j4) = gj;
            *reinterpret_cast<float4*>(Gi + r * kGP + j4) = gi;
        }
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
        for (int c = 0; c < kT; ++c) {
            const float4 a0 = *reinterpret_cast<const float4*>(At + c * kAP + ty * 8);
            const float4 a1 = *reinterpret_cast<const float4*>(At + c * kAP + ty * 8 + 4);
            const float4 g = *reinterpret_cast<const float4*>(Gj + c * kGP + tx * 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], gv[b], acc[a][b]);
        }
        // contract with G_I over this thread's 8 rows, then over the 16 row groups
        float q[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float4 gi = *reinterpret_cast<const float4*>(Gi + (ty * 8 + a) * kGP + tx * 4);
            q[0] = fmaf(gi.x, acc[a][0], q[0]);
            q[1] = fmaf(gi.y, acc[a][1], q[1]);
            q[2] = fmaf(gi.z, acc[a][2], q[2]);
            q[3] = fmaf(gi.w, acc[a][3], q[3]);
        }
        *reinterpret_cast<float4*>(red + ty * kPC + tx * 4) = make_float4(q[0], q[1], q[2], q[3]);
        __syncthreads();
        if (threadIdx.x < kPC) {
            float v = 0.f;
#pragma unroll
            for (int g = 0; g < 16; ++g) v += red[g * kPC + threadIdx.x];
            part[(size_t)t * m + pc + threadIdx.x] = v;
        }
    }
}

// q[j] = sum_t w_t part[t][j] (w = 1 on the diagonal tiles, 2 off it), FP64,
// one block per probe, fixed order.
__global__ void k_hutch_reduce(const float* __restrict__ part, int ntiles, int nt, int m,
                               double* __restrict__ q) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    double v = 0.0;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int I, J;
        tile_coords_h(t, nt, I, J);
        v += (I == J ? 1.0 : 2.0) * (double)part[(size_t)t * m + j];
    }
    v = msp::warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        q[j] = s;
    }
}

// mean and standard error of q (single block, fixed order)
__global__ void k_mean_se(const double* __restrict__ q, int m, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) s += q[j];
    s = msp::warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double mean = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mean += red[w];
    mean /= m;
    __syncthreads();
    double d = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) d += (q[j] - mean) * (q[j] - mean);
    d = msp::warp_sum(d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ss = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ss += red[w];
        out[0] = mean;
        out[1] = m > 1 ? sqrt(ss / (m - 1) / m) : 0.0;
    }
}

msp_status hutch_impl(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda, int64_t m,
                      uint64_t seed, double* q_dev, double* ms_dev) {
    if (dt != MSP_F32)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: A must be FP32");
    if (n < 1 || lda < n || m < kPC || m % kPC != 0 || m > 4096)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: need lda >= n >= 1 and probes a multiple of %d in [%d, 4096]",
                             kPC, kPC);
    const int64_t nt = (n + kT - 1) / kT, n_pad = nt * kT;
    const int64_t ntiles = msp_packed_tiles(n);
    const size_t b_pack = round_up(ntiles * kT * kT * 4, 256);
    const size_t b_g = round_up(n_pad * m * 4, 256);
    const size_t b_part = round_up(ntiles * m * 4, 256);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, b_pack + b_g + b_part, &scr));
    char* c = (char*)scr;
    float* packed = (float*)c; c += b_pack;
    float* G = (float*)c; c += b_g;
    float* part = (float*)c;
    MSP_TRY(msp_pack_upper(ctx, (const float*)A, lda, n, packed));
    k_probes<<<(unsigned)((n_pad * m + 255) / 256), 256, 0, ctx->stream>>>(n, n_pad, (int)m, seed, G);
    MSP_CHECK_LAUNCH(ctx);
    static bool attr = false;
    if (!attr) {
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hutch_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kHutchSmem));
        attr = true;
    }
    k_hutch_tile<<<(unsigned)ntiles, 256, kHutchSmem, ctx->stream>>>(packed, (int)nt, G, (int)m, part);
    MSP_CHECK_LAUNCH(ctx);
    k_hutch_reduce<<<(unsigned)m, 256, 0, ctx->stream>>>(part, (int)ntiles, (int)nt, (int)m, q_dev);
    MSP_CHECK_LAUNCH(ctx);
    if (ms_dev) {
        k_mean_se<<<1, 256, 0, ctx->stream>>>(q_dev, (int)m, ms_dev);
        MSP_CHECK_LAUNCH(ctx);
    }
    return MSP_OK;
}

}  // namespace

extern "C" {

msp_status msp_hutchinson(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda,
                          int64_t probes, uint64_t seed, double* q) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !q) return msp_set_error(ctx, MSP_EINVAL, "hutchinson: NULL argument");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ctx->device) cudaSetDevice(ctx->device);
    return hutch_impl(ctx, A, dtype, n, lda, probes, seed, q, nullptr);
}

msp_status msp_schatten(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda, double p,
                        int64_t probes, uint64_t seed, double* norm, double* norm_pow, double* std_err) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A) return msp_set_error(ctx, MSP_EINVAL, "schatten: NULL A");
    if (p != 1.0)
        return msp_set_error(ctx, MSP_EINVAL,
                             "schatten: only p = 1 (PSD A, |A|_1 = tr A) is implemented; p = %g needs "
                             "shifted MSP solves", p);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ctx->device) cudaSetDevice(ctx->device);
    double* buf = nullptr;
    MSP_TRY(msp_alloc(ctx, (void**)&buf, (size_t)(probes + 2) * 8));
    msp_status st = hutch_impl(ctx, A, dtype, n, lda, probes, seed, buf, buf + probes);
    double* h = (double*)ctx->host_flags + 16;
    if (st == MSP_OK) {
        cudaError_t e = cudaMemcpyAsync(h, buf + probes, 16, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = msp_set_error(ctx, MSP_ECUDA, "schatten: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(buf, ctx->stream);
    if (st != MSP_OK) return st;
    if (norm) *norm = h[0];
    if (norm_pow) *norm_pow = h[0];
    if (std_err) *std_err = h[1];
    return MSP_OK;
}

}  // extern "C"
