// Schatten-1 norm of a PSD matrix by Hutchinson's estimator on sm_103a.
//
// For PSD A, |A|_1 = tr(A) (the p = 1 case of the norm estimators of
// Section 3.2); the estimate is (1/m) sum_j q_j, q_j = g_j^T A g_j, with
// Rademacher probes g_j drawn from the counter-based generator
// (row i of probe j is negative iff the top bit of
//  draw(seed, 7 + 2 (j / 256), i, j mod 256) is set).
//
// A is read once, upper 128 x 128 tiles only (A symmetric):
//   q_j = sum_{I <= J} (2 - [I == J]) g_{I,j}^T A_IJ g_{J,j}.
//
// Tensor-core path (k_hutch_tc; FP32 A with 16-byte aligned rows): a
// persistent kernel, one CTA per SM, walks a contiguous range of upper tiles
// in column order (so G_J changes rarely). Each tile arrives from the dense
// A in two 128 x 64 FP32 chunks by TMA; the threads split every entry
// exactly into three BF16 terms a = hi + mid + lo (8 significant bits each,
// the whole FP32 significand) written as K-major SWIZZLE_128B operand tiles;
// one thread issues tcgen05.mma kind::f16 (M = 128, N = probes of the group,
// K = 16) for the three terms against the BF16 probe block G_J (+-1, exact),
// accumulating T = A_IJ G_J in FP32 tensor memory (two accumulators: the
// epilogue of tile u reads one while the MMAs of tile u + 1 fill the other).
// The epilogue reads T by lanes (row r of the tile), multiplies by the sign
// of g_{I,j} at row r, sums over the 32 rows of a warp by a shuffle
// reduce-scatter (lane l ends with column l) and keeps per-probe FP64 sums
// over the CTA's tiles. k_hutch_tc_reduce adds the CTAs' sums in fixed order.
// Groups of at most 256 probes are separate passes over A.
//
// SIMT path (k_hutch_tile, any lda): A is packed into upper tiles first, one
// block per tile forms T = A_IJ G_J for chunks of 64 probes on the FP32 pipe.
#include "msp_internal.cuh"
#include "tc.cuh"

#include <mutex>

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

// ---------------------------------------------------- tensor-core path

constexpr int kTcThreads = 256;
constexpr int kTcTerms = 3;                                  // BF16 terms of each FP32 entry
constexpr uint32_t kTcA32Bytes = 128 * 64 * 4;               // one FP32 chunk (128 rows x 64)
constexpr uint32_t kTcTermBytes = 128 * 128;                 // one BF16 term tile (128 rows x 128 B)
constexpr uint32_t kTcOffSplit = 2 * kTcA32Bytes;            // two FP32 stages first
constexpr uint32_t kTcOffG = kTcOffSplit + 2 * kTcTerms * kTcTermBytes;
constexpr uint32_t kTcGBytes = 2 * 256 * 128;                // G_J: two K atoms of <= 256 probe rows
constexpr uint32_t kTcOffBar = kTcOffG + kTcGBytes;
constexpr size_t kTcSmem = kTcOffBar + 128 + 1024;           // barriers, flags, alignment slack
static_assert(kTcSmem <= 232448, "tensor-core Hutchinson kernel exceeds shared memory");

// Upper tile t in column order: t = J (J + 1) / 2 + I, 0 <= I <= J.
__device__ inline void tile_coords_col(int64_t t, int& I, int& J) {
    int j = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)j * (j + 1) / 2 > t) --j;
    while ((int64_t)(j + 1) * (j + 2) / 2 <= t) ++j;
    J = j;
    I = (int)(t - (int64_t)j * (j + 1) / 2);
}

// One FP32 value as three BF16 terms a = hi + mid + lo: each term is the
// round-to-nearest BF16 of what the previous terms leave, and each
// subtraction is exact in FP32 (the rounding error of a narrower rounding).
__device__ inline void split3(float a, float b, uint32_t& h, uint32_t& m, uint32_t& l) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
    const float ra = a - __low2float(h2), rb = b - __high2float(h2);
    const __nv_bfloat162 m2 = __floats2bfloat162_rn(ra, rb);
    const float sa = ra - __low2float(m2), sb = rb - __high2float(m2);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(sa, sb);
    h = *reinterpret_cast<const uint32_t*>(&h2);
    m = *reinterpret_cast<const uint32_t*>(&m2);
    l = *reinterpret_cast<const uint32_t*>(&l2);
}

// Sum over the 32 lanes of each of the 32 values v[0..31] (column c = index):
// a butterfly reduce-scatter after which lane l holds the sum of column l in
// v[0]. 31 shuffles.
__device__ inline float reduce_scatter32(float* v, int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = upper ? v[i] : v[i + w];
            const float keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// Probe block of one group as BF16 +-1, probe-major: Gt[j][i], j < m, i < n_pad
// (0 for i >= n).
__global__ void k_probes_bf16(int64_t n, int64_t n_pad, int m, uint64_t seed, __nv_bfloat16* __restrict__ Gt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pad * m) return;
    const int j = (int)(e / n_pad);
    const int64_t i = e % n_pad;
    float v = 0.f;
    if (i < n) {
        const uint64_t u = msp::draw(seed, (uint32_t)(7 + 2 * (j / 256)), (uint64_t)i, (uint32_t)(j % 256));
        v = (u >> 63) ? -1.f : 1.f;
    }
    Gt[e] = __float2bfloat16_rn(v);
}

// Sign bits: bits[i][w] bit b set iff probe 32 w + b is negative at row i.
// One warp per (row, word).
__global__ void k_probe_bits(int64_t n, int64_t n_pad, int m, uint64_t seed, uint32_t* __restrict__ bits) {
    const int words = m / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n_pad * words) return;
    const int64_t i = wid / words;
    const int j = (int)(wid % words) * 32 + lane;
    bool neg = false;
    if (i < n) {
        const uint64_t u = msp::draw(seed, (uint32_t)(7 + 2 * (j / 256)), (uint64_t)i, (uint32_t)(j % 256));
        neg = (u >> 63) != 0;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) bits[wid] = b;
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_hutch_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmG,
           const uint32_t* __restrict__ gbits, int words_per_row, int p0, int N, int64_t ntiles,
           double* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (msp::smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    float* sA32 = reinterpret_cast<float*>(sm);
    uint8_t* sSplit = sm + kTcOffSplit;
    uint8_t* sG = sm + kTcOffG;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTcOffBar);
    uint64_t* full = bar;          // [2] FP32 chunk landed
    uint64_t* mdone = bar + 2;     // [2] MMAs reading split buffer b complete
    uint64_t* afull = bar + 4;     // [2] accumulator a complete
    uint64_t* gfull = bar + 6;     // G_J landed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcOffBar + 64);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + kTcOffBar + 68);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int nchunks = (int)(2 * (t1 - t0));
    const uint32_t idesc = msp::tc::idesc_bf16_f32(128, N);

    if (tid == 0) {
        for (int i = 0; i < 7; ++i) msp::mbar_init(&bar[i], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        msp::tc::prefetch_tensormap(&tmA);
        msp::tc::prefetch_tensormap(&tmG);
    }
    if (warp == 0) msp::tc::tmem_alloc(tslot, 512);
    msp::tc::fence_before_sync();
    __syncthreads();
    msp::tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    auto issue_a = [&](int g) {   // FP32 chunk g into stage g & 1 (thread 0)
        int I, J;
        tile_coords_col(t0 + (g >> 1), I, J);
        msp::mbar_arrive_expect_tx(&full[g & 1], kTcA32Bytes);
        msp::tc::tma_load_2d(sA32 + (g & 1) * (128 * 64), &tmA, J * 128 + (g & 1) * 64, I * 128, &full[g & 1]);
    };
    if (tid == 0)
        for (int g = 0; g < 2 && g < nchunks; ++g) issue_a(g);

    const int quarter = warp & 3, half = warp >> 2;
    const int ncol32 = N / 64;               // 32-column chunks per half
    double qacc[4] = {0.0, 0.0, 0.0, 0.0};
    int jcur = -1, gloads = 0, a_issued = nchunks < 2 ? nchunks : 2, mma_last = -1;

    auto epilogue = [&](int u) -> bool {
        int I, J;
        tile_coords_col(t0 + u, I, J);
        // warp-uniform outcome: the tensor-memory loads below are warp-collective
        const bool okw = msp::mbar_wait_timed(&afull[u & 1], (u >> 1) & 1, err);
        if (!__all_sync(0xffffffffu, okw)) return false;
        msp::tc::fence_after_sync();
        const double wgt = (I == J) ? 1.0 : 2.0;
        const int row = quarter * 32 + lane;
        const uint32_t* rb = gbits + ((int64_t)I * 128 + row) * words_per_row + (p0 >> 5) + half * ncol32;
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((u & 1) * 256 + half * (N / 2));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < ncol32) {
                float v[32];
                msp::tc::tmem_ld32(tbase + c * 32, v);
                const uint32_t w = __ldg(rb + c);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(__float_as_uint(v[i]) ^ (((w >> i) & 1u) << 31));
                qacc[c] += wgt * (double)reduce_scatter32(v, lane);
            }
        }
        msp::tc::fence_before_sync();
        return true;
    };

    int g = 0;
    for (; g < nchunks; ++g) {
        const int s = g & 1, u = g >> 1, kc = g & 1;
        int I, J;
        tile_coords_col(t0 + u, I, J);
        bool ok = msp::mbar_wait_timed(&full[s], (g >> 1) & 1, err);
        if (ok && g >= 2) ok = msp::mbar_wait_timed(&mdone[s], ((g - 2) >> 1) & 1, err);
        if (!ok) *s_abort = 1;
        __syncthreads();
        if (*s_abort) break;
        // the FP32 chunk as three BF16 operand tiles (K-major, 128-byte swizzle)
        const float4* src = reinterpret_cast<const float4*>(sA32 + s * (128 * 64));
        uint8_t* dst = sSplit + s * (kTcTerms * kTcTermBytes);
#pragma unroll 4
        for (int q = 0; q < 8; ++q) {
            const int e = tid + kTcThreads * q;
            const int row = e >> 4, c4 = e & 15;
            const float4 v = src[e];
            uint32_t h0, m0, l0, h1, m1, l1;
            split3(v.x, v.y, h0, m0, l0);
            split3(v.z, v.w, h1, m1, l1);
            const uint32_t off = (uint32_t)row * 128u + ((uint32_t)((c4 >> 1) ^ (row & 7)) << 4) + ((c4 & 1) << 3);
            *reinterpret_cast<uint2*>(dst + off) = make_uint2(h0, h1);
            *reinterpret_cast<uint2*>(dst + kTcTermBytes + off) = make_uint2(m0, m1);
            *reinterpret_cast<uint2*>(dst + 2 * kTcTermBytes + off) = make_uint2(l0, l1);
        }
        msp::tc::fence_proxy_async();
        msp::tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            msp::tc::fence_after_sync();
            if (g + 2 < nchunks) {
                msp::tc::fence_proxy_async();
                issue_a(g + 2);
                a_issued = g + 3;
            }
            bool okg = true;
            if (J != jcur) {
                // every MMA reading the previous G_J must be complete
                if (mma_last >= 0) okg = msp::mbar_wait_timed(&mdone[mma_last & 1], (mma_last >> 1) & 1, err);
                if (okg) {
                    msp::mbar_arrive_expect_tx(gfull, 2u * (uint32_t)N * 128u);
                    msp::tc::tma_load_2d(sG, &tmG, J * 128, p0, gfull);
                    msp::tc::tma_load_2d(sG + N * 128, &tmG, J * 128 + 64, p0, gfull);
                    okg = msp::mbar_wait_timed(gfull, gloads & 1, err);
                    ++gloads;
                }
                jcur = J;
            }
            if (!okg) {
                *s_abort = 1;
            } else {
                msp::tc::fence_after_sync();
                const uint32_t dt = tmem + (uint32_t)((u & 1) * 256);
                const uint32_t a0 = msp::smem_u32(dst), b0 = msp::smem_u32(sG + kc * N * 128);
#pragma unroll
                for (int term = kTcTerms - 1; term >= 0; --term) {      // smallest term first
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = msp::tc::sdesc_kmajor_sw128(a0 + term * kTcTermBytes + ks * 32);
                        const uint64_t bd = msp::tc::sdesc_kmajor_sw128(b0 + ks * 32);
                        msp::tc::mma_bf16(dt, ad, bd, idesc, kc > 0 || term != kTcTerms - 1 || ks > 0);
                    }
                }
                msp::tc::mma_commit(&mdone[s]);
                if (kc == 1) msp::tc::mma_commit(&afull[u & 1]);
                mma_last = g;
            }
        }
        __syncwarp();
        // the previous tile's epilogue overlaps this tile's MMAs
        if (kc == 0 && u > 0 && !epilogue(u - 1)) *s_abort = 1;
    }
    __syncthreads();
    if (*s_abort == 0 && nchunks > 0 && !epilogue((nchunks >> 1) - 1)) *s_abort = 1;
    __syncthreads();
    if (*s_abort) {
        // bounded waits for this CTA's own copies and MMAs in flight, then free
        if (tid == 0) {
            for (int c = g; c < a_issued; ++c) msp::mbar_wait_timed(&full[c & 1], (c >> 1) & 1, err);
            if (mma_last >= 0) msp::mbar_wait_timed(&mdone[mma_last & 1], (mma_last >> 1) & 1, err);
        }
        __syncthreads();
    }
    // per-probe sums of the CTA: the four row quarters added in order
    double* red = reinterpret_cast<double*>(sm);    // 4 x 256, over the FP32 stages (all consumed)
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < ncol32) red[quarter * 256 + half * (N / 2) + c * 32 + lane] = qacc[c];
    __syncthreads();
    if (tid < N) {
        double v = 0.0;
        if (!*s_abort)
            for (int qq = 0; qq < 4; ++qq) v += red[qq * 256 + tid];
        part[(int64_t)blockIdx.x * N + tid] = v;
    }
    msp::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) msp::tc::tmem_dealloc(tmem, 512);
}

// q[p0 + j] = sum over CTAs of part[cta][j], fixed order; one warp per probe.
__global__ void k_hutch_tc_reduce(const double* __restrict__ part, int ctas, int N, int p0, double* __restrict__ q) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= N) return;
    double v = 0.0;
    for (int c = lane; c < ctas; c += 32) v += part[(int64_t)c * N + j];
    v = msp::warp_sum(v);
    if (lane == 0) q[p0 + j] = v;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 msp_tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

namespace {

// Tensor-core Hutchinson: q_j for j < m into q_dev (device FP64).
msp_status hutch_tc(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t m, uint64_t seed,
                    double* q_dev) {
    auto enc = msp_tensor_map_encoder();
    const int64_t nt = (n + 127) / 128, n_pad = nt * 128;
    const int64_t ntiles = nt * (nt + 1) / 2;
    const int grid = (int)std::min<int64_t>(ntiles, ctx->num_sms);
    const size_t b_g = round_up(n_pad * m * 2, 256);
    const size_t b_bits = round_up(n_pad * (m / 32) * 4, 256);
    const size_t b_part = round_up((int64_t)grid * 256 * 8, 256);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, b_g + b_bits + b_part, &scr));
    char* c = (char*)scr;
    __nv_bfloat16* Gt = (__nv_bfloat16*)c; c += b_g;
    uint32_t* bits = (uint32_t*)c; c += b_bits;
    double* part = (double*)c;
    k_probes_bf16<<<(unsigned)((n_pad * m + 255) / 256), 256, 0, ctx->stream>>>(n, n_pad, (int)m, seed, Gt);
    MSP_CHECK_LAUNCH(ctx);
    {
        const int64_t warps = n_pad * (m / 32);
        k_probe_bits<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, ctx->stream>>>(n, n_pad, (int)m, seed, bits);
        MSP_CHECK_LAUNCH(ctx);
    }
    CUtensorMap tmA;
    {
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
        const cuuint32_t box[2] = {64, 128};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box,
                               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return msp_set_error(ctx, MSP_ECUDA, "hutchinson: cuTensorMapEncodeTiled(A) failed (%d)", (int)r);
    }
    static bool attr = false;
    if (!attr) {
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hutch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kTcSmem));
        attr = true;
    }
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    for (int64_t p0 = 0; p0 < m; p0 += 256) {
        const int N = (int)std::min<int64_t>(256, m - p0);
        CUtensorMap tmG;
        const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)m};
        const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)N};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Gt, dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return msp_set_error(ctx, MSP_ECUDA, "hutchinson: cuTensorMapEncodeTiled(G) failed (%d)", (int)r);
        k_hutch_tc<<<grid, kTcThreads, kTcSmem, ctx->stream>>>(tmA, tmG, bits, (int)(m / 32), (int)p0, N, ntiles,
                                                               part, &ctl->error);
        MSP_CHECK_LAUNCH(ctx);
        k_hutch_tc_reduce<<<(unsigned)((N + 7) / 8), 256, 0, ctx->stream>>>(part, grid, N, (int)p0, q_dev);
        MSP_CHECK_LAUNCH(ctx);
    }
    return MSP_OK;
}

// The device-side wait status of the tensor-core path (ctl->error), read
// back after a stream synchronisation.
msp_status hutch_check(msp_ctx* ctx) {
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    int* h = (int*)ctx->host_flags;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(h, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (h[0] != 0)
        return msp_set_error(ctx, (msp_status)h[0], "hutchinson: a device-side wait gave up (status %d)", h[0]);
    return MSP_OK;
}

msp_status hutch_simt(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t m, uint64_t seed,
                      double* q_dev);

msp_status hutch_impl(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda, int64_t m,
                      uint64_t seed, double* q_dev, double* ms_dev) {
    if (dt != MSP_F32)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: A must be FP32");
    if (n < 1 || lda < n || m < kPC || m % kPC != 0 || m > 4096)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: need lda >= n >= 1 and probes a multiple of %d in [%d, 4096]",
                             kPC, kPC);
    // the device-side wait status of this call (read back by hutch_check)
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(&((CtlBlock*)ctx->ctl)->error, 0, sizeof(int), ctx->stream));
    if ((lda % 4) == 0 && ((uintptr_t)A & 15) == 0 && msp_tensor_map_encoder()) {
        MSP_TRY(hutch_tc(ctx, (const float*)A, n, lda, m, seed, q_dev));
    } else {
        MSP_TRY(hutch_simt(ctx, (const float*)A, n, lda, m, seed, q_dev));
    }
    if (ms_dev) {
        k_mean_se<<<1, 256, 0, ctx->stream>>>(q_dev, (int)m, ms_dev);
        MSP_CHECK_LAUNCH(ctx);
    }
    return MSP_OK;
}

// SIMT path: pack the upper tiles, then one block per tile on the FP32 pipe.
msp_status hutch_simt(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t m, uint64_t seed,
                      double* q_dev) {
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
    MSP_TRY(msp_pack_upper(ctx, A, lda, n, packed));
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
    MSP_TRY(hutch_impl(ctx, A, dtype, n, lda, probes, seed, q, nullptr));
    return hutch_check(ctx);
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
        if (e != cudaSuccess) st = msp_set_error(ctx, MSP_ECUDA, "schatten: %s", cudaGetErrorString(e));
        else st = hutch_check(ctx);   // synchronises the stream
    }
    cudaFreeAsync(buf, ctx->stream);
    if (st != MSP_OK) return st;
    if (norm) *norm = h[0];
    if (norm_pow) *norm_pow = h[0];
    if (std_err) *std_err = h[1];
    return MSP_OK;
}

}  // extern "C"
