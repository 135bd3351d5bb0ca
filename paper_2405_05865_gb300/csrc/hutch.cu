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
// persistent kernel, one CTA per SM, walks a contiguous range of the lower
// tiles (J, I), I <= J, row block by row block. As A is symmetric,
// q_j = sum_J g_J^T U_J with U_J = sum_{I <= J} w_IJ A_JI G_I, w = 1 on the
// diagonal and 2 off it. Each tile arrives from the dense A by TMA in four
// 128 x 32 FP32 chunks, each with the matching 32 x m block of the 16-bit
// probes G_I (+-1, exact). Converter warps split every entry into 16-bit
// terms written as K-major SWIZZLE_64B operand tiles: by default two FP16
// terms of s w a (s a power of two from the largest diagonal entry, so for
// PSD A every |s w a| <= 2^15; hi + lo carry 22 significant bits), or three
// BF16 terms (8 bits each, the whole FP32 significand, exact) for matrices
// that leave the FP16 range. One thread issues tcgen05.mma kind::f16
// (M = 128, N = probes of the group, K = 16) per term, accumulating U_J in
// FP32 tensor memory over the whole row block. Warp roles: TMA producers of
// A and of G, the MMA issuer, eight converter warps, four epilogue warps;
// mbarriers connect a six-stage ring of FP32 chunks, three G slots and three
// split slots. At the end of a row block the epilogue reads U_J by lanes
// (row r of the block), multiplies by the sign of g_{J,j} at row r, sums
// over the 32 rows of a warp by a shuffle reduce-scatter (lane l ends with
// column l) and keeps per-probe FP64 sums; two accumulators let the next
// row block's MMAs overlap it. k_hutch_tc_reduce adds the CTAs' sums in
// fixed order (and undoes s, exactly). Groups of at most 256 probes are
// separate passes over A.
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

// warp roles: 0 TMA producer of A (and tensor-memory owner), 1 TMA
// producer of G, 2 MMA issuer, 3..10 converters (FP32 -> 16-bit terms),
// 11..14 epilogue (tensor-memory lane quarters 3, 0, 1, 2)
constexpr int kTcConvWarps = 8;
constexpr int kTcConvWarp0 = 3;
constexpr int kTcEpiWarp0 = kTcConvWarp0 + kTcConvWarps;
constexpr int kTcThreads = 32 * (kTcEpiWarp0 + 4);
constexpr int kTcK = 32;                                     // columns of A per chunk (64-byte BF16 rows)
constexpr int kTcAStages = 6;                                // FP32 chunks in flight per SM
constexpr int kTcGSlots = 3;                                 // G chunks
constexpr int kTcSSlots = 3;                                 // split-term tiles
constexpr uint32_t kTcA32Bytes = 128 * kTcK * 4;             // one FP32 chunk (128 rows x 32)
constexpr uint32_t kTcGBytes = 256 * kTcK * 2;               // one G chunk: <= 256 probe rows x 32 BF16
constexpr uint32_t kTcTermBytes = 128 * kTcK * 2;            // one BF16 term tile (128 rows x 64 B)
constexpr int kTcMaxTerms = 3;
constexpr uint32_t kTcOffG = kTcAStages * kTcA32Bytes;
constexpr uint32_t kTcOffSplit = kTcOffG + kTcGSlots * kTcGBytes;
constexpr uint32_t kTcOffBar = kTcOffSplit + kTcSSlots * kTcMaxTerms * kTcTermBytes;
constexpr int kTcBars = 2 * kTcAStages + 2 * kTcGSlots + 2 * kTcSSlots + 4;
constexpr size_t kTcSmem = kTcOffBar + 8 * kTcBars + 64 + 1024;   // barriers, flags, alignment slack
static_assert(kTcSmem <= 232448, "tensor-core Hutchinson kernel exceeds shared memory");

// Upper tile t in column order: t = J (J + 1) / 2 + I, 0 <= I <= J.
__device__ inline void tile_coords_col(int64_t t, int& I, int& J) {
    int j = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)j * (j + 1) / 2 > t) --j;
    while ((int64_t)(j + 1) * (j + 2) / 2 <= t) ++j;
    J = j;
    I = (int)(t - (int64_t)j * (j + 1) / 2);
}

// Walk of consecutive lower tiles in row-block order: (I, J) -> (I + 1, J),
// or (0, J + 1) after the diagonal. Integer only (the FP64 pipe of this part
// is too narrow for a square root per step).
struct TileWalk {
    int I, J;
    __device__ explicit TileWalk(int64_t t) { tile_coords_col(t, I, J); }
    __device__ void next() {
        if (++I > J) {
            ++J;
            I = 0;
        }
    }
    __device__ bool ends_row() const { return I == J; }
};

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

// Two FP16 terms x ~ hi + lo (11 + 11 significant bits: error <= 2^-22 |x|
// while x - hi is a normal FP16, else <= 2^-25); x must be below 65504.
__device__ inline void split2h(float a, float b, uint32_t& h, uint32_t& l) {
    const __half2 h2 = __floats2half2_rn(a, b);
    const __half2 l2 = __floats2half2_rn(a - __low2float(h2), b - __high2float(h2));
    h = *reinterpret_cast<const uint32_t*>(&h2);
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

// The probes as 16-bit +-1 (FP16 or BF16 bit patterns), probe-major:
// Gt[j][i], j < m, i < n_pad (0 for i >= n).
__global__ void k_probes_16(int64_t n, int64_t n_pad, int m, uint64_t seed, bool fp16, uint16_t* __restrict__ Gt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pad * m) return;
    const int j = (int)(e / n_pad);
    const int64_t i = e % n_pad;
    uint16_t v = 0;
    if (i < n) {
        const uint64_t u = msp::draw(seed, (uint32_t)(7 + 2 * (j / 256)), (uint64_t)i, (uint32_t)(j % 256));
        const uint16_t one = fp16 ? 0x3C00 : 0x3F80;
        v = (u >> 63) ? (uint16_t)(one | 0x8000) : one;
    }
    Gt[e] = v;
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

// MODE 3: three BF16 terms (exact). MODE 2: two FP16 terms of scale * w * a
// (scale a power of two from the largest diagonal entry, so that every
// |2 scale a_ij| <= 2^15 for PSD A; an entry beyond the FP16 range sets
// *ovf).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
k_hutch_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmG,
           const float* __restrict__ scale_dev,
           const uint32_t* __restrict__ gbits, int words_per_row, int p0, int N, int64_t ntiles,
           double* __restrict__ part, int* __restrict__ err, int* __restrict__ ovf) {
    constexpr int CPT = 128 / kTcK;          // chunks per tile
    constexpr int TERMS = MODE;
    constexpr int PER = (128 * kTcK / 4) / (32 * kTcConvWarps);   // float4 per converter thread
    static_assert(PER * 32 * kTcConvWarps == 128 * kTcK / 4, "converter threads must divide the chunk");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (msp::smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    float* sA32 = reinterpret_cast<float*>(sm);
    uint8_t* sG = sm + kTcOffG;
    uint8_t* sSplit = sm + kTcOffSplit;
    const uint32_t s_a32 = msp::smem_u32(sA32), s_split = msp::smem_u32(sSplit);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTcOffBar);
    uint64_t* afull = bar;                               // [A stages] FP32 chunk landed (TMA)
    uint64_t* aempty = afull + kTcAStages;               // [A stages] chunk split (converter warps)
    uint64_t* gfull = aempty + kTcAStages;               // [G slots] G chunk landed (TMA)
    uint64_t* gfree = gfull + kTcGSlots;                 // [G slots] its MMAs done (commit)
    uint64_t* sready = gfree + kTcGSlots;                // [split slots] terms written (converter warps)
    uint64_t* sfree = sready + kTcSSlots;                // [split slots] their MMAs done (commit)
    uint64_t* accf = sfree + kTcSSlots;                  // [2] accumulator complete (commit)
    uint64_t* acce = accf + 2;                           // [2] accumulator read (epilogue warps)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcOffBar + 8 * kTcBars);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + kTcOffBar + 8 * kTcBars + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int nchunks = (int)(CPT * (t1 - t0));

    if (tid == 0) {
        for (int i = 0; i < kTcAStages; ++i) {
            msp::mbar_init(&afull[i], 1);
            msp::mbar_init(&aempty[i], kTcConvWarps);
        }
        for (int i = 0; i < kTcGSlots; ++i) {
            msp::mbar_init(&gfull[i], 1);
            msp::mbar_init(&gfree[i], 1);
        }
        for (int i = 0; i < kTcSSlots; ++i) {
            msp::mbar_init(&sready[i], kTcConvWarps);
            msp::mbar_init(&sfree[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            msp::mbar_init(&accf[i], 1);
            msp::mbar_init(&acce[i], 4);
        }
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
    // a bounded wait of one role; on timeout every role stops at its next check
    auto wait = [&](uint64_t* b, int parity) -> bool {
        if (*s_abort) return false;
        if (!msp::mbar_wait_sleep(b, (uint32_t)(parity & 1), err)) {
            *s_abort = 1;
            return false;
        }
        return true;
    };

    int a_last[kTcAStages], g_last[kTcGSlots];   // producers: last chunk issued per stage / slot
    int mma_last = -1;
    double qacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < kTcAStages; ++i) a_last[i] = -1;
    for (int i = 0; i < kTcGSlots; ++i) g_last[i] = -1;

    if (warp == 0 || warp == 1) {
        // ---- producers (A and G each on its own warp, so that neither ring
        // waits for the other): chunk g covers columns I*128 + (g mod CPT)*32
        // .. +32 of the lower tile (J, I), with the matching 32 rows of every
        // probe.
        if (lane == 0) {
            TileWalk tw(t0);
            for (int g = 0; g < nchunks; ++g) {
                if (g > 0 && g % CPT == 0) tw.next();
                const int I = tw.I, J = tw.J;
                const int x = I * 128 + (g % CPT) * kTcK;
                if (warp == 0) {
                    const int a = g % kTcAStages;
                    if (g >= kTcAStages && !wait(&aempty[a], g / kTcAStages - 1)) break;
                    msp::mbar_arrive_expect_tx(&afull[a], kTcA32Bytes);
                    msp::tc::tma_load_2d(sA32 + a * (128 * kTcK), &tmA, x, J * 128, &afull[a]);
                    a_last[a] = g;
                } else {
                    const int r = g % kTcGSlots;
                    if (g >= kTcGSlots && !wait(&gfree[r], g / kTcGSlots - 1)) break;
                    msp::mbar_arrive_expect_tx(&gfull[r], (uint32_t)N * (kTcK * 2));
                    msp::tc::tma_load_2d(sG + r * kTcGBytes, &tmG, x, p0, &gfull[r]);
                    g_last[r] = g;
                }
            }
        }
    } else if (warp == 2) {
        // ---- MMA issuer: U_J (+)= w A_JI G_I over the row block's chunks
        if (lane == 0) {
            const uint32_t idesc = MODE == 2 ? msp::tc::idesc_f16_f32(128, N) : msp::tc::idesc_bf16_f32(128, N);
            int seg = -1, seg_J = -1;
            TileWalk tw(t0);
            for (int g = 0; g < nchunks; ++g) {
                const int u = g / CPT, kc = g % CPT, r = g % kTcGSlots, b = g % kTcSSlots;
                if (g > 0 && kc == 0) tw.next();
                const int J = tw.J;
                const bool first = (kc == 0 && J != seg_J);
                if (first) {
                    ++seg;
                    seg_J = J;
                    if (seg >= 2 && !wait(&acce[seg & 1], (seg >> 1) - 1)) break;
                }
                // the row block ends at its diagonal tile or with the range
                const bool last = (kc == CPT - 1 && (tw.ends_row() || t0 + u + 1 == t1));
                if (!wait(&gfull[r], g / kTcGSlots) || !wait(&sready[b], g / kTcSSlots)) break;
                msp::tc::fence_after_sync();
                const uint32_t dt = tmem + (uint32_t)((seg & 1) * 256);
                const uint32_t a0 = msp::smem_u32(sSplit + b * (kTcMaxTerms * kTcTermBytes));
                const uint32_t b0 = msp::smem_u32(sG + r * kTcGBytes);
#pragma unroll
                for (int term = TERMS - 1; term >= 0; --term) {      // smallest term first
#pragma unroll
                    for (int ks = 0; ks < kTcK / 16; ++ks) {
                        const uint64_t ad = msp::tc::sdesc_kmajor_sw64(a0 + term * kTcTermBytes + ks * 32);
                        const uint64_t bd = msp::tc::sdesc_kmajor_sw64(b0 + ks * 32);
                        msp::tc::mma_bf16(dt, ad, bd, idesc, !(first && term == TERMS - 1 && ks == 0));
                    }
                }
                msp::tc::mma_commit(&gfree[r]);
                msp::tc::mma_commit(&sfree[b]);
                if (last) msp::tc::mma_commit(&accf[seg & 1]);
                mma_last = g;
            }
        }
    } else if (warp < kTcEpiWarp0) {
        // ---- converters: w a (MODE 2: scale w a) as 16-bit operand terms
        // (K-major, 64-byte swizzle); w = 2 off the diagonal (the tile stands
        // for itself and its transpose), exact in every term
        const int ct = tid - 32 * kTcConvWarp0;
        const float scale = MODE == 2 ? __ldg(scale_dev) : 1.0f;
        TileWalk tw(t0);
        float4 cur[PER];
        for (int g = 0; g < nchunks; ++g) {
            const int a = g % kTcAStages, b = g % kTcSSlots;
            if (g > 0 && g % CPT == 0) tw.next();
            const int I = tw.I, J = tw.J;
            // warp-uniform decisions (the warp meets at __syncwarp below)
            if (!__all_sync(0xffffffffu, wait(&afull[a], g / kTcAStages))) break;
#pragma unroll
            for (int q = 0; q < PER; ++q)
                cur[q] = msp::lds128(s_a32 + (uint32_t)a * kTcA32Bytes + 16u * (uint32_t)(ct + 32 * kTcConvWarps * q));
            if (g >= kTcSSlots && !__all_sync(0xffffffffu, wait(&sfree[b], g / kTcSSlots - 1))) break;
            const float wgt = ((I == J) ? 1.0f : 2.0f) * scale;
            const uint32_t dst = s_split + (uint32_t)b * (kTcMaxTerms * kTcTermBytes);
            if constexpr (MODE == 2) {
                // the scaled entries must stay inside the FP16 range (PSD A)
                float mx = 0.f;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(cur[q].x), fabsf(cur[q].y)), fmaxf(fabsf(cur[q].z), fabsf(cur[q].w))));
                if (!(wgt * mx <= 65504.f)) atomicOr(ovf, 1);
            }
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int e = ct + 32 * kTcConvWarps * q;
                const int row = e >> 3, c4 = e & 7;
                const float4 v = cur[q];
                const uint32_t off =
                    (uint32_t)row * 64u + ((uint32_t)((c4 >> 1) ^ ((row >> 1) & 3)) << 4) + ((c4 & 1) << 3);
                uint32_t h0, m0, l0, h1, m1, l1;
                if constexpr (MODE == 3) {
                    split3(wgt * v.x, wgt * v.y, h0, m0, l0);
                    split3(wgt * v.z, wgt * v.w, h1, m1, l1);
                    msp::sts64(dst + 2 * kTcTermBytes + off, l0, l1);
                } else {
                    split2h(wgt * v.x, wgt * v.y, h0, m0);
                    split2h(wgt * v.z, wgt * v.w, h1, m1);
                }
                msp::sts64(dst + off, h0, h1);
                msp::sts64(dst + kTcTermBytes + off, m0, m1);
            }
            msp::tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                msp::mbar_arrive(&aempty[a]);
                msp::mbar_arrive(&sready[b]);
            }
        }
    } else {
        // ---- epilogue: at the end of each row block J of this CTA's range,
        // q_j += sum_r g_{J,j}[r] U_J[r][j] (lane l ends with column l of
        // each group of 32)
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        int seg = -1;
        int64_t t = t0;
        TileWalk tw(t0);
        while (t < t1) {
            const int J = tw.J;
            // this row block's tiles in the range: up to its diagonal
            while (!tw.ends_row() && t + 1 < t1) {
                tw.next();
                ++t;
            }
            ++t;
            tw.next();
            ++seg;
            if (!__all_sync(0xffffffffu, wait(&accf[seg & 1], seg >> 1))) break;
            msp::tc::fence_after_sync();
            const uint32_t* rb = gbits + ((int64_t)J * 128 + row) * words_per_row + (p0 >> 5);
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((seg & 1) * 256);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < N / 32) {
                    float v[32];
                    msp::tc::tmem_ld32(tbase + c * 32, v);
                    const uint32_t w = __ldg(rb + c);
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        v[i] = __uint_as_float(__float_as_uint(v[i]) ^ (((w >> i) & 1u) << 31));
                    qacc[c] += (double)reduce_scatter32(v, lane);
                }
            }
            msp::tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&acce[seg & 1]);
        }
    }
    __syncthreads();
    if (*s_abort) {
        // bounded waits for this CTA's own copies and MMAs in flight, then free
        if (warp == 0 && lane == 0)
            for (int i = 0; i < kTcAStages; ++i)
                if (a_last[i] >= 0) msp::mbar_wait_timed(&afull[i], (uint32_t)((a_last[i] / kTcAStages) & 1), err);
        if (warp == 1 && lane == 0)
            for (int i = 0; i < kTcGSlots; ++i)
                if (g_last[i] >= 0) msp::mbar_wait_timed(&gfull[i], (uint32_t)((g_last[i] / kTcGSlots) & 1), err);
        if (warp == 2 && lane == 0 && mma_last >= 0)
            msp::mbar_wait_timed(&gfree[mma_last % kTcGSlots], (uint32_t)((mma_last / kTcGSlots) & 1), err);
        __syncthreads();
    }
    // per-probe sums of the CTA: the four row quarters added in order
    double* red = reinterpret_cast<double*>(sm);    // 4 x 256 over the FP32 stages (consumed)
    if (warp >= kTcEpiWarp0) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < N / 32) red[(warp & 3) * 256 + c * 32 + lane] = qacc[c];
    }
    __syncthreads();
    if (tid < N) {
        double v = 0.0;
        if (!*s_abort)
            for (int qq = 0; qq < 4; ++qq) v += red[qq * 256 + tid];
        part[(int64_t)blockIdx.x * N + tid] = v;
    }
    msp::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        msp::tc::tmem_dealloc(tmem, 512);
    }
}

// q[p0 + j] = sum over CTAs of part[cta][j], fixed order; one warp per probe.
__global__ void k_hutch_tc_reduce(const double* __restrict__ part, int ctas, int N, int p0,
                                  const float* __restrict__ scale_dev, double* __restrict__ q) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= N) return;
    double v = 0.0;
    for (int c = lane; c < ctas; c += 32) v += part[(int64_t)c * N + j];
    v = msp::warp_sum(v);
    if (lane == 0) q[p0 + j] = scale_dev ? v / (double)__ldg(scale_dev) : v;   // a power of two: exact
}

// scale = 2^(14 - e) with 2^e >= max_i A_ii (one block; e from frexp), so
// |2 scale a_ij| <= 2^15 for every entry of a PSD A; 1 if A has no positive
// diagonal entry.
__global__ void k_diag_scale(const float* __restrict__ A, int64_t lda, int64_t n, float* __restrict__ scale) {
    __shared__ float red[32];
    float mx = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, A[i * lda + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        int e = 0;
        if (m > 0.f && isfinite(m)) frexpf(m, &e);     // m < 2^e
        *scale = ldexpf(1.0f, 14 - e);
    }
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

// Tensor-core Hutchinson: q_j for j < m into q_dev (device FP64). mode 2:
// FP16 two-term products (the converters flag any scaled entry beyond the
// FP16 range in ctl->pad0, checked by the caller); mode 3: BF16 three-term.
template <int MODE>
msp_status hutch_tc_launch(msp_ctx* ctx, const CUtensorMap& tmA, const CUtensorMap& tmG, const float* scale,
                           const uint32_t* bits, int wpr, int p0, int N, int64_t ntiles, int grid, double* part,
                           int* err, int* ovf) {
    // per call: the attribute belongs to the current device
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hutch_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
    k_hutch_tc<MODE><<<grid, kTcThreads, kTcSmem, ctx->stream>>>(tmA, tmG, scale, bits, wpr, p0, N, ntiles, part,
                                                                  err, ovf);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status hutch_tc(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t m, uint64_t seed,
                    double* q_dev, int mode) {
    auto enc = msp_tensor_map_encoder();
    const int64_t nt = (n + 127) / 128, n_pad = nt * 128;
    const int64_t ntiles = nt * (nt + 1) / 2;
    const int grid = (int)std::min<int64_t>(ntiles, ctx->num_sms);
    const size_t b_g = round_up(n_pad * m * 2, 256);
    const size_t b_bits = round_up(n_pad * (m / 32) * 4, 256);
    const size_t b_part = round_up((int64_t)grid * 256 * 8, 256);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, b_g + b_bits + b_part + 256, &scr));
    char* c = (char*)scr;
    uint16_t* Gt = (uint16_t*)c; c += b_g;
    uint32_t* bits = (uint32_t*)c; c += b_bits;
    double* part = (double*)c; c += b_part;
    float* scale = (float*)c;
    k_probes_16<<<(unsigned)((n_pad * m + 255) / 256), 256, 0, ctx->stream>>>(n, n_pad, (int)m, seed, mode == 2, Gt);
    MSP_CHECK_LAUNCH(ctx);
    {
        const int64_t warps = n_pad * (m / 32);
        k_probe_bits<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, ctx->stream>>>(n, n_pad, (int)m, seed, bits);
        MSP_CHECK_LAUNCH(ctx);
    }
    if (mode == 2) {
        k_diag_scale<<<1, 1024, 0, ctx->stream>>>(A, lda, n, scale);
        MSP_CHECK_LAUNCH(ctx);
    }
    CUtensorMap tmA;
    {
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
        const cuuint32_t box[2] = {kTcK, 128};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box,
                               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return msp_set_error(ctx, MSP_ECUDA, "hutchinson: cuTensorMapEncodeTiled(A) failed (%d)", (int)r);
    }
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    for (int64_t p0 = 0; p0 < m; p0 += 256) {
        const int N = (int)std::min<int64_t>(256, m - p0);
        CUtensorMap tmG;
        const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)m};
        const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 2};
        const cuuint32_t box[2] = {kTcK, (cuuint32_t)N};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmG, mode == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                               Gt, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return msp_set_error(ctx, MSP_ECUDA, "hutchinson: cuTensorMapEncodeTiled(G) failed (%d)", (int)r);
        if (mode == 2)
            MSP_TRY(hutch_tc_launch<2>(ctx, tmA, tmG, scale, bits, (int)(m / 32), (int)p0, N, ntiles, grid, part,
                                       &ctl->error, &ctl->pad0));
        else
            MSP_TRY(hutch_tc_launch<3>(ctx, tmA, tmG, scale, bits, (int)(m / 32), (int)p0, N, ntiles, grid, part,
                                       &ctl->error, &ctl->pad0));
        k_hutch_tc_reduce<<<(unsigned)((N + 7) / 8), 256, 0, ctx->stream>>>(part, grid, N, (int)p0,
                                                                           mode == 2 ? scale : nullptr, q_dev);
        MSP_CHECK_LAUNCH(ctx);
    }
    return MSP_OK;
}

// The device-side wait status of the tensor-core path (ctl->error), read
// back after a stream synchronisation.
// *overflow: an FP16 two-term pass met an entry beyond the FP16 range.
msp_status hutch_check(msp_ctx* ctx, bool* overflow = nullptr) {
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    int* h = (int*)ctx->host_flags;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(h, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(h + 1, &ctl->pad0, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (overflow) *overflow = h[1] != 0;
    if (h[0] != 0)
        return msp_set_error(ctx, (msp_status)h[0], "hutchinson: a device-side wait gave up (status %d)", h[0]);
    return MSP_OK;
}

msp_status hutch_simt(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t m, uint64_t seed,
                      double* q_dev);

// rows 16-byte aligned: the tensor-core path (TMA)
bool hutch_tc_ok(const void* A, int64_t lda) {
    return (lda % 4) == 0 && ((uintptr_t)A & 15) == 0 && msp_tensor_map_encoder() != nullptr;
}

msp_status hutch_impl(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda, int64_t m,
                      uint64_t seed, double* q_dev, double* ms_dev, int mode) {
    if (dt != MSP_F32)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: A must be FP32");
    if (n < 1 || lda < n || m < kPC || m % kPC != 0 || m > 4096)
        return msp_set_error(ctx, MSP_EINVAL, "hutchinson: need lda >= n >= 1 and probes a multiple of %d in [%d, 4096]",
                             kPC, kPC);
    // the device-side wait status and the FP16 range flag of this call (read
    // back by hutch_check)
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(&((CtlBlock*)ctx->ctl)->error, 0, sizeof(int), ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(&((CtlBlock*)ctx->ctl)->pad0, 0, sizeof(int), ctx->stream));
    if (hutch_tc_ok(A, lda)) {
        MSP_TRY(hutch_tc(ctx, (const float*)A, n, lda, m, seed, q_dev, mode));
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
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hutch_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHutchSmem));
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
    bool ovf = false;
    MSP_TRY(hutch_impl(ctx, A, dtype, n, lda, probes, seed, q, nullptr, ctx->hutch_terms));
    MSP_TRY(hutch_check(ctx, &ovf));
    if (ovf && ctx->hutch_terms == 2) {
        // an entry beyond the FP16 range (|a_ij| > max_k a_kk: not PSD): the
        // exact BF16 three-term products
        MSP_TRY(hutch_impl(ctx, A, dtype, n, lda, probes, seed, q, nullptr, 3));
        MSP_TRY(hutch_check(ctx));
    }
    return MSP_OK;
}

msp_status msp_set_hutchinson_terms(msp_ctx* ctx, int terms) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (terms != 2 && terms != 3) return msp_set_error(ctx, MSP_EINVAL, "hutchinson terms must be 2 or 3");
    ctx->hutch_terms = terms;
    return MSP_OK;
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
    double* h = (double*)ctx->host_flags + 16;
    msp_status st = MSP_OK;
    for (int mode : {ctx->hutch_terms, 3}) {
        st = hutch_impl(ctx, A, dtype, n, lda, probes, seed, buf, buf + probes, mode);
        bool ovf = false;
        if (st == MSP_OK) {
            cudaError_t e = cudaMemcpyAsync(h, buf + probes, 16, cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) st = msp_set_error(ctx, MSP_ECUDA, "schatten: %s", cudaGetErrorString(e));
            else st = hutch_check(ctx, &ovf);   // synchronises the stream
        }
        // an entry beyond the FP16 range (not PSD): again with three BF16 terms
        if (st != MSP_OK || !ovf || mode == 3) break;
    }
    cudaFreeAsync(buf, ctx->stream);
    if (st != MSP_OK) return st;
    if (norm) *norm = h[0];
    if (norm_pow) *norm_pow = h[0];
    if (std_err) *std_err = h[1];
    return MSP_OK;
}

}  // extern "C"
