// The Gram of the level-2 sketch on the tensor cores (Algorithm 1 step 4):
//   M2 = X^T X + lam W   (X = C~, K x s FP32 row-major; s x s, FP64 out),
// the contraction msp_build_factor factors. The preconditioner is SPD only
// while M2 - X^T X = lam W + (Gram error) stays positive definite, and lam W
// can be tiny next to X^T X, so the Gram must be nearly exact: every entry of
// q X (q a power of two with q max|x| <= 2^14) is split into three FP16 terms
// h + m + l (11 + 11 + 11 significant bits, which hold an FP32 significand),
// and the six term products of order up to 2^-22 (hh, hm, mh, mm, hl, lh) are
// accumulated; the dropped ml, lm, ll are of order 2^-33. Steps:
//   k_absmax         max |x| (one pass over X), q from its exponent;
//   k_split_t        H^T, M^T, L^T as s_t x K_pad FP16 (K contiguous, the
//                    K-major operand layout), through 32 x 32 shared tiles;
//   k_gram_tc        per work item (upper 128 x 128 tile pair (I, J), slice of
//                    rows of X): TMA (SWIZZLE_64B) loads of the three terms of
//                    tiles I and J in chunks of 32 rows, six tcgen05.mma per 16
//                    rows into FP32 accumulators in tensor memory: hh alone in
//                    one of two alternate buffers, drained every 64 rows into
//                    per-thread float-float sums (TwoSum, Knuth), and the five
//                    smaller products (2^-11 of hh) in a third accumulator
//                    drained every 512 rows. The FP32 accumulation in
//                    tensor memory is not compensated, so its error grows with
//                    the MMA steps between drains (measured): 4 for hh. The
//                    item's 128 x 128 partial is written in FP64;
//   k_gram_tc_finish M2 = (sum over slices, in order, in FP64) / q^2 + lam W,
//                    mirrored, identity on the padding.
// Warp roles in k_gram_tc: 0 TMA producer (and tensor-memory owner), 1 MMA
// issuer, 2..9 drain (tensor-memory lane quarter = warp mod 4, 64 columns
// each).
#include "msp_internal.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kGT = 128;                                   // output tile side
constexpr int kGK = 32;                                    // rows of X per chunk (64-byte FP16 rows)
constexpr int kGTerms = 3;                                 // FP16 terms per entry
constexpr int kGStages = 4;
constexpr int kGDrain = 2;                                 // chunks per tensor-memory drain
constexpr int kGEpiWarps = 8;
constexpr uint32_t kGOpBytes = kGT * kGK * 2;              // one term tile: 8 KB
constexpr uint32_t kGStageBytes = 2 * kGTerms * kGOpBytes; // terms of I and J: 48 KB
constexpr uint32_t kGOffBar = kGStages * kGStageBytes;
constexpr size_t kGSmem = kGOffBar + 256 + 1024;
constexpr int kGThreads = (2 + kGEpiWarps) * 32;
// tensor memory (512 columns): two 128-column accumulators of the hh product
// (alternate 64-row groups), the accumulator of the five smaller products,
// and the drain's low parts (the high parts stay in registers)
constexpr uint32_t kGTmemCols = 512;
constexpr uint32_t kGCrossCol = 2 * kGT;
constexpr uint32_t kGLoCol = 3 * kGT;
constexpr int kGCrossGroups = 8;       // groups between drains of the small-product accumulator

// the five smaller term products (term of tile I, term of tile J), smallest
// first; 0 = h, 1 = m, 2 = l
__device__ constexpr int kPairI[5] = {0, 2, 1, 0, 1};
__device__ constexpr int kPairJ[5] = {2, 0, 1, 1, 0};

// the small-product accumulator is drained with group g
__device__ inline bool cross_drain(int g, int ngroups) { return (g + 1) % kGCrossGroups == 0 || g == ngroups - 1; }

// max |x| over K rows of s columns (ld), as the bits of a non-negative float;
// blocks over rows, threads over columns
__global__ void k_absmax(const float* __restrict__ X, int64_t K, int64_t ld, int64_t s,
                         unsigned int* __restrict__ out) {
    float m = 0.f;
    for (int64_t r = blockIdx.x; r < K; r += gridDim.x)
        for (int64_t c = threadIdx.x; c < s; c += blockDim.x) m = fmaxf(m, fabsf(X[r * ld + c]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// q = 2^(14 - e) with max < 2^e (1 for an all-zero X)
__global__ void k_scale_of(const unsigned int* __restrict__ mx, float* __restrict__ q) {
    const float m = __uint_as_float(*mx);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);
    *q = ldexpf(1.0f, 14 - max(e, -100));   // q m < 2^14; q finite
}

// H^T, M^T, L^T (s_t x K_pad FP16, zero beyond K and s) from v = q x:
// h = fp16(v), m = fp16(v - h), l = fp16(v - h - m) (both differences exact
// in FP32); 32 x 32 tiles, block (32, 8).
__global__ void k_split_t(const float* __restrict__ X, int64_t K, int64_t ld, int64_t s, int64_t K_pad,
                          const float* __restrict__ qp, __half* __restrict__ Ht, __half* __restrict__ Mt,
                          __half* __restrict__ Lt) {
    __shared__ float tile[32][33];
    const float q = *qp;
    const int64_t k0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t k = k0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (k < K && c < s) ? q * X[k * ld + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, k = k0 + threadIdx.x;
        const float v = tile[threadIdx.x][i];
        const __half h = __float2half_rn(v);
        const float r1 = __fsub_rn(v, __half2float(h));
        const __half m = __float2half_rn(r1);
        const __half l = __float2half_rn(__fsub_rn(r1, __half2float(m)));
        Ht[c * K_pad + k] = h;
        Mt[c * K_pad + k] = m;
        Lt[c * K_pad + k] = l;
    }
}

// (hi, lo) += v by TwoSum: hi + lo carries the exact running sum to within
// one rounding of lo
__device__ inline void two_sum_acc(float& hi, float& lo, float v) {
    const float t = __fadd_rn(hi, v);
    const float bp = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    hi = t;
    lo = __fadd_rn(lo, e);
}

// upper tile pair p (row-major over ta <= tb) of nt tiles
__device__ inline void pair_of(int p, int nt, int& ta, int& tb) {
    int a = 0;
    while (p >= nt - a) {
        p -= nt - a;
        ++a;
    }
    ta = a;
    tb = a + p;
}

__global__ void __launch_bounds__(kGThreads, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmM,
          const __grid_constant__ CUtensorMap tmL, int nt, int64_t K_pad, int64_t slice_k, int ns,
          double* __restrict__ P, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (msp::smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kGOffBar);
    uint64_t* full = bar;                     // [stages] terms landed (TMA)
    uint64_t* empty = bar + kGStages;         // [stages] their MMAs done (commit)
    uint64_t* accf = bar + 2 * kGStages;      // [2] accumulator buffer complete (commit)
    uint64_t* acce = bar + 2 * kGStages + 2;  // [2] accumulator buffer drained (drain warps)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kGOffBar + 128);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + kGOffBar + 132);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x, p = item / ns, sl = item % ns;
    int ta, tb;
    pair_of(p, nt, ta, tb);
    const bool diag = (ta == tb);
    const int64_t k0 = (int64_t)sl * slice_k;
    const int nchunks = (int)((std::min<int64_t>(K_pad, k0 + slice_k) - k0) / kGK);
    const int ngroups = (nchunks + kGDrain - 1) / kGDrain;

    if (tid == 0) {
        for (int i = 0; i < 2 * kGStages + 2; ++i) msp::mbar_init(&bar[i], 1);
        for (int i = 0; i < 2; ++i) msp::mbar_init(&acce[i], kGEpiWarps);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        msp::tc::prefetch_tensormap(&tmH);
        msp::tc::prefetch_tensormap(&tmM);
        msp::tc::prefetch_tensormap(&tmL);
    }
    if (warp == 0) msp::tc::tmem_alloc(tslot, kGTmemCols);
    msp::tc::fence_before_sync();
    __syncthreads();
    msp::tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    auto wait = [&](uint64_t* b, int parity) -> bool {
        if (*s_abort) return false;
        if (!msp::mbar_wait_timed(b, (uint32_t)(parity & 1), err)) {
            *s_abort = 1;
            return false;
        }
        return true;
    };
    int issued = 0, mma_done_upto = -1;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t tx = (diag ? 1u : 2u) * kGTerms * kGOpBytes;
            for (int c = 0; c < nchunks; ++c) {
                const int st = c % kGStages;
                if (c >= kGStages && !wait(&empty[st], c / kGStages - 1)) break;
                uint8_t* base = sm + st * kGStageBytes;
                const int x = (int)(k0 + (int64_t)c * kGK);
                msp::mbar_arrive_expect_tx(&full[st], tx);
#pragma unroll
                for (int t = 0; t < kGTerms; ++t) {
                    const CUtensorMap* mp = t == 0 ? &tmH : (t == 1 ? &tmM : &tmL);
                    msp::tc::tma_load_2d(base + t * kGOpBytes, mp, x, ta * kGT, &full[st]);
                    if (!diag) msp::tc::tma_load_2d(base + (kGTerms + t) * kGOpBytes, mp, x, tb * kGT, &full[st]);
                }
                issued = c + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = msp::tc::idesc_f16_f32(kGT, kGT);
            bool cross_fresh = true;
            for (int c = 0; c < nchunks; ++c) {
                const int st = c % kGStages;
                const int g = c / kGDrain, b = g & 1;
                const bool first = (c % kGDrain) == 0;
                // buffer b was drained with group g - 2; the small-product
                // accumulator, when group g - 1 drained it
                if (first && g >= 2 && !wait(&acce[b], g / 2 - 1)) break;
                if (first && g >= 1 && cross_drain(g - 1, ngroups) && !wait(&acce[(g - 1) & 1], (g - 1) / 2)) break;
                if (!wait(&full[st], c / kGStages)) break;
                msp::tc::fence_after_sync();
                const uint32_t base = msp::smem_u32(sm + st * kGStageBytes);
                const uint32_t bj = diag ? base : base + kGTerms * kGOpBytes;
                const uint32_t dh = tmem + (uint32_t)(b * kGT), dx = tmem + kGCrossCol;
#pragma unroll
                for (int ks = 0; ks < kGK / 16; ++ks) {
#pragma unroll
                    for (int pr = 0; pr < 5; ++pr) {
                        const uint64_t ad = msp::tc::sdesc_kmajor_sw64(base + kPairI[pr] * kGOpBytes + ks * 32);
                        const uint64_t bd = msp::tc::sdesc_kmajor_sw64(bj + kPairJ[pr] * kGOpBytes + ks * 32);
                        msp::tc::mma_bf16(dx, ad, bd, idesc, !(cross_fresh && ks == 0 && pr == 0));
                    }
                    msp::tc::mma_bf16(dh, msp::tc::sdesc_kmajor_sw64(base + ks * 32),
                                      msp::tc::sdesc_kmajor_sw64(bj + ks * 32), idesc, !(first && ks == 0));
                }
                cross_fresh = false;
                msp::tc::mma_commit(&empty[st]);
                if ((c % kGDrain) == kGDrain - 1 || c == nchunks - 1) {
                    msp::tc::mma_commit(&accf[b]);
                    cross_fresh = cross_drain(g, ngroups);
                }
                mma_done_upto = c;
            }
        }
    } else {
        // drain: row quarter*32 + lane of the tile, columns half*64 .. + 63;
        // high parts in registers, low parts in tensor memory
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
        float hi[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) hi[j] = 0.f;
        bool ok = true;
        for (int g = 0; g < ngroups; ++g) {
            const int b = g & 1;
            ok = wait(&accf[b], g / 2);
            if (!__all_sync(0xffffffffu, ok)) break;
            msp::tc::fence_after_sync();
            const bool xd = cross_drain(g, ngroups);
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                float v[32], lo[32];
                msp::tc::tmem_ld32(lane_base + (uint32_t)(b * kGT + cc * 32), v);
                if (g > 0) {
                    msp::tc::tmem_ld32(lane_base + kGLoCol + (uint32_t)(cc * 32), lo);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) lo[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) two_sum_acc(hi[cc * 32 + i], lo[i], v[i]);
                if (xd) {
                    msp::tc::tmem_ld32(lane_base + kGCrossCol + (uint32_t)(cc * 32), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) two_sum_acc(hi[cc * 32 + i], lo[i], v[i]);
                }
                msp::tc::tmem_st32(lane_base + kGLoCol + (uint32_t)(cc * 32), lo);
            }
            msp::tc::tmem_wait_st();
            msp::tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&acce[b]);
        }
        if (__all_sync(0xffffffffu, ok) && ngroups > 0) {
            const int row = quarter * 32 + lane;
            double* dst = P + ((int64_t)item * kGT + row) * kGT + half * 64;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                float lo[32];
                msp::tc::tmem_ld32(lane_base + kGLoCol + (uint32_t)(cc * 32), lo);
#pragma unroll
                for (int j = 0; j < 32; j += 2)
                    *reinterpret_cast<double2*>(dst + cc * 32 + j) =
                        make_double2((double)hi[cc * 32 + j] + (double)lo[j],
                                     (double)hi[cc * 32 + j + 1] + (double)lo[j + 1]);
            }
        }
    }
    __syncthreads();
    if (*s_abort) {
        // bounded waits for this CTA's copies and MMAs in flight, then free
        if (warp == 0 && lane == 0)
            for (int c = std::max(0, issued - kGStages); c < issued; ++c)
                msp::mbar_wait_timed(&full[c % kGStages], (uint32_t)((c / kGStages) & 1), err);
        if (warp == 1 && lane == 0 && mma_done_upto >= 0)
            msp::mbar_wait_timed(&empty[mma_done_upto % kGStages], (uint32_t)((mma_done_upto / kGStages) & 1), err);
        __syncthreads();
    }
    msp::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        msp::tc::tmem_dealloc(tmem, kGTmemCols);
    }
}

// M2[a][b] = (sum over slices of the tile partial, FP64, slice order) / q^2
//            + lam (W ? W[a][b] : [a == b]); the upper partial mirrored;
//            identity on the padding.
template <typename TW>
__global__ void k_gram_tc_finish(const double* __restrict__ P, int nt, int ns, const float* __restrict__ qp,
                                 const TW* __restrict__ W, double lam, int64_t s, int64_t s_pad,
                                 double* __restrict__ M2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    const int64_t a = e / s_pad, b = e % s_pad;
    if (a >= s || b >= s) {
        M2[e] = (a == b) ? 1.0 : 0.0;
        return;
    }
    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    const int ta = (int)(lo / kGT), tb = (int)(hi / kGT);
    const int64_t p = (int64_t)ta * nt - (int64_t)ta * (ta - 1) / 2 + (tb - ta);
    // within the pair's tile: row from the first tile, column from the second
    const int64_t r = lo % kGT, c = hi % kGT;
    double v = 0.0;
    for (int sl = 0; sl < ns; ++sl) v += P[((p * ns + sl) * kGT + r) * kGT + c];
    const double q = (double)*qp;
    v /= q * q;
    v += W ? lam * (double)W[e] : (a == b ? lam : 0.0);
    M2[e] = v;
}

}  // namespace

// M2 = X^T X + lam W (W: s_pad x s_pad; null: + lam I) for X: K x s FP32
// (leading dimension ld, no alignment needed), FP64 s_pad x s_pad out with
// the identity on the padding. The tiles cover s_t = s_pad rounded up to 128
// (zero columns beyond s). Callers check msp_gram_tc_ok first (the
// tensor-map encoder exists); otherwise they use the FP32-pipe Gram.
bool msp_gram_tc_ok(int64_t s_pad) { return s_pad % 32 == 0 && msp_tensor_map_encoder() != nullptr; }

msp_status msp_gram_tc(msp_ctx* ctx, const float* X, int64_t K, int64_t ld, int64_t s, int64_t s_pad,
                       const float* W, double lam, double* M2) {
    auto enc = msp_tensor_map_encoder();
    if (!enc || s_pad % 32 != 0 || K < 1 || s < 1 || s > s_pad || ld < s || K >= (1ll << 30))
        return msp_set_error(ctx, MSP_EINVAL, "gram_tc: unsupported arguments");
    const int64_t s_t = round_up(s_pad, kGT);
    const int nt = (int)(s_t / kGT);
    const int64_t K_pad = round_up(K, kGK);
    const int npairs = nt * (nt + 1) / 2;
    // slices: the fewest (<= 64) whose work items fill the SMs' waves to 85%,
    // else the count that fills them best
    const int64_t nch = K_pad / kGK;
    const int sms = std::max(1, ctx->num_sms);
    int ns = 1;
    double best = -1.0;
    for (int64_t c = 1; c <= std::min<int64_t>(64, nch); ++c) {
        const int64_t per = (nch + c - 1) / c;              // chunks per slice
        const int64_t cnt = (nch + per - 1) / per;          // slices actually used
        const int64_t it = (int64_t)npairs * cnt;
        const double eff = (double)it / (double)(((it + sms - 1) / sms) * sms);
        if (eff > best + 1e-9) {
            best = eff;
            ns = (int)cnt;
        }
        if (eff >= 0.85) break;
    }
    const int64_t slice_k = ((nch + ns - 1) / ns) * kGK;
    ns = (int)((K_pad + slice_k - 1) / slice_k);
    const int64_t items = (int64_t)npairs * ns;
    const size_t b_t = round_up(s_t * K_pad * 2, 256);
    const size_t b_p = round_up(items * kGT * kGT * 8, 256);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, kGTerms * b_t + b_p + 256, &scr));
    char* c = (char*)scr;
    __half* T[kGTerms];
    for (int t = 0; t < kGTerms; ++t) {
        T[t] = (__half*)c;
        c += b_t;
    }
    double* P = (double*)c; c += b_p;
    unsigned int* mx = (unsigned int*)c;
    float* q = (float*)(c + 16);
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, 4, ctx->stream));
    k_absmax<<<(unsigned)std::min<int64_t>(K, 4 * ctx->num_sms), 256, 0, ctx->stream>>>(X, K, ld, s, mx);
    MSP_CHECK_LAUNCH(ctx);
    k_scale_of<<<1, 1, 0, ctx->stream>>>(mx, q);
    MSP_CHECK_LAUNCH(ctx);
    k_split_t<<<dim3((unsigned)(K_pad / 32), (unsigned)(s_t / 32)), dim3(32, 8), 0, ctx->stream>>>(
        X, K, ld, s, K_pad, q, T[0], T[1], T[2]);
    MSP_CHECK_LAUNCH(ctx);
    CUtensorMap tm[kGTerms];
    for (int t = 0; t < kGTerms; ++t) {
        const cuuint64_t dims[2] = {(cuuint64_t)K_pad, (cuuint64_t)s_t};
        const cuuint64_t strides[1] = {(cuuint64_t)K_pad * 2};
        const cuuint32_t box[2] = {kGK, kGT};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tm[t], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)T[t], dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return msp_set_error(ctx, MSP_ECUDA, "gram_tc: cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    // per call: the attribute belongs to the current device
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem));
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(&ctl->error, 0, sizeof(int), ctx->stream));
    k_gram_tc<<<(unsigned)items, kGThreads, kGSmem, ctx->stream>>>(tm[0], tm[1], tm[2], nt, K_pad, slice_k, ns, P,
                                                                     &ctl->error);
    MSP_CHECK_LAUNCH(ctx);
    const unsigned fb = (unsigned)((s_pad * s_pad + 255) / 256);
    k_gram_tc_finish<float><<<fb, 256, 0, ctx->stream>>>(P, nt, ns, q, W, lam, s, s_pad, M2);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

extern "C" msp_status msp_set_gram_tensor_cores(msp_ctx* ctx, int on) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    ctx->gram_tc = on != 0;
    return MSP_OK;
}
