// The sketch pass over a symmetric FP32 A in device memory (Algorithm 1,
// steps 2-3, with the packed tiles the solves keep of A), in one read of A:
//   C = A Pi           computed as A^T Pi: the CTA for rows [i0, i0 + 32) of
//                      C reads the column block A[:, i0 .. i0 + 32) in chunks
//                      of kSJ rows by TMA (box {32, 256}, twice per chunk;
//                      128-byte rows, no transpose needed), so that row j of
//                      the staged chunk holds the 32 values column c of C
//                      gathers for an entry (j, sign);
//   packed tiles       the 128 x 128 upper tiles of A the packed A pass reads,
//                      stored from the staged chunks by TMA (the column block
//                      is a 32-column slice of one tile column);
// (The norm-bound row statistics of the backward-error rule are a pass of
// their own: taken from the staged chunks here they cost more issue slots
// in this gather-bound kernel than a separate HBM-bound pass over A.)
// Gathers: one thread per column c of C, 32 accumulators (the block's rows).
// An entry (j, sign) of column c reads the 128-byte row j of the chunk as
// eight 16-byte pieces; lane l reads them in the order (q + l) mod 8, so the
// 32 lanes of a warp hit every bank group four times per instruction whatever
// their rows j are (no bank conflicts), and accumulator slot q holds the
// rows of piece (q + l) mod 8.
// Chunks: kSWin chunks of kSJ rows are resident at once. A thread walks its
// column's CSR entries in order (ascending j), and a lane whose next entry
// lies in a later resident chunk goes on with it while its warp-mates finish
// the earlier one: a warp's gather steps follow its busiest lane over the
// window, not over each chunk (entries per column are Poisson-like, about 4
// per chunk at s = 1024 and 12 per window, so the busiest of 32 lanes is
// far above the mean for one chunk and less so for three). A warp releases a
// chunk once all its lanes are past it; the last warp of the block to release
// chunk k stores its packed tiles and refills the stage with chunk k + kSWin.
// Each accumulator takes its FMAs in the order of the column's entries.
#include "msp_internal.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cstdint>

namespace {

constexpr int kSR = 32;                            // rows of C per CTA (columns of A)
constexpr int kSJ = 512;                           // rows of A per chunk
constexpr int kSBox = 256;                         // rows per TMA box
constexpr int kSWin = 3;                           // resident chunks (stages)
constexpr uint32_t kSStageBytes = kSJ * kSR * 4;   // 64 KB
constexpr int kSTile = 128;                        // packed tile side

struct SymArgs {
    int64_t n, s_pad;
    int nch;                 // chunks (cover the tile rows up to nt * 128)
    int nt;                  // tiles per side
    int ib0;                 // first 32-row block of C of this launch
    const int32_t* ptr;      // [s_pad + 1] CSR column starts
    const int32_t* ent;      // (j << 1) | negative, CSR by column
    float scale;
    float* C;
    int* err;
};

// upper tile (I, J), I <= J, row-major over the upper triangle
__device__ inline int64_t tile_index(int I, int J, int nt) {
    return (int64_t)I * nt - (int64_t)I * (I - 1) / 2 + (J - I);
}

// acc[q][.] += sg * (piece (q + lane) mod 8 of the 128-byte row)
__device__ __forceinline__ void gather_row(float (&acc)[8][4], const uint8_t* row, uint32_t lrot, float sg) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(row + ((lrot + 16u * q) & 112u));
        acc[q][0] = fmaf(sg, x.x, acc[q][0]);
        acc[q][1] = fmaf(sg, x.y, acc[q][1]);
        acc[q][2] = fmaf(sg, x.z, acc[q][2]);
        acc[q][3] = fmaf(sg, x.w, acc[q][3]);
    }
}

// Non-blocking test of the phase of the given parity (acquire on success).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(msp::smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__global__ void __launch_bounds__(1024, 1)
k_sketch_sym(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmP, SymArgs a,
             int pack) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (msp::smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kSWin * kSStageBytes);
    int* rel = reinterpret_cast<int*>(full + kSWin);        // [kSWin] warps past the stage's chunks
    int* s_issued = rel + kSWin;                             // chunks issued
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_issued + 1);

    const int tid = threadIdx.x, lane = tid & 31, nw = (int)(blockDim.x >> 5);
    const int64_t i0 = ((int64_t)a.ib0 + blockIdx.y) * kSR;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + tid;      // column of C
    const bool lead = (blockIdx.x == 0);                            // packs the tiles
    const int Jt = (int)(i0 / kSTile);
    const int nch = a.nch;

    auto issue = [&](int k, int st) {
        msp::mbar_arrive_expect_tx(&full[st], kSStageBytes);
        for (int b = 0; b < kSJ / kSBox; ++b)
            msp::tc::tma_load_2d(sm + st * kSStageBytes + b * kSBox * kSR * 4, &tmA, (int32_t)i0,
                                 k * kSJ + b * kSBox, &full[st]);
    };
    if (tid == 0) {
        for (int s = 0; s < kSWin; ++s) {
            msp::mbar_init(&full[s], 1);
            rel[s] = 0;
        }
        *s_issued = nch < kSWin ? nch : kSWin;
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        msp::tc::prefetch_tensormap(&tmA);
        for (int k = 0; k < (nch < kSWin ? nch : kSWin); ++k) issue(k, k);
    }
    __syncthreads();

    // bounded wait for chunk k (every lane; false for the whole warp if any
    // lane gave up or another warp has)
    auto wait_chunk = [&](int k) -> bool {
        bool ok = (*s_abort == 0) &&
                  msp::mbar_wait_sleep(&full[k % kSWin], (uint32_t)((k / kSWin) & 1), a.err);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) *s_abort = 1;
        return ok;
    };
    // chunk k is done with in this warp; the block's last warp stores its
    // packed tiles and refills the stage
    auto release = [&](int k) {
        __syncwarp();
        if (lane == 0) {
            const int st = k % kSWin;
            __threadfence_block();
            const int old = atomicAdd(&rel[st], 1);
            if (old == nw * (k / kSWin + 1) - 1) {
                __threadfence_block();
                if (pack && lead) {
                    const int64_t j0 = (int64_t)k * kSJ;
                    for (int h = 0; h < kSJ / kSTile; ++h) {
                        const int I = (int)(j0 / kSTile) + h;
                        if (I <= Jt && I < a.nt)
                            msp::tc::tma_store_2d(&tmP, (int32_t)(i0 % kSTile),
                                                  (int32_t)(tile_index(I, Jt, a.nt) * kSTile),
                                                  sm + st * kSStageBytes + h * kSTile * kSR * 4);
                    }
                    msp::tc::bulk_commit();
                    msp::tc::bulk_wait_read();
                }
                if (k + kSWin < nch && *s_abort == 0) {
                    msp::tc::fence_proxy_async();
                    issue(k + kSWin, st);
                    atomicMax(s_issued, k + kSWin + 1);
                }
            }
        }
        __syncwarp();
    };

    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[q][t] = 0.f;
    const uint32_t lrot = (uint32_t)lane * 16u;

    const bool col_ok = c < a.s_pad;
    int e = col_ok ? __ldg(&a.ptr[c]) : 0;
    const int e_end = col_ok ? __ldg(&a.ptr[c + 1]) : 0;
    // the next three entries, loads in flight ahead of their gathers
    int32_t v0 = (e < e_end) ? __ldg(&a.ent[e]) : 0;
    int32_t v1 = (e + 1 < e_end) ? __ldg(&a.ent[e + 1]) : 0;
    int32_t v2 = (e + 2 < e_end) ? __ldg(&a.ent[e + 2]) : 0;
    int loaded = 0, released = 0;       // warp-uniform: chunks seen complete, chunks released
    bool ok = true;
    for (;;) {
        const int kl = (e < e_end) ? ((v0 >> 1) / kSJ) : nch;      // chunk of this lane's next entry
        const int kmin = (int)__reduce_min_sync(0xffffffffu, (unsigned)kl);
        while (released < kmin) {
            if (loaded <= released) {
                if (!(ok = wait_chunk(released))) break;
                loaded = released + 1;
            }
            release(released);
            ++released;
        }
        if (!ok || kmin >= nch) break;
        if (loaded <= kmin) {
            if (!(ok = wait_chunk(kmin))) break;
            loaded = kmin + 1;
        } else if (loaded < nch && loaded < kmin + kSWin && __any_sync(0xffffffffu, kl >= loaded)) {
            // a later chunk may have landed: lanes there need not wait
            const bool t = mbar_test(&full[loaded % kSWin], (uint32_t)((loaded / kSWin) & 1));
            if (__all_sync(0xffffffffu, t)) ++loaded;
        }
        if (kl < loaded) {
            const int32_t jr = (v0 >> 1) - kl * kSJ;
            gather_row(acc, sm + (kl % kSWin) * kSStageBytes + jr * (kSR * 4), lrot, (v0 & 1) ? -1.f : 1.f);
            ++e;
            v0 = v1;
            v1 = v2;
            v2 = (e + 2 < e_end) ? __ldg(&a.ent[e + 2]) : 0;
        }
    }
    __syncthreads();
    if (*s_abort) {
        // bounded waits for the loads that may still be in flight (the last
        // kSWin chunks issued; every earlier one was waited for) before exit
        if (tid == 0) {
            const int iss = *s_issued;
            for (int k = iss > kSWin ? iss - kSWin : 0; k < iss; ++k)
                msp::mbar_wait_timed(&full[k % kSWin], (uint32_t)((k / kSWin) & 1), a.err);
        }
        if (lane == 0 && pack && lead) msp::tc::bulk_wait_all();
        return;
    }
    if (lane == 0 && pack && lead) msp::tc::bulk_wait_all();
    if (col_ok) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t r0 = i0 + 4 * ((q + lane) & 7);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (r0 + t < a.n) a.C[(r0 + t) * a.s_pad + c] = acc[q][t] * a.scale;
        }
    }
}

// The lower triangle of tile column J = J0 + blockIdx.y of a symmetric
// row-major A from its upper triangle: tile (I, J), I = blockIdx.x >= J, is
// the transpose of tile (J, I) (blocks with I < J return at once); on the
// diagonal tile only the entries below the diagonal are written. 32 x 33
// shared-memory transposes, coalesced both ways. It reads only tile rows J
// and writes only tile column J, so it completes the column block of A that
// the one-pass kernel stages for the rows of C in that tile column.
__global__ void __launch_bounds__(256) k_mirror_lower_cols(float* __restrict__ A, int64_t lda, int64_t n, int J0) {
    __shared__ float tr[32][33];
    const int J = J0 + (int)blockIdx.y, I = (int)blockIdx.x;
    if (I < J) return;
    const bool diag = (I == J);
    const int64_t r0 = (int64_t)I * kSTile, c0 = (int64_t)J * kSTile;   // destination (rows r0.., cols c0..)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;               // 32 x 8
    for (int bi = 0; bi < kSTile; bi += 32)
        for (int bj = 0; bj < kSTile; bj += 32) {
            if (diag && bj > bi) continue;          // block-uniform: the upper half of a diagonal tile stays
            // source block A[c0 + bj + y][r0 + bi + x] (rows of the upper tile (J, I))
            for (int y = ty; y < 32; y += 8) {
                const int64_t sr = c0 + bj + y, sc = r0 + bi + tx;
                tr[y][tx] = (sr < n && sc < n) ? A[sr * lda + sc] : 0.f;
            }
            __syncthreads();
            // strictly lower entries only on the diagonal tile; their sources
            // lie strictly above the diagonal and are never written
            for (int y = ty; y < 32; y += 8) {
                const int64_t dr = r0 + bi + y, dc = c0 + bj + tx;
                if (dr < n && dc < n && (!diag || dr > dc)) A[dr * lda + dc] = tr[tx][y];
            }
            __syncthreads();
        }
}

}  // namespace

// Fills the lower triangle of tile columns [J0, J1) (the diagonal tiles
// included) from the upper triangle, which must already be in place in tile
// rows [J0, J1). Afterwards the columns [J0, J1) * 128 of A are complete.
msp_status msp_mirror_lower_cols(msp_ctx* ctx, float* A, int64_t lda, int64_t n, int64_t J0, int64_t J1) {
    const int64_t nt = (n + kSTile - 1) / kSTile;
    J1 = std::min(J1, nt);
    if (J0 < 0 || J0 >= J1) return MSP_OK;
    k_mirror_lower_cols<<<dim3((unsigned)nt, (unsigned)(J1 - J0)), 256, 0, ctx->stream>>>(A, lda, n, (int)J0);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

bool msp_sketch_sym_ok(const void* A, int64_t n, int64_t lda, int64_t s_pad, int gamma) {
    const int64_t groups = (s_pad + 1023) / 1024;
    return msp_tensor_map_encoder() != nullptr && ((uintptr_t)A & 15) == 0 && lda % 4 == 0 && n >= kSR &&
           s_pad % 64 == 0 && s_pad <= 2048 && s_pad % groups == 0 && (s_pad / groups) % 32 == 0 &&
           gamma >= 1 && n < (1ll << 30);
}

msp_status msp_sketch_sym_blocks(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t s_pad,
                                 const int32_t* ptr, const int32_t* ent, int gamma, float* C, float* packed,
                                 int64_t ib0, int64_t ib1) {
    auto enc = msp_tensor_map_encoder();
    if (!enc || !msp_sketch_sym_ok(A, n, lda, s_pad, gamma))
        return msp_set_error(ctx, MSP_EINVAL, "sketch_sym: unsupported arguments");
    const int nt = (int)((n + kSTile - 1) / kSTile);
    // chunks up to the last tile row, so that the padding of the packed
    // tiles is written (zeros: the loads beyond n are zero-filled)
    const int nch = (int)(((int64_t)nt * kSTile + kSJ - 1) / kSJ);
    // column groups of at most 1024 columns, each a multiple of 32
    const int groups = (int)((s_pad + 1023) / 1024);
    const int threads = (int)(s_pad / groups);
    CUtensorMap tmA, tmP;
    {
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kSR, (cuuint32_t)kSBox};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return msp_set_error(ctx, MSP_ECUDA, "sketch_sym: tensor map of A failed (%d)", (int)r);
    }
    if (packed) {
        const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
        const cuuint64_t dims[2] = {(cuuint64_t)kSTile, (cuuint64_t)(ntiles * kSTile)};
        const cuuint64_t strides[1] = {(cuuint64_t)kSTile * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kSR, (cuuint32_t)kSTile};
        const cuuint32_t es[2] = {1, 1};
        const CUresult r = enc(&tmP, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)packed, dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return msp_set_error(ctx, MSP_ECUDA, "sketch_sym: tensor map of the packed tiles failed (%d)", (int)r);
    } else {
        tmP = tmA;   // unused
    }
    SymArgs a;
    a.n = n;
    a.s_pad = s_pad;
    a.nch = nch;
    a.nt = nt;
    // row blocks of C (32 rows each) up to the last tile column (blocks past n
    // only write the zero padding of the packed tiles)
    ib1 = std::min<int64_t>(ib1, (int64_t)nt * kSTile / kSR);
    if (ib0 < 0 || ib0 >= ib1) return MSP_OK;
    a.ib0 = (int)ib0;
    a.ptr = ptr;
    a.ent = ent;
    a.scale = (float)(1.0 / std::sqrt((double)gamma));
    a.C = C;
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    a.err = &ctl->error;
    const size_t smem = (size_t)kSWin * kSStageBytes + 64 + 1024;
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sketch_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the first launch of a pass clears the error word (a pass may come in
    // several launches over consecutive block ranges, in order on one stream)
    if (ib0 == 0) MSP_CUDA_TRY(ctx, cudaMemsetAsync(&ctl->error, 0, sizeof(int), ctx->stream));
    // grid: column groups x the 32-column blocks [ib0, ib1)
    dim3 grid((unsigned)groups, (unsigned)(ib1 - ib0));
    k_sketch_sym<<<grid, threads, smem, ctx->stream>>>(tmA, tmP, a, packed ? 1 : 0);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_sketch_sym_pass(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t s_pad,
                               const int32_t* ptr, const int32_t* ent, int gamma, float* C, float* packed) {
    return msp_sketch_sym_blocks(ctx, A, n, lda, s_pad, ptr, ent, gamma, C, packed, 0, INT64_MAX);
}

extern "C" msp_status msp_set_sketch_one_pass(msp_ctx* ctx, int on) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    ctx->sketch_sym = on != 0;
    return MSP_OK;
}
