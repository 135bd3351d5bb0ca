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
// rows of piece (q + l) mod 8. A thread's first three entries of a chunk are
// read with all loads in flight together. The threads of a warp have different
// numbers of entries in a chunk (about 4 on average at s = 1024, kSJ = 512),
// so a warp runs as many gather steps as its busiest thread: long chunks
// narrow that spread. Chunks stream through kSStages stages of shared memory;
// thread 0 refills a stage once every warp has passed it.
#include "msp_internal.cuh"
#include "tc.cuh"

#include <algorithm>

namespace {

constexpr int kSR = 32;                            // rows of C per CTA (columns of A)
constexpr int kSJ = 512;                           // rows of A per chunk
constexpr int kSBox = 256;                         // rows per TMA box
constexpr int kSStages = 2;
constexpr uint32_t kSStageBytes = kSJ * kSR * 4;   // 64 KB
constexpr int kSTile = 128;                        // packed tile side

struct SymArgs {
    int64_t n, s_pad;
    int nch;                 // chunks (cover the tile rows up to nt * 128)
    int nt;                  // tiles per side
    const int32_t* tab;      // [s_pad][nch + 1] first entry of column c in chunk k
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

__global__ void __launch_bounds__(1024, 1)
k_sketch_sym(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmP, SymArgs a,
             int pack) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (msp::smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kSStages * kSStageBytes);
    volatile int* s_abort = reinterpret_cast<volatile int*>(full + kSStages);

    const int tid = threadIdx.x, lane = tid & 31;
    // blockIdx.x: column group (the groups of a row block run side by side,
    // so the block's repeated reads of A are served by L2); blockIdx.y: row block
    const int64_t i0 = (int64_t)blockIdx.y * kSR;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + tid;      // column of C
    const bool lead = (blockIdx.x == 0);                            // packs the tiles
    const int Jt = (int)(i0 / kSTile);                              // tile column of the block
    const int nch = a.nch;

    auto issue = [&](int k, int st) {
        msp::mbar_arrive_expect_tx(&full[st], kSStageBytes);
        for (int b = 0; b < kSJ / kSBox; ++b)
            msp::tc::tma_load_2d(sm + st * kSStageBytes + b * kSBox * kSR * 4, &tmA, (int32_t)i0,
                                 k * kSJ + b * kSBox, &full[st]);
    };
    if (tid == 0) {
        for (int s = 0; s < kSStages; ++s) msp::mbar_init(&full[s], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        msp::tc::prefetch_tensormap(&tmA);
        for (int k = 0; k < (nch < kSStages ? nch : kSStages); ++k) issue(k, k);
    }
    __syncthreads();

    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[q][t] = 0.f;
    // this lane's rotation of the pieces (bytes within a 128-byte row)
    const uint32_t lrot = (uint32_t)lane * 16u;

    const bool col_ok = c < a.s_pad;
    int e0 = col_ok ? __ldg(&a.tab[c * (nch + 1)]) : 0;
    int e1n = col_ok ? __ldg(&a.tab[c * (nch + 1) + 1]) : 0;
    int issued = nch < kSStages ? nch : kSStages, k_stop = nch;
    for (int k = 0; k < nch; ++k) {
        const int st = k % kSStages;
        const int e1 = e1n;
        if (col_ok && k + 1 < nch) e1n = __ldg(&a.tab[c * (nch + 1) + k + 2]);
        // this chunk's first three entries, loads in flight together (a
        // fourth one spills at the 64-register limit of 1024 threads)
        int32_t v3[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) v3[u] = (e0 + u < e1) ? __ldg(&a.ent[e0 + u]) : 0;
        bool ok = true;
        if (*s_abort == 0) ok = msp::mbar_wait_timed(&full[st], (uint32_t)((k / kSStages) & 1), a.err);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) *s_abort = 1;
            k_stop = k;
            break;
        }
        const uint8_t* stage = sm + st * kSStageBytes;
        const int64_t j0 = (int64_t)k * kSJ;
        // packed tiles: rows j0 .. j0 + kSJ cover tile rows j0 / 128 ..; the
        // slice of tile (I, Jt) for I <= Jt
        if (pack && lead && tid == 0) {
            for (int h = 0; h < kSJ / kSTile; ++h) {
                const int I = (int)(j0 / kSTile) + h;
                if (I <= Jt && I < a.nt)
                    msp::tc::tma_store_2d(&tmP, (int32_t)(i0 % kSTile), (int32_t)(tile_index(I, Jt, a.nt) * kSTile),
                                          stage + h * kSTile * kSR * 4);
            }
            msp::tc::bulk_commit();
        }
        // gathers of this column's entries in the chunk
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (e0 + u < e1) {
                const int32_t v = v3[u];
                gather_row(acc, stage + ((v >> 1) - (int32_t)j0) * (kSR * 4), lrot, (v & 1) ? -1.f : 1.f);
            }
        }
        for (int e = e0 + 3; e < e1; ++e) {
            const int32_t v = __ldg(&a.ent[e]);
            gather_row(acc, stage + ((v >> 1) - (int32_t)j0) * (kSR * 4), lrot, (v & 1) ? -1.f : 1.f);
        }
        e0 = e1;
        __syncthreads();
        // every warp is past chunk k: refill its stage with chunk k + kSStages
        if (tid == 0 && k + kSStages < nch) {
            if (pack && lead) msp::tc::bulk_wait_read();
            msp::tc::fence_proxy_async();
            issue(k + kSStages, st);
            issued = k + kSStages + 1;
        }
    }
    if (*s_abort) {
        // bounded waits for the loads still in flight (chunks k_stop ..
        // issued - 1, none of them waited for yet) before the block exits
        if (tid == 0)
            for (int k = k_stop; k < issued; ++k)
                msp::mbar_wait_timed(&full[k % kSStages], (uint32_t)((k / kSStages) & 1), a.err);
        if (tid == 0 && pack && lead) msp::tc::bulk_wait_all();
        return;
    }
    if (tid == 0 && pack && lead) msp::tc::bulk_wait_all();
    // C rows i0 + 4 ((q + lane) mod 8) + t of column c
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

}  // namespace

bool msp_sketch_sym_ok(const void* A, int64_t n, int64_t lda, int64_t s_pad, int gamma) {
    const int64_t groups = (s_pad + 1023) / 1024;
    return msp_tensor_map_encoder() != nullptr && ((uintptr_t)A & 15) == 0 && lda % 4 == 0 && n >= kSR &&
           s_pad % 64 == 0 && s_pad <= 2048 && s_pad % groups == 0 && (s_pad / groups) % 32 == 0 &&
           gamma >= 1 && n < (1ll << 30);
}

msp_status msp_sketch_sym_pass(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t s_pad,
                               const int32_t* ptr, const int32_t* ent, int gamma, float* C, float* packed) {
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
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, (size_t)s_pad * (nch + 1) * 4, &scr));
    int32_t* tab = (int32_t*)scr;
    MSP_TRY(msp_chunk_starts(ctx, ptr, ent, s_pad, kSJ, nch, tab));
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
    a.tab = tab;
    a.ent = ent;
    a.scale = (float)(1.0 / std::sqrt((double)gamma));
    a.C = C;
    CtlBlock* ctl = (CtlBlock*)ctx->ctl;
    a.err = &ctl->error;
    const size_t smem = (size_t)kSStages * kSStageBytes + 64 + 1024;
    MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sketch_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(&ctl->error, 0, sizeof(int), ctx->stream));
    // grid: column groups x every 32-column block up to the last tile column
    // (blocks past n only write the zero padding of the packed tiles)
    dim3 grid((unsigned)groups, (unsigned)((int64_t)nt * kSTile / kSR));
    k_sketch_sym<<<grid, threads, smem, ctx->stream>>>(tmA, tmP, a, packed ? 1 : 0);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

extern "C" msp_status msp_set_sketch_one_pass(msp_ctx* ctx, int on) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    ctx->sketch_sym = on != 0;
    return MSP_OK;
}
