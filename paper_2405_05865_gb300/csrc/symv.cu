// Packed symmetric A pass on sm_103a: q = (A + lam I) p reading each of the
// n(n+1)/2 distinct entries of the symmetric A once.
//
// Storage: A is packed once (per sketch) into the upper-triangular 128 x 128
// tiles (I <= J), tile (I, J) at index I*nt - I*(I-1)/2 + (J - I), each tile a
// contiguous row-major 128 x 128 FP32 block (64 KB), zero-padded past n.
//
// k_symv_packed: one persistent block per SM. Warp 8 is the producer: it
// streams the block's tiles (round-robin over the tile list) into a 3-stage
// shared-memory ring with cp.async.bulk, each stage completed on an mbarrier
// by the copy engine's byte count. Warps 0-7 consume: for tile (I, J) they
// form rowpart = A_IJ p_J (contribution to q_I) and, off the diagonal,
// colpart = A_IJ^T p_I (contribution to q_J). Partials go to
//   part[slot][segment]:  rowpart -> part[J][I], colpart -> part[I][J],
// each (slot, segment) written exactly once, so q_i = sum_slot part[slot][i]
// + lam p_i is formed deterministically by the consumer of q. The block
// partials of p^T (A + lam I) p = sum_tiles (2 - [I==J]) p_I^T A_IJ p_J +
// lam |p|^2 are combined by the last block, which writes alpha = rz / pq.
// Every wait on an mbarrier is bounded in wall-clock time (MSP_ETIMEOUT).
#include "msp_internal.cuh"

#include <atomic>

namespace {

constexpr int kTile = 128;
constexpr int kStages = 3;
constexpr int kConsumerWarps = 8;
constexpr int kSymvThreads = (kConsumerWarps + 1) * 32;
constexpr int kTileBytes = kTile * kTile * 4;
constexpr int kChunk = 16384;                 // bytes per bulk copy (4 per tile)
// a stage holds the tile and the two 128-float segments p_I and p_J
constexpr int kStageBytes = kTileBytes + 2 * kTile * 4;
constexpr size_t kSymvSmem =
    (size_t)kStages * kStageBytes + (size_t)kStages * kConsumerWarps * kTile * 4 + 1024;

__device__ inline uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ inline void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and *err = MSP_ETIMEOUT) after kWaitLimitNs.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = msp::globaltimer_ns();
    for (int spins = 0;; ++spins) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spins & 63) == 63) {
            if (msp::globaltimer_ns() - t0 > msp::kWaitLimitNs) {
                atomicExch(err, (int)MSP_ETIMEOUT);
                return false;
            }
        }
    }
}

__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Same, with an L2 eviction-priority policy (evict-first for data read once).
__device__ inline void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                     uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
        "%2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ inline uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// tile index -> (I, J), I <= J, row-major over the upper triangle
__device__ inline void tile_coords(int t, int nt, int& I, int& J) {
    // I = largest i with start(i) <= t, start(i) = i*nt - i*(i-1)/2
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

// Pack the upper tiles [tile0, tile0 + count) of dense row-major A (n x n,
// lda) into `packed`; a block takes tiles tile0 + blockIdx.x, + gridDim.x, ...
__global__ void __launch_bounds__(256) k_pack_upper(const float* __restrict__ A, int64_t lda,
                                                   int64_t n, int nt, int tile0, int count,
                                                   float* __restrict__ packed) {
    constexpr int kPer = kTile * kTile / 4 / 256;     // float4 per thread per tile (16)
    for (int tix = tile0 + (int)blockIdx.x; tix < tile0 + count; tix += (int)gridDim.x) {
        int I, J;
        tile_coords(tix, nt, I, J);
        float* dst = packed + (int64_t)tix * kTile * kTile;
        const int64_t r0 = (int64_t)I * kTile, c0 = (int64_t)J * kTile;
        const bool vec = (lda % 4 == 0) && (((uintptr_t)A & 15) == 0) && (c0 + kTile <= n);
        // four loads in flight per thread before their stores
        for (int g = 0; g < kPer; g += 4) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = (g + u) * 256 + (int)threadIdx.x;
                const int r = e / (kTile / 4), c4 = (e % (kTile / 4)) * 4;
                const int64_t gr = r0 + r, gc = c0 + c4;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gr < n) {
                    if (vec) {
                        v[u] = __ldcs(reinterpret_cast<const float4*>(A + gr * lda + gc));
                    } else {
                        if (gc + 0 < n) v[u].x = A[gr * lda + gc + 0];
                        if (gc + 1 < n) v[u].y = A[gr * lda + gc + 1];
                        if (gc + 2 < n) v[u].z = A[gr * lda + gc + 2];
                        if (gc + 3 < n) v[u].w = A[gr * lda + gc + 3];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) reinterpret_cast<float4*>(dst)[(g + u) * 256 + (int)threadIdx.x] = v[u];
        }
    }
}

struct SymvArgs {
    const float* packed;
    int nt;                 // tiles per side
    int ntiles;             // nt (nt + 1) / 2
    int64_t n;
    int64_t n_pad;          // nt * 128 (length of p, segment space of part)
    float lam;
    const float* p;         // n_pad, zero past n
    float* part;            // nt x n_pad
    double* dpart;          // gridDim.x
    CtlBlock* ctl;
};

__global__ void __launch_bounds__(kSymvThreads, 1) k_symv_packed(SymvArgs a) {
    CtlBlock* ctl = a.ctl;
    if (ctl->done | ctl->error) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = smem_raw;                                        // kStages stages
    float* colred = reinterpret_cast<float*>(smem_raw + (size_t)kStages * kStageBytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(colred + (size_t)kStages * kConsumerWarps * kTile);
    uint64_t* empty = full + kStages;
    __shared__ double red[32];
    __shared__ bool am_last;
    __shared__ int s_abort;
    __shared__ int col_count[kStages];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
            col_count[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();

    const int G = gridDim.x;
    // tiles of this block: t = blockIdx.x + k G
    const int my_tiles = (a.ntiles > (int)blockIdx.x) ? (a.ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    double acc_dot = 0.0;

    if (warp == kConsumerWarps) {
        // ---------------- producer
        if (lane == 0) {
            int issued = 0;
            const uint64_t pol = policy_evict_first();
            for (int k = 0; k < my_tiles; ++k) {
                const int s = k % kStages;
                const uint32_t ph = (uint32_t)((k / kStages) & 1);
                if (k >= kStages) {
                    // wait until the consumers released this stage (use k - kStages)
                    if (!mbar_wait(&empty[s], ph ^ 1u, &ctl->error)) { s_abort = 1; break; }
                }
                const int t = (int)blockIdx.x + k * G;
                int I, J;
                tile_coords(t, a.nt, I, J);
                const char* src = reinterpret_cast<const char*>(a.packed) + (size_t)t * kTileBytes;
                unsigned char* dst = ring + (size_t)s * kStageBytes;
                mbar_arrive_expect_tx(&full[s], kStageBytes);
#pragma unroll
                for (int c = 0; c < kTileBytes / kChunk; ++c)
                    bulk_g2s_hint(dst + c * kChunk, src + c * kChunk, kChunk, &full[s], pol);
                bulk_g2s(dst + kTileBytes, a.p + (int64_t)I * kTile, kTile * 4, &full[s]);
                bulk_g2s(dst + kTileBytes + kTile * 4, a.p + (int64_t)J * kTile, kTile * 4, &full[s]);
                issued = k + 1;
            }
            // drain: every issued copy must have landed before the block exits
            for (int k = (issued > kStages ? issued - kStages : 0); k < issued; ++k) {
                const int s = k % kStages;
                const uint32_t ph = (uint32_t)((k / kStages) & 1);
                if (!mbar_wait(&full[s], ph, &ctl->error)) break;
            }
        }
    } else {
        // ---------------- consumers
        const int ct = threadIdx.x;                 // 0..255
        for (int k = 0; k < my_tiles; ++k) {
            const int s = k % kStages;
            const uint32_t ph = (uint32_t)((k / kStages) & 1);
            if (!mbar_wait(&full[s], ph, &ctl->error)) { s_abort = 1; break; }
            const int t = (int)blockIdx.x + k * G;
            int I, J;
            tile_coords(t, a.nt, I, J);
            const float* tb = reinterpret_cast<const float*>(ring + (size_t)s * kStageBytes);
            const float* pI = tb + kTile * kTile;            // p_I staged with the tile
            const float4 pj = reinterpret_cast<const float4*>(pI + kTile)[lane];
            float rv[16];
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int r = warp + kConsumerWarps * kk;
                const float4 v = reinterpret_cast<const float4*>(tb + r * kTile)[lane];
                rv[kk] = v.x * pj.x + v.y * pj.y + v.z * pj.z + v.w * pj.w;
                const float pr = pI[r];
                c0 += v.x * pr;
                c1 += v.y * pr;
                c2 += v.z * pr;
                c3 += v.w * pr;
            }
            // column partials: each warp fills its slot of this stage's buffer;
            // the last of the 8 warps to finish sums the slots in warp order
            // (deterministic) before it releases the stage, so the buffer is
            // never rewritten while being read and no warp ever blocks
            float* cr = colred + (size_t)s * kConsumerWarps * kTile;
            reinterpret_cast<float4*>(cr + warp * kTile)[lane] = make_float4(c0, c1, c2, c3);
            __syncwarp();
            int arrived = 0;
            if (lane == 0) {
                __threadfence_block();
                arrived = atomicAdd(&col_count[s], 1);
            }
            arrived = __shfl_sync(0xffffffffu, arrived, 0);
            if (arrived == kConsumerWarps - 1) {
                __threadfence_block();
                if (I != J) {
#pragma unroll
                    for (int q = 0; q < kTile / 32; ++q) {
                        const int c = lane + 32 * q;
                        float v = 0.f;
#pragma unroll
                        for (int w = 0; w < kConsumerWarps; ++w) v += cr[w * kTile + c];
                        a.part[(int64_t)I * a.n_pad + (int64_t)J * kTile + c] = v;
                    }
                }
                __syncwarp();
                if (lane == 0) col_count[s] = 0;
            }
            // transpose-reduce the 16 row partials across the warp
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const bool up = (lane >> 4) & 1;
                float send = up ? rv[kk] : rv[kk + 8];
                float keep = up ? rv[kk + 8] : rv[kk];
                rv[kk] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const bool up = (lane >> 3) & 1;
                float send = up ? rv[kk] : rv[kk + 4];
                float keep = up ? rv[kk + 4] : rv[kk];
                rv[kk] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const bool up = (lane >> 2) & 1;
                float send = up ? rv[kk] : rv[kk + 2];
                float keep = up ? rv[kk + 2] : rv[kk];
                rv[kk] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            {
                const bool up = (lane >> 1) & 1;
                float send = up ? rv[0] : rv[1];
                float keep = up ? rv[1] : rv[0];
                rv[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
            rv[0] += __shfl_xor_sync(0xffffffffu, rv[0], 1);
            const float w_tile = (I == J) ? 1.f : 2.f;
            float tdot = 0.f;
            if ((lane & 1) == 0) {
                const int r = warp + kConsumerWarps * (lane >> 1);
                a.part[(int64_t)J * a.n_pad + (int64_t)I * kTile + r] = rv[0];
                tdot = pI[r] * rv[0];
            }
            // this warp's 16 rows of p_I^T A_IJ p_J: FP32 within the tile, one
            // FP64 add per warp and tile
            tdot = msp::warp_sum(tdot);
            if (lane == 0) acc_dot += (double)(w_tile * tdot);
            // stage (tile and column buffer) consumed: release it to the producer
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        // lam |p|^2 over a slice of p
        const int64_t i0 = a.n * blockIdx.x / G, i1 = a.n * (blockIdx.x + 1) / G;
        for (int64_t i = i0 + ct; i < i1; i += kConsumerWarps * 32) {
            const double pv = (double)a.p[i];
            acc_dot += (double)a.lam * pv * pv;
        }
    }
    // block partial of p^T (A + lam I) p, then the last block forms alpha
    double v = msp::warp_sum(acc_dot);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kConsumerWarps + 1; ++w) tot += red[w];
        a.dpart[blockIdx.x] = tot;
        __threadfence();
        unsigned int tk = atomicAdd(&ctl->last_block_counter, 1u);
        am_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the G block partials with all loads in flight together (not one
    // thread's chain of L2 round trips): strided per thread, then the warp
    // tree and the warps in order (a fixed order)
    double all = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) all += __ldcg(&a.dpart[b]);
    all = msp::warp_sum(all);
    __syncthreads();
    if (lane == 0) red[warp] = all;
    __syncthreads();
    if (threadIdx.x == 0) {
        all = 0.0;
        for (int w = 0; w < kConsumerWarps + 1; ++w) all += red[w];
        ctl->last_block_counter = 0;
        ctl->pq = all;
        if (s_abort) { /* error already recorded */ }
        else if (!isfinite(all)) ctl->error = MSP_ENONFINITE;
        else if (!(all > 0.0)) ctl->error = MSP_ENOTPD;
        else ctl->alpha = ctl->rz / all;
    }
}

}  // namespace

int64_t msp_packed_tiles(int64_t n) {
    const int64_t nt = (n + kTile - 1) / kTile;
    return nt * (nt + 1) / 2;
}

msp_status msp_pack_upper(msp_ctx* ctx, const float* A, int64_t lda, int64_t n, float* packed) {
    const int64_t nt = (n + kTile - 1) / kTile;
    const int64_t ntiles = nt * (nt + 1) / 2;
    if (ntiles >= (1ll << 31)) return msp_set_error(ctx, MSP_EINVAL, "pack: n too large");
    k_pack_upper<<<(unsigned)ntiles, 256, 0, ctx->stream>>>(A, lda, n, (int)nt, 0, (int)ntiles, packed);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// The lower triangle of a symmetric row-major A from its upper triangle (the
// diagonal included): A[i][j] = A[j][i] for i > j. One 128 x 128 tile (I, J),
// J <= I, per block, tile t = I (I + 1) / 2 + J; on a diagonal tile only the
// entries below the diagonal are written. 32 x 33 shared-memory transposes,
// coalesced both ways.
__global__ void __launch_bounds__(256) k_mirror_lower(float* __restrict__ A, int64_t lda, int64_t n, int t0) {
    __shared__ float tr[32][33];
    // tiles (I, J) with J <= I, tile row after tile row: row I starts at I (I + 1) / 2
    const int t = t0 + (int)blockIdx.x;
    int I = (int)((sqrtf(1.0f + 8.0f * (float)t) - 1.0f) * 0.5f);
    while (I > 0 && (int64_t)I * (I + 1) / 2 > t) --I;
    while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
    const int J = t - I * (I + 1) / 2;
    const bool diag = (I == J);
    const int64_t r0 = (int64_t)I * kTile, c0 = (int64_t)J * kTile;   // destination block (rows r0.., cols c0..)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;             // 32 x 8
    for (int bi = 0; bi < kTile; bi += 32)
        for (int bj = 0; bj < kTile; bj += 32) {
            if (diag && bj > bi) continue;          // block-uniform: the upper half of a diagonal tile stays
            // read the source block A[c0 + bj + y][r0 + bi + x] (rows of the upper tile)
            for (int y = ty; y < 32; y += 8) {
                const int64_t sr = c0 + bj + y, sc = r0 + bi + tx;
                tr[y][tx] = (sr < n && sc < n) ? A[sr * lda + sc] : 0.f;
            }
            __syncthreads();
            // on a diagonal tile only the strictly lower entries are written; their
            // sources lie strictly above the diagonal and are never written
            for (int y = ty; y < 32; y += 8) {
                const int64_t dr = r0 + bi + y, dc = c0 + bj + tx;
                if (dr < n && dc < n && (!diag || dr > dc)) A[dr * lda + dc] = tr[tx][y];
            }
            __syncthreads();
        }
}

// Fills the lower triangle of tile rows [I0, I1) (the diagonal tiles included)
// from the upper triangle, which must already be in place for those rows and
// for every row above them.
msp_status msp_mirror_lower_rows(msp_ctx* ctx, float* A, int64_t lda, int64_t n, int64_t I0, int64_t I1) {
    const int64_t nt = (n + kTile - 1) / kTile;
    I1 = std::min(I1, nt);
    if (I0 >= I1) return MSP_OK;
    const int64_t t0 = I0 * (I0 + 1) / 2, t1 = I1 * (I1 + 1) / 2;
    k_mirror_lower<<<(unsigned)(t1 - t0), 256, 0, ctx->stream>>>(A, lda, n, (int)t0);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// The tiles whose tile row lies in [I0, I1): contiguous in the packed order
// (tile rows one after another), and they read only rows [I0, I1) * 128 of A.
msp_status msp_pack_upper_rows(msp_ctx* ctx, const float* A, int64_t lda, int64_t n, int64_t I0, int64_t I1,
                               float* packed) {
    const int64_t nt = (n + kTile - 1) / kTile;
    if (I0 < 0 || I1 > nt || I0 >= I1) return MSP_OK;
    auto start = [&](int64_t i) { return i * nt - i * (i - 1) / 2; };
    const int64_t t0 = start(I0), t1 = start(I1);
    k_pack_upper<<<(unsigned)(t1 - t0), 256, 0, ctx->stream>>>(A, lda, n, (int)nt, (int)t0, (int)(t1 - t0), packed);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_symv_packed(msp_ctx* ctx, const float* packed, int64_t n, float lam, const float* p,
                           float* part, double* dpart, int grid) {
    // the attribute belongs to a device: set once per device (bit of a mask)
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (!(attr_set.load() & bit)) {
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_symv_packed,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSymvSmem));
        attr_set.fetch_or(bit);
    }
    SymvArgs a;
    a.packed = packed;
    a.nt = (int)((n + kTile - 1) / kTile);
    a.ntiles = a.nt * (a.nt + 1) / 2;
    a.n = n;
    a.n_pad = (int64_t)a.nt * kTile;
    a.lam = lam;
    a.p = p;
    a.part = part;
    a.dpart = dpart;
    a.ctl = (CtlBlock*)ctx->ctl;
    k_symv_packed<<<grid, kSymvThreads, kSymvSmem, ctx->stream>>>(a);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}
