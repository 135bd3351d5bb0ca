// Sparse sketches of Algorithm 1 on sm_103a:
//   * the pattern of a sparse embedding (Definition 2.1),
//   * its transpose as CSR (the list of (j, sign) per sketch column c),
//   * C = A Pi (Pi = S^T): one pass over A, gathering each output column's
//     ~n*gamma/s source columns from a shared-memory tile of A,
//   * row gathers out[r,:] = scale * sum_{(j,sign) in list(r)} sign * in[j,:],
//     which give W = Pi^T C = S C and C~ = Phi C.
#include "msp_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace {

// ---------------------------------------------------------------- pattern

// One thread per column j of the embedding (row j of Pi). Floyd's sampling:
// for q = 0..gamma-1, t = rows - gamma + q, r = mulhi(u_q, t + 1) in [0, t];
// keep r unless already chosen, else keep t. Then sort ascending and draw the
// sign of the q-th smallest from the top bit of draw(stream + 1, j, q).
__global__ void k_pattern(int64_t n, int rows, int gamma, uint64_t seed, int stream,
                          int32_t* __restrict__ idx, int8_t* __restrict__ sgn,
                          int32_t* __restrict__ counts) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c[MSP_MAX_GAMMA];
    for (int q = 0; q < gamma; ++q) {
        uint64_t t = (uint64_t)(rows - gamma + q);
        uint64_t u = msp::draw(seed, (uint32_t)stream, (uint64_t)j, (uint32_t)q);
        int r = (int)__umul64hi(u, t + 1ull);
        bool seen = false;
        for (int k = 0; k < q; ++k) seen |= (c[k] == r);
        c[q] = seen ? (int)t : r;
    }
    for (int a = 1; a < gamma; ++a) {          // insertion sort, gamma <= 64
        int v = c[a], b = a - 1;
        while (b >= 0 && c[b] > v) { c[b + 1] = c[b]; --b; }
        c[b + 1] = v;
    }
    for (int q = 0; q < gamma; ++q) {
        uint64_t u = msp::draw(seed, (uint32_t)(stream + 1), (uint64_t)j, (uint32_t)q);
        idx[j * gamma + q] = c[q];
        sgn[j * gamma + q] = (u >> 63) ? (int8_t)-1 : (int8_t)1;
        if (counts) atomicAdd(&counts[c[q]], 1);
    }
}

// counts[c] = number of pattern entries equal to c
__global__ void k_hist(int64_t m, const int32_t* __restrict__ idx, int32_t* __restrict__ counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) atomicAdd(&counts[idx[i]], 1);
}

// Exclusive scan of counts[0..m) into ptr[0..m], single block.
__global__ void k_scan(const int32_t* __restrict__ counts, int64_t m, int32_t* __restrict__ ptr) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < m; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int32_t v = i < m ? counts[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) warp_tot[lane] = t;   // inclusive over warps
        }
        __syncthreads();
        int32_t before = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + x - v;
        if (i < m) ptr[i] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) ptr[m] = carry;
}

// Scatter (j, sign) into each row's bucket (order made canonical below).
__global__ void k_fill(int64_t n, int gamma, const int32_t* __restrict__ idx,
                       const int8_t* __restrict__ sgn, const int32_t* __restrict__ ptr,
                       int32_t* __restrict__ cursor, int32_t* __restrict__ ent) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int q = 0; q < gamma; ++q) {
        int c = idx[j * gamma + q];
        int pos = ptr[c] + atomicAdd(&cursor[c], 1);
        ent[pos] = (int32_t)((j << 1) | (sgn[j * gamma + q] < 0 ? 1 : 0));
    }
}

// Sort every bucket by j (entries in a bucket have distinct j): warp per
// bucket, each entry placed at its rank. Reads `in`, writes `out`.
__global__ void k_sort_buckets(int64_t m, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ in, int32_t* __restrict__ out) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= m) return;
    int lo = ptr[b], hi = ptr[b + 1];
    for (int e = lo + lane; e < hi; e += 32) {
        int32_t v = in[e];
        int32_t jv = v >> 1;
        int rank = 0;
        for (int k = lo; k < hi; ++k) rank += ((in[k] >> 1) < jv);
        out[lo + rank] = v;
    }
}

// ------------------------------------------------------------ C = A Pi

// Block: R rows of A x all s_pad outputs. Thread t owns output columns
// c = t + k*blockDim.x (k < NC) for the R rows (NC*R accumulators). A is
// streamed in chunks of J columns into shared memory transposed to
// tile[jj][0..R), stored as R/VW vectors of VW elements (16 bytes) whose
// order is XOR-swizzled by (jj >> 1) so that the transposing vector stores of
// 8 consecutive columns hit 8 distinct bank groups. One list entry (j, sign)
// then costs R/VW vector loads. Each thread walks its columns' sorted lists
// with a cursor per column.
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int W = 4; };
template <> struct V16<double> { using type = double2; static constexpr int W = 2; };

// Start of every J-row chunk in each column's entry list (entries sorted by
// row): tab[c * (nch + 1) + t] = first entry of column c with row >= t J,
// t = 0..nch. One thread per (column, chunk), binary search.
__global__ void k_chunk_starts(const int32_t* __restrict__ ptr, const int32_t* __restrict__ ent,
                               int64_t s_pad, int J, int nch, int32_t* __restrict__ tab) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * (nch + 1)) return;
    const int64_t c = e / (nch + 1);
    const int tch = (int)(e % (nch + 1));
    int lo = ptr[c], hi = ptr[c + 1];
    const int64_t jt = (int64_t)tch * J;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)(ent[mid] >> 1) < jt) lo = mid + 1;
        else hi = mid;
    }
    tab[e] = lo;
}

// A entry widened to the accumulation type (BF16 storage: exact).
__device__ inline float widen(float v) { return v; }
__device__ inline double widen(double v) { return v; }
__device__ inline float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, int R, int NC, typename TA = T>
__global__ void __launch_bounds__(256) k_sketch_apply(
    const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n, int64_t s_pad,
    const int32_t* __restrict__ tab, int nch, const int32_t* __restrict__ ent, T scale,
    T* __restrict__ C, int J) {
    using VT = typename V16<T>::type;
    constexpr int VW = V16<T>::W;
    constexpr int NV = R / VW;                  // vectors per tile row (4)
    static_assert(NV == 4, "swizzle assumes four 16-byte vectors per tile row");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* tile = reinterpret_cast<VT*>(smem_raw);    // J x NV vectors
    const int64_t i0 = (int64_t)blockIdx.x * R;
    const int nthr = blockDim.x;
    T acc[NC][R];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[k][r] = T(0);
    int chunk = 0;
    for (int64_t j0 = 0; j0 < n; j0 += J, ++chunk) {
        const int jlen = (int)min((int64_t)J, n - j0);
        __syncthreads();
        for (int jj = threadIdx.x; jj < jlen; jj += nthr) {
            T v[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[r] = (i0 + r < m) ? (T)widen(__ldcs(&A[(i0 + r) * lda + j0 + jj])) : T(0);
            const int sw = (jj >> 1) & 3;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                VT x;
                if constexpr (VW == 4) x = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                else x = make_double2(v[2 * q], v[2 * q + 1]);
                tile[jj * NV + (q ^ sw)] = x;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const int c = threadIdx.x + k * nthr;
            const int e0 = __ldg(&tab[(int64_t)c * (nch + 1) + chunk]);
            const int e1 = __ldg(&tab[(int64_t)c * (nch + 1) + chunk + 1]);
            // fixed bounds: the entry loads of a chunk are independent
#pragma unroll 4
            for (int e = e0; e < e1; ++e) {
                const int32_t v = __ldg(&ent[e]);
                const int jl = (v >> 1) - (int32_t)j0;
                const int sw = (jl >> 1) & 3;
                const T sg = (v & 1) ? T(-1) : T(1);
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const VT x = tile[jl * NV + (q ^ sw)];
                    if constexpr (VW == 4) {
                        acc[k][4 * q + 0] = fma(sg, x.x, acc[k][4 * q + 0]);
                        acc[k][4 * q + 1] = fma(sg, x.y, acc[k][4 * q + 1]);
                        acc[k][4 * q + 2] = fma(sg, x.z, acc[k][4 * q + 2]);
                        acc[k][4 * q + 3] = fma(sg, x.w, acc[k][4 * q + 3]);
                    } else {
                        acc[k][2 * q + 0] = fma(sg, x.x, acc[k][2 * q + 0]);
                        acc[k][2 * q + 1] = fma(sg, x.y, acc[k][2 * q + 1]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        int c = threadIdx.x + k * nthr;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (i0 + r < m) C[(i0 + r) * s_pad + c] = acc[k][r] * scale;
    }
}

template <typename T, int R, typename TA = T>
msp_status launch_sketch_apply_r(msp_ctx* ctx, const TA* A, int64_t lda, int64_t m, int64_t n,
                                 int64_t s_pad, const int32_t* ptr, const int32_t* ent,
                                 T scale, T* C) {
    // s_pad is a multiple of 128: the smallest NC with s_pad / NC a multiple
    // of 32 and at most 256 threads (two blocks per SM fit up to NC = 4)
    int nc = 0;
    for (int cand : {1, 2, 3, 4, 6, 8}) {
        if (s_pad % cand == 0 && (s_pad / cand) % 32 == 0 && s_pad / cand <= 256) {
            nc = cand;
            break;
        }
    }
    if (nc == 0)
        return msp_set_error(ctx, MSP_EINVAL, "sketch: unsupported s_pad %lld", (long long)s_pad);
    const int threads = (int)(s_pad / nc);
    const int J = (int)((64 * 1024) / (sizeof(T) * R));
    size_t smem = (size_t)J * R * sizeof(T);
    dim3 grid((unsigned)((m + R - 1) / R));
    const int nch = (int)((n + J - 1) / J);
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, (size_t)s_pad * (nch + 1) * 4, &scr));
    int32_t* tab = (int32_t*)scr;
    {
        const int64_t cnt = s_pad * (nch + 1);
        k_chunk_starts<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(ptr, ent, s_pad, J, nch, tab);
        MSP_CHECK_LAUNCH(ctx);
    }
#define MSP_SK_CASE(NCV)                                                              \
    case NCV: {                                                                       \
        auto kern = k_sketch_apply<T, R, NCV, TA>;                                    \
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(kern,                                  \
                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));        \
        kern<<<grid, threads, smem, ctx->stream>>>(A, lda, m, n, s_pad, tab, nch, ent, \
                                                  scale, C, J);                       \
        break;                                                                        \
    }
    switch (nc) {
        MSP_SK_CASE(1)
        MSP_SK_CASE(2)
        MSP_SK_CASE(3)
        MSP_SK_CASE(4)
        MSP_SK_CASE(6)
        MSP_SK_CASE(8)
        default:
            return msp_set_error(ctx, MSP_EINVAL, "sketch: unsupported s_pad %lld",
                                 (long long)s_pad);
    }
#undef MSP_SK_CASE
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// ------------------------------------------------------------ row gathers

// out[r, c] = scale * sum_{(j,neg) in list(r)} (+-) in[j, c]; block per output
// row, threads over columns.
template <typename T>
__global__ void k_gather_rows(int64_t rows_out, int64_t width, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ ent, const T* __restrict__ in,
                              int64_t ld_in, T scale, T* __restrict__ out, int64_t ld_out) {
    int64_t r = blockIdx.x;
    if (r >= rows_out) return;
    const int lo = ptr[r], hi = ptr[r + 1];
    for (int64_t c = threadIdx.x; c < width; c += blockDim.x) {
        T acc = T(0);
        for (int e = lo; e < hi; ++e) {
            int32_t v = __ldg(&ent[e]);
            T a = in[(int64_t)(v >> 1) * ld_in + c];
            acc += (v & 1) ? -a : a;
        }
        out[r * ld_out + c] = acc * scale;
    }
}

}  // namespace

// ------------------------------------------------------------- host side

msp_status msp_pattern_launch(msp_ctx* ctx, int64_t n, int64_t rows, int gamma,
                              uint64_t seed, int stream, int32_t* idx, int8_t* sgn,
                              int32_t* counts) {
    if (n <= 0 || rows <= 0 || gamma < 1 || gamma > MSP_MAX_GAMMA || gamma > rows ||
        n >= (1ll << 30) || rows >= (1ll << 30) || stream < 0 || stream > 254)
        return msp_set_error(ctx, MSP_EINVAL,
                             "pattern: need 1 <= gamma <= min(rows, %d), n, rows < 2^30",
                             MSP_MAX_GAMMA);
    int threads = 256;
    k_pattern<<<(unsigned)((n + threads - 1) / threads), threads, 0, ctx->stream>>>(
        n, (int)rows, gamma, seed, stream, idx, sgn, counts);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_build_csr(msp_ctx* ctx, int64_t n, int64_t rows, int gamma,
                         const int32_t* idx, const int8_t* sgn, int32_t* ptr,
                         int32_t* ent) {
    // counts, cursor and an unsorted copy of the entries live in scratch
    size_t need = (size_t)rows * 4 * 2 + (size_t)n * gamma * 4;
    void* scr = nullptr;
    MSP_TRY(msp_scratch(ctx, need, &scr));
    int32_t* counts = (int32_t*)scr;
    int32_t* cursor = counts + rows;
    int32_t* tmp = cursor + rows;
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(counts, 0, (size_t)rows * 8, ctx->stream));
    {
        const int threads = 256;
        int64_t m = n * gamma;
        k_hist<<<(unsigned)((m + threads - 1) / threads), threads, 0, ctx->stream>>>(m, idx, counts);
        MSP_CHECK_LAUNCH(ctx);
    }
    k_scan<<<1, 1024, 0, ctx->stream>>>(counts, rows, ptr);
    MSP_CHECK_LAUNCH(ctx);
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, gamma, idx, sgn, ptr,
                                                                  cursor, tmp);
    MSP_CHECK_LAUNCH(ctx);
    int64_t warps = rows;
    k_sort_buckets<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, ctx->stream>>>(rows, ptr,
                                                                                  tmp, ent);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_sketch_apply(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n,
                            int64_t lda, int64_t s_pad, const int32_t* ptr,
                            const int32_t* ent, int gamma, void* C) {
    return msp_sketch_apply_rows(ctx, A, dt, n, n, lda, s_pad, ptr, ent, gamma, C);
}

msp_status msp_sketch_apply_rows(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t m, int64_t n,
                                 int64_t lda, int64_t s_pad, const int32_t* ptr,
                                 const int32_t* ent, int gamma, void* C) {
    // accumulators per thread: R rows x NC columns; R = 4 vectors of 16 bytes
    double scale = 1.0 / sqrt((double)gamma);
    if (s_pad > (dt != MSP_F64 ? MSP_MAX_S_SINGLE : 1024))
        return msp_set_error(ctx, MSP_EINVAL, "sketch: s_pad %lld above the supported maximum",
                             (long long)s_pad);
    if (dt == MSP_F32)
        return launch_sketch_apply_r<float, 16>(ctx, (const float*)A, lda, m, n, s_pad, ptr, ent,
                                                (float)scale, (float*)C);
    if (dt == MSP_BF16)   // BF16 A read, FP32 accumulation and C
        return launch_sketch_apply_r<float, 16, __nv_bfloat16>(ctx, (const __nv_bfloat16*)A, lda, m, n, s_pad,
                                                               ptr, ent, (float)scale, (float*)C);
    return launch_sketch_apply_r<double, 8>(ctx, (const double*)A, lda, m, n, s_pad, ptr, ent,
                                            scale, (double*)C);
}

msp_status msp_chunk_starts(msp_ctx* ctx, const int32_t* ptr, const int32_t* ent, int64_t s_pad, int J, int nch,
                            int32_t* tab) {
    const int64_t cnt = s_pad * (nch + 1);
    k_chunk_starts<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(ptr, ent, s_pad, J, nch, tab);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

msp_status msp_gather_rows(msp_ctx* ctx, msp_dtype dt, int64_t rows_out, int64_t width,
                           const int32_t* ptr, const int32_t* ent, const void* in,
                           int64_t ld_in, double scale, void* out, int64_t ld_out) {
    int threads = (int)std::min<int64_t>(1024, round_up(width, 32));
    if (dt == MSP_F32)
        k_gather_rows<float><<<(unsigned)rows_out, threads, 0, ctx->stream>>>(
            rows_out, width, ptr, ent, (const float*)in, ld_in, (float)scale, (float*)out, ld_out);
    else
        k_gather_rows<double><<<(unsigned)rows_out, threads, 0, ctx->stream>>>(
            rows_out, width, ptr, ent, (const double*)in, ld_in, scale, (double*)out, ld_out);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}
