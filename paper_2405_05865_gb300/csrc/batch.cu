// Batched MSP (many instances, up to 16 right-hand sides each) on sm_103a.
//
// Set-up (msp_batch_create): the sketch, W, M2 and its factor of every
// instance (Algorithm 1 steps 1-4) are built by worker contexts, one host
// thread and one stream each, so the small latency-bound factor kernels of
// different instances overlap on the GPU. Each A is then copied into the
// tile layout of the batched A pass: 128 x 64 FP32 tiles, tile (I, K) of
// row block I and column block K at (I * nk + K) * 8192 floats, each tile
// contiguous (32 KB, one bulk copy), zero-padded to n_pad = ceil(n/128)*128,
// with the 16-byte granule g of row r stored at granule g ^ (r & 7) so that
// eight lanes reading one granule column of eight rows hit distinct banks.
//
// Solve (msp_batch_solve): ONE persistent cooperative kernel, one block per
// SM, runs every step for every (instance, column) until all columns meet
// the tolerance. Vectors are [n_pad][16] FP32 rows per instance (column c of
// the 16 is right-hand side c), concatenated over instances. Per level-1
// iteration t (flexible PCG, Section 6; preconditioner SolveM1 with the
// direct level 2, Section 4):
//   S2  G = C^T R            items (instance, 64-column strip of C)
//       + convergence flags  one block per instance decides, fixed order
//   S3  Y1 = L^{-1} G        items (instance, 128-row chunk of s)
//   S4  Y2 = L^{-T} Y1
//   S5  Z = (R - C Y2)/lam~  items (instance, 128-row block), dots z.r, z.q
//   S6  beta, P = Z + beta P
//   SA  Q = (A + lam I) P    dynamic items over the row blocks: a producer
//                            warp streams A tiles + P slices by bulk copy
//                            into a 4-stage mbarrier ring; each of 8 warps
//                            takes 8 of the 64 columns of a tile for all 128
//                            rows on the tensor cores (mma.sync m16n8k8 TF32,
//                            split 3xTF32 for FP32 accuracy): FP32 FMA at 16
//                            products per loaded element could not keep up
//                            with HBM. The level-2 mat-vecs stay on FP32 FMA
//                            (see fma_tile).
//   S1  alpha, X_w += alpha P, R -= alpha Q
// with a grid barrier between steps. Around it, the FP64 refinement
// (MSP_PREC_MIXED): R64 = B - (A + lam I) X is formed by the same tile
// stream with compensated FP32 products (x = x_hi + x_lo, TwoProduct and
// TwoSum per term, FP64 combination), the correction solve starts from
// R64 / |R64| per column, and X += |R64| X_w. Every scalar of a column is
// its own (no coupling between columns). All reductions use a fixed order.
#include "msp_internal.cuh"
#include "bulk.cuh"

#include <algorithm>
#include <map>
#include <tuple>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

namespace {

constexpr int kM = 16;                          // right-hand sides per instance (padded)
constexpr int kRB = 128;                        // rows per row block
constexpr int kKT = 64;                         // columns per k tile
constexpr int kWorkWarps = 8;
constexpr int kWorkers = kWorkWarps * 32;       // 256
constexpr int kThreads = kWorkers + 32;         // + producer warp
constexpr int kStages = 4;
constexpr int kTileFloats = kRB * kKT;          // 8192
constexpr int kTileBytes = kTileFloats * 4;     // 32 KB
constexpr int kSliceFloats = kKT * kM;          // 1024
constexpr int kSliceBytes = kSliceFloats * 4;   // 4 KB
constexpr int kStageBytes = kTileBytes + 2 * kSliceBytes;
// A unit of the streamed A passes is one 128-row block times at most
// BArgs::ut tiles (ut x 64 columns); smaller units balance a pass across the
// SMs better, larger ones pay the per-unit reduction less often. The width
// is a run-time choice (msp_batch_autotune); kUtMin bounds the partial
// buffers.
constexpr int kUtMin = 16;
constexpr int kRingBytes = kStages * kStageBytes;   // 160 KB
constexpr int kRedBytes = 65536;
constexpr int kMiscBytes = 2048;
constexpr size_t kSmem = (size_t)kRingBytes + kRedBytes + kMiscBytes;
// smem map of the mat-vec steps (S3-S5): 3 tiles, the staged vector block
constexpr int kMvTiles = 3;
constexpr int kVsOffset = kMvTiles * kTileBytes;          // 96 KB

// device-timer classes of BCtl::t_ns
enum { kTA = 0, kTG, kTTri, kTZ, kTVec, kTResid, kTCheck, kTimerClasses };

struct BInst {
    const float* At;      // tile-major A
    const float* Ct;      // tile-major C (n_pad x s_pad)
    const float* C;       // n x s_pad
    const float* Bl;      // L^{-1}, s_pad x s_pad (lower)
    const float* Bu;      // L^{-T} (upper)
    const double* B;
    double* X;
    int64_t ldb, ldx;
    int n, n_pad, s_pad, m;
    int nb;               // row blocks n_pad / 128
    int nkc;              // units per row block: ceil(n_pad / 64 / ut)
    int qoff;             // first row of the instance in the unit-partial arrays
    int voff;             // first row in the [.][16] vector arrays
    int soff;             // first row in the s-length arrays
    int boff;             // first row block in the partial arrays
    float lam, inv_lt;
    double lam64;
};

struct BCtl {
    unsigned int bar_word, bar_spare;     // grid barrier: generation << 16 | arrivals
    int error;
    int ctrA, ctrR;
    int active[2];
    int unfinished[2];
    int sweepsA, sweepsR;     // A passes and residual passes run
    int ctrG, ctrT1, ctrT2, ctrZ;   // dynamic item counters of S2, S3, S4, S5
    int pad0;
    unsigned long long tilesA;   // A tiles streamed by the level-1 passes
    unsigned long long tilesR;   // A tiles streamed by the residual passes
    unsigned long long bytesG;   // C bytes read by G = C^T R
    unsigned long long bytesZ;   // C bytes read by Z = (R - C Y) / lambda~
    // device-timer nanoseconds per step class, taken by block 0 between grid
    // barriers (each includes its barrier)
    unsigned long long t_ns[kTimerClasses];
};

struct BArgs {
    const BInst* inst;
    int count, nrows, nstrips, nchunks;
    const int2* rows;     // (instance, row block), largest n first
    const int2* strips;   // (instance, 64-column strip of C)
    const int2* chunks;   // (instance, 128-row chunk of s)
    int nunits;
    int ut;               // tiles per unit
    const int2* units;    // (instance, row block | unit << 16), largest first
    float* Qp;            // [nkc][n_pad][16] partial A P per unit
    double* Rp;           // [nkc][n_pad][16] partial A X per unit (residual)
    int* rbcnt;           // per row block: units finished in the current pass
    float *P, *Q, *R, *Z, *XW, *XH, *XL;
    double* R64;
    float *G, *Y1, *Y2;
    double *p_pq, *p_rr, *p_zr, *p_zq, *p_r64, *p_xx;
    double *bb, *scale, *alpha, *rz;    // per column; rz holds two generations
    int *act, *fin;                     // per column
    int *iact;                          // two generations x count
    int *istep, *iters, *ierr, *isteps; // per instance
    double* rel;                        // per instance: largest |r| / |b|
    double* berr;                       // per instance: largest backward-error bound
    const double* anorm;                // per instance: L <= |A|_2
    BCtl* ctl;
    double tol, tol2, rtol2;
    int max_outer, max_steps, crit;
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__device__ __forceinline__ float comp(const float4& v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// ------------------------------------------------------------ tile math

// acc[i][c] += sum over the warp's 8 columns k of the tile of T[lane+32i][k] V[k][c]
// in FP32 FMA (the level-2 mat-vecs: the Woodbury form (r - C M2^{-1} C^T r)
// cancels up to lambda_max / lambda~, so these keep FP32 rounding).
// T: 128 x 64 swizzled tile; V: 64 rows of 16.
__device__ __forceinline__ void fma_tile(float (&acc)[4][16], const float* __restrict__ T,
                                         const float* __restrict__ V, int w, int lane) {
    const float4* T4 = reinterpret_cast<const float4*>(T);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const int sw = lane & 7;
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
        const int g = 2 * w + gi;
        float4 a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = T4[(lane + 32 * i) * 16 + (g ^ sw)];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int k = 4 * g + kk;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 v = V4[k * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float av = comp(a[i], kk);
                    acc[i][4 * j + 0] = fmaf(av, v.x, acc[i][4 * j + 0]);
                    acc[i][4 * j + 1] = fmaf(av, v.y, acc[i][4 * j + 1]);
                    acc[i][4 * j + 2] = fmaf(av, v.z, acc[i][4 * j + 2]);
                    acc[i][4 * j + 3] = fmaf(av, v.w, acc[i][4 * j + 3]);
                }
            }
        }
    }
}

// After fma_tile accumulation: warps exchange through `red` so that warp w
// ends with rows 16w + (lane & 15), columns 8 (lane >> 4) + 0..7, summed
// over the 8 column groups in warp order.
__device__ __forceinline__ void reduce_scatter_fma(const float (&acc)[4][16], float* red, float (&out)[8],
                                                   int w, int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 16; ++c) red[((w * 4 + i) * 16 + c) * 32 + lane] = acc[i][c];
    msp::bar_workers<kWorkers>();
    const int i = w >> 1, srcl = 16 * (w & 1) + (lane & 15), ch = lane >> 4;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
        const int c = 8 * ch + c8;
        float v = 0.f;
#pragma unroll
        for (int ww = 0; ww < kWorkWarps; ++ww) v += red[((ww * 4 + i) * 16 + c) * 32 + srcl];
        out[c8] = v;
    }
}

// x = hi + lo with hi the TF32 value nearest x and lo the TF32 value
// nearest the exact FP32 remainder x - hi ("3xTF32": the products
// hi*hi + hi*lo + lo*hi keep about FP32 accuracy).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// d += a b on the tensor cores: one 16 x 8 x 8 TF32 product, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(float& d0, float& d1, float& d2, float& d3, const uint32_t (&a)[4],
                                         uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc += T[:, 8w..8w+7] V[8w..8w+7, :] for the 128 x 64 swizzled tile T and
// the 64 x 16 block V: warp w takes one 8-column step of the tile for all
// 128 rows (eight 16 x 8 x 8 products per 8 right-hand sides) in 3xTF32.
// Lane (g, t) = (lane / 4, lane % 4) holds rows g, g + 8 and columns t, t + 4
// of each 16-row A fragment; the tile's granule swizzle (granule j of row r
// at j ^ (r % 8)) makes those loads hit 32 distinct banks. Accumulator
// layout: acc[mt / 2][(mt % 2) * 8 + nt * 4 + e] is row 16 mt + g + 8 (e / 2),
// column 8 nt + 2 t + e % 2.
__device__ __forceinline__ void mma_tile(float (&acc)[4][16], const float* __restrict__ T,
                                         const float* __restrict__ V, int w, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int k0 = 8 * w;
    uint32_t bh[2][2], bl[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        split_tf32(V[(k0 + t) * kM + 8 * nt + g], bh[nt][0], bl[nt][0]);
        split_tf32(V[(k0 + t + 4) * kM + 8 * nt + g], bh[nt][1], bl[nt][1]);
    }
    const int c0 = ((2 * w) ^ g) * 4 + t, c1 = ((2 * w + 1) ^ g) * 4 + t;
#pragma unroll
    for (int mt = 0; mt < 8; ++mt) {
        const int r0 = 16 * mt + g;
        uint32_t ah[4], al[4];
        split_tf32(T[r0 * kKT + c0], ah[0], al[0]);
        split_tf32(T[(r0 + 8) * kKT + c0], ah[1], al[1]);
        split_tf32(T[r0 * kKT + c1], ah[2], al[2]);
        split_tf32(T[(r0 + 8) * kKT + c1], ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float* d = &acc[mt >> 1][(mt & 1) * 8 + nt * 4];
            mma_tf32(d[0], d[1], d[2], d[3], al, bh[nt][0], bh[nt][1]);
            mma_tf32(d[0], d[1], d[2], d[3], ah, bl[nt][0], bl[nt][1]);
            mma_tf32(d[0], d[1], d[2], d[3], ah, bh[nt][0], bh[nt][1]);
        }
    }
}

// s + c += a (xh + xl) with the product a*xh split exactly (FMA) and the sum
// kept as an unevaluated pair (TwoSum, Knuth); a*xl is below the pair's
// rounding and goes to the correction term.
__device__ __forceinline__ void two_prod_acc(float& s, float& c, float a, float xh, float xl) {
    const float p = a * xh;
    const float e = fmaf(a, xh, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    c += err + e;
    c = fmaf(a, xl, c);
    s = t;
}

// Compensated tile: warp w = (row half h, column group kg); rows 64h+lane+32i,
// 16 columns 16kg.. of the tile.
__device__ __forceinline__ void comp_tile(float (&s)[2][16], float (&c)[2][16],
                                          const float* __restrict__ T, const float* __restrict__ XH,
                                          const float* __restrict__ XL, int h, int kg, int lane) {
    const float4* T4 = reinterpret_cast<const float4*>(T);
    const float4* H4 = reinterpret_cast<const float4*>(XH);
    const float4* L4 = reinterpret_cast<const float4*>(XL);
    const int sw = lane & 7;
#pragma unroll 1
    for (int gi = 0; gi < 4; ++gi) {
        const int g = 4 * kg + gi;
        float4 a[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) a[i] = T4[(64 * h + lane + 32 * i) * 16 + (g ^ sw)];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int k = 4 * g + kk;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 xh = H4[k * 4 + j];
                const float4 xl = L4[k * 4 + j];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float av = comp(a[i], kk);
                    two_prod_acc(s[i][4 * j + 0], c[i][4 * j + 0], av, xh.x, xl.x);
                    two_prod_acc(s[i][4 * j + 1], c[i][4 * j + 1], av, xh.y, xl.y);
                    two_prod_acc(s[i][4 * j + 2], c[i][4 * j + 2], av, xh.z, xl.z);
                    two_prod_acc(s[i][4 * j + 3], c[i][4 * j + 3], av, xh.w, xl.w);
                }
            }
        }
    }
}

// After mma_tile accumulation over a row block: warps exchange through `red`
// (8 warps x 128 rows x 16 columns) so that warp w ends with rows
// 16w + (lane & 15), columns 8 (lane >> 4) + 0..7, summed over the 8 column
// steps in warp order.
__device__ __forceinline__ void reduce_scatter(const float (&acc)[4][16], float* red, float (&out)[8],
                                               int w, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 8; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = 16 * mt + g + 8 * h, col = 8 * nt + 2 * t;
                const float* d = &acc[mt >> 1][(mt & 1) * 8 + nt * 4 + 2 * h];
                *reinterpret_cast<float2*>(red + (w * kRB + row) * kM + col) = make_float2(d[0], d[1]);
            }
    msp::bar_workers<kWorkers>();
    const int row = 16 * w + (lane & 15), ch = lane >> 4;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) out[c8] = 0.f;
#pragma unroll
    for (int ww = 0; ww < kWorkWarps; ++ww) {
        const float4 u0 = ld4(red + (ww * kRB + row) * kM + 8 * ch);
        const float4 u1 = ld4(red + (ww * kRB + row) * kM + 8 * ch + 4);
        out[0] += u0.x; out[1] += u0.y; out[2] += u0.z; out[3] += u0.w;
        out[4] += u1.x; out[5] += u1.y; out[6] += u1.z; out[7] += u1.w;
    }
}

// Column sums over the 16 rows of a warp in the reduce_scatter layout
// (lanes l and l ^ 1..8 share columns), then over the 8 warps in order.
// Called by all worker threads; thread c < 16 of warp 0 gets column c.
__device__ __forceinline__ double colsum_rs(const float (&v)[8], float* wsum, int w, int lane) {
    float d[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
        d[c8] = v[c8];
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) d[c8] += __shfl_xor_sync(0xffffffffu, d[c8], o);
    }
    if ((lane & 15) == 0)
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) wsum[w * 16 + 8 * (lane >> 4) + c8] = d[c8];
    msp::bar_workers<kWorkers>();
    double t = 0.0;
    if (w == 0 && lane < 16) {
        float f = 0.f;
        for (int ww = 0; ww < kWorkWarps; ++ww) f += wsum[ww * 16 + lane];
        t = (double)f;
    }
    return t;
}

// Same for the row-vector layout (thread = row tid >> 1, columns 8 (tid & 1)..)
__device__ __forceinline__ double colsum_rv(const float (&v)[8], float* wsum, int w, int lane) {
    float d[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
        d[c8] = v[c8];
#pragma unroll
        for (int o = 2; o < 32; o <<= 1) d[c8] += __shfl_xor_sync(0xffffffffu, d[c8], o);
    }
    if (lane < 2)
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) wsum[w * 16 + 8 * lane + c8] = d[c8];
    msp::bar_workers<kWorkers>();
    double t = 0.0;
    if (w == 0 && lane < 16) {
        float f = 0.f;
        for (int ww = 0; ww < kWorkWarps; ++ww) f += wsum[ww * 16 + lane];
        t = (double)f;
    }
    msp::bar_workers<kWorkers>();
    return t;
}

// --------------------------------------------------- the streamed A passes

// What a streamed pass reads: A tiles with P slices (level-1 A pass), A
// tiles with x_hi / x_lo slices (residual), C tiles with Y2 slices (Z step),
// a 64-column strip of C tiles down the row blocks with R rows (G step).
enum { kModeA = 0, kModeR = 1, kModeZ = 2, kModeG = 3 };

template <int Mode>
__device__ __noinline__ void producer(const BArgs& a, unsigned char* ring, uint64_t* full, uint64_t* empty,
                         int2* hdr, uint32_t& kring, int* counter,
                         const int* flag) {
    const uint64_t pol = msp::policy_evict_first();
    int* err = &a.ctl->error;
    bool stop = false;
    while (!stop) {
        const int it = atomicAdd(counter, 1);
        const int nitems = (Mode == kModeZ) ? a.nrows : (Mode == kModeG) ? a.nstrips : a.nunits;
        int inst = -1, rb = 0, nk = 1, k0 = 0, k1 = 1;
        if (it < nitems) {
            const int2 w = (Mode == kModeZ) ? a.rows[it] : (Mode == kModeG) ? a.strips[it] : a.units[it];
            inst = w.x;
            rb = w.y & 0xffff;
            if (!ld_volatile(flag + inst)) continue;
            if (Mode == kModeG) {
                // rb holds the strip; the loop runs over the row blocks
                nk = a.inst[inst].s_pad / kKT;
                k0 = 0;
                k1 = a.inst[inst].nb;
            } else if (Mode == kModeZ) {
                nk = a.inst[inst].s_pad / kKT;
                k0 = 0;
                k1 = nk;
            } else {
                nk = a.inst[inst].n_pad / kKT;
                k0 = (w.y >> 16) * a.ut;
                k1 = min(nk, k0 + a.ut);
            }
        }
        for (int kt = k0; kt < k1; ++kt) {
            const int s = (int)(kring % kStages);
            if (kring >= kStages &&
                !msp::mbar_wait_timed(&empty[s], ((kring / kStages) & 1u) ^ 1u, err)) {
                stop = true;
                break;
            }
            unsigned char* st = ring + (size_t)s * kStageBytes;
            if (it >= nitems) {
                hdr[s] = make_int2(-1, 0);
                msp::mbar_arrive(&full[s]);
                ++kring;
                stop = true;
                break;
            }
            hdr[s] = make_int2(it, 2 * kt + (kt == k1 - 1 ? 1 : 0));
            if (kt == k0) {
                if (Mode == kModeZ) atomicAdd(&a.ctl->bytesZ, (unsigned long long)(k1 - k0) * kTileBytes);
                else if (Mode == kModeG) atomicAdd(&a.ctl->bytesG, (unsigned long long)(k1 - k0) * kTileBytes);
                else atomicAdd(Mode == kModeR ? &a.ctl->tilesR : &a.ctl->tilesA, (unsigned long long)(k1 - k0));
            }
            const BInst& I = a.inst[inst];
            const int64_t tile = (Mode == kModeG) ? ((int64_t)kt * nk + rb) : ((int64_t)rb * nk + kt);
            const float* At = (Mode == kModeZ || Mode == kModeG ? I.Ct : I.At) + tile * kTileFloats;
            msp::mbar_arrive_expect_tx(&full[s], kTileBytes + (Mode == kModeR || Mode == kModeG ? 2 : 1) * kSliceBytes);
            msp::bulk_g2s_hint(st, At, kTileBytes / 2, &full[s], pol);
            msp::bulk_g2s_hint(st + kTileBytes / 2, At + kTileFloats / 2, kTileBytes / 2, &full[s], pol);
            if (Mode == kModeA) {
                const int64_t vrow = (int64_t)I.voff + (int64_t)kt * kKT;
                msp::bulk_g2s(st + kTileBytes, a.P + vrow * kM, kSliceBytes, &full[s]);
            } else if (Mode == kModeR) {
                const int64_t vrow = (int64_t)I.voff + (int64_t)kt * kKT;
                msp::bulk_g2s(st + kTileBytes, a.XH + vrow * kM, kSliceBytes, &full[s]);
                msp::bulk_g2s(st + kTileBytes + kSliceBytes, a.XL + vrow * kM, kSliceBytes, &full[s]);
            } else if (Mode == kModeZ) {
                const int64_t srow = (int64_t)I.soff + (int64_t)kt * kKT;
                msp::bulk_g2s(st + kTileBytes, a.Y2 + srow * kM, kSliceBytes, &full[s]);
            } else {
                const int64_t vrow = (int64_t)I.voff + (int64_t)kt * kRB;
                msp::bulk_g2s(st + kTileBytes, a.R + vrow * kM, 2 * kSliceBytes, &full[s]);
            }
            ++kring;
        }
    }
    // every issued copy must land before the block moves on or exits
    const uint32_t k0 = kring > (uint32_t)kStages ? kring - kStages : 0u;
    for (uint32_t k = k0; k < kring; ++k)
        if (!msp::mbar_wait_timed(&full[k % kStages], (k / kStages) & 1u, err)) break;
}

// Unit partials of a row block that spans several units: every unit writes
// its part; the block that finishes the row block's last unit (counter, with
// fences between the parts and the count) sums the parts in unit order, so
// the result does not depend on which block finished last. Returns whether
// this block is that one (uniform over the worker threads).
__device__ __forceinline__ bool last_unit(int* cnt, int nkc, int* sflag, int tid) {
    __threadfence();
    msp::bar_workers<kWorkers>();
    if (tid == 0) {
        const int k = atomicAdd(cnt, 1);
        *sflag = (k == nkc - 1);
        if (k == nkc - 1) *cnt = 0;
    }
    msp::bar_workers<kWorkers>();
    const bool last = *(volatile int*)sflag != 0;
    if (last) __threadfence();
    return last;
}

// SA consumers: Q = (A + lam I) P and the block partials of p^T q.
__device__ __noinline__ void consume_A(const BArgs& a, unsigned char* ring, uint64_t* full, uint64_t* empty,
                          const int2* hdr, uint32_t& kring, float* red,
                          float* wsum, int* sflag, int w, int lane) {
    float acc[4][16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[i][c] = 0.f;
    int* err = &a.ctl->error;
    while (true) {
        const int s = (int)(kring % kStages);
        if (!msp::mbar_wait_timed(&full[s], (kring / kStages) & 1u, err)) return;
        const int2 h = hdr[s];
        ++kring;
        if (h.x < 0) {
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&empty[s]);
            return;
        }
        const float* T = reinterpret_cast<const float*>(ring + (size_t)s * kStageBytes);
        mma_tile(acc, T, T + kTileFloats, w, lane);
        __syncwarp();
        if (lane == 0) msp::mbar_arrive(&empty[s]);
        if (!(h.y & 1)) continue;
        const int2 u = a.units[h.x];
        const int2 item = make_int2(u.x, u.y & 0xffff);
        const int kc = u.y >> 16;
        const BInst& I = a.inst[item.x];
        // ---- unit complete
        float out[8];
        reduce_scatter(acc, red, out, w, lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[i][c] = 0.f;
        const int ch = lane >> 4;
        const int row = item.y * kRB + 16 * w + (lane & 15);
        const int64_t vrow = (int64_t)I.voff + row;
        if (I.nkc > 1) {
            float* qp = a.Qp + ((int64_t)I.qoff + (int64_t)kc * I.n_pad + row) * kM + 8 * ch;
            st4(qp, make_float4(out[0], out[1], out[2], out[3]));
            st4(qp + 4, make_float4(out[4], out[5], out[6], out[7]));
            if (!last_unit(a.rbcnt + I.boff + item.y, I.nkc, sflag, w * 32 + lane)) continue;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) out[c8] = 0.f;
            for (int k = 0; k < I.nkc; ++k) {
                const float* q2 = a.Qp + ((int64_t)I.qoff + (int64_t)k * I.n_pad + row) * kM + 8 * ch;
                const float4 u0 = __ldcg(reinterpret_cast<const float4*>(q2));
                const float4 u1 = __ldcg(reinterpret_cast<const float4*>(q2 + 4));
                out[0] += u0.x; out[1] += u0.y; out[2] += u0.z; out[3] += u0.w;
                out[4] += u1.x; out[5] += u1.y; out[6] += u1.z; out[7] += u1.w;
            }
        }
        const float4 p0 = ld4(a.P + vrow * kM + 8 * ch), p1 = ld4(a.P + vrow * kM + 8 * ch + 4);
        const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
        float q[8], d[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            q[c8] = fmaf(I.lam, pv[c8], out[c8]);
            d[c8] = pv[c8] * q[c8];
        }
        st4(a.Q + vrow * kM + 8 * ch, make_float4(q[0], q[1], q[2], q[3]));
        st4(a.Q + vrow * kM + 8 * ch + 4, make_float4(q[4], q[5], q[6], q[7]));
        const double t = colsum_rs(d, wsum, w, lane);
        if (w == 0 && lane < 16) a.p_pq[((int64_t)I.boff + item.y) * kM + lane] = t;
    }
}

// Refinement residual consumers: R64 = B - lam X - A X with A X from
// compensated FP32 tiles, and the block partials of |r|^2 (FP64).
__device__ __noinline__ void consume_R(const BArgs& a, unsigned char* ring, uint64_t* full, uint64_t* empty,
                          const int2* hdr, uint32_t& kring, double* redd,
                          double* wsumd, int* sflag, int w, int lane) {
    float s[2][16], c[2][16];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) s[i][j] = c[i][j] = 0.f;
    const int h = w >> 2, kg = w & 3;
    int* err = &a.ctl->error;
    while (true) {
        const int st = (int)(kring % kStages);
        if (!msp::mbar_wait_timed(&full[st], (kring / kStages) & 1u, err)) return;
        const int2 hd = hdr[st];
        ++kring;
        if (hd.x < 0) {
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&empty[st]);
            return;
        }
        const float* T = reinterpret_cast<const float*>(ring + (size_t)st * kStageBytes);
        comp_tile(s, c, T, T + kTileFloats, T + kTileFloats + kSliceFloats, h, kg, lane);
        __syncwarp();
        if (lane == 0) msp::mbar_arrive(&empty[st]);
        if (!(hd.y & 1)) continue;
        const int2 u = a.units[hd.x];
        const int2 item = make_int2(u.x, u.y & 0xffff);
        const int kc = u.y >> 16;
        const BInst& I = a.inst[item.x];
        // ---- unit complete: combine the 4 column groups in FP64
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                redd[((w * 2 + i) * 16 + j) * 32 + lane] = (double)s[i][j] + (double)c[i][j];
                s[i][j] = c[i][j] = 0.f;
            }
        msp::bar_workers<kWorkers>();
        const int r = 16 * w + (lane & 15);
        const int hh = r >> 6, i = (r & 63) >> 5, srcl = r & 31, ch = lane >> 4;
        const int row = item.y * kRB + r;
        const int64_t vrow = (int64_t)I.voff + row;
        double v8[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int col = 8 * ch + c8;
            double v = 0.0;
#pragma unroll
            for (int g = 0; g < 4; ++g) v += redd[(((4 * hh + g) * 2 + i) * 16 + col) * 32 + srcl];
            v8[c8] = v;
        }
        if (I.nkc > 1) {
            double* rp = a.Rp + ((int64_t)I.qoff + (int64_t)kc * I.n_pad + row) * kM + 8 * ch;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) rp[c8] = v8[c8];
            if (!last_unit(a.rbcnt + I.boff + item.y, I.nkc, sflag, w * 32 + lane)) continue;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) v8[c8] = 0.0;
            for (int k = 0; k < I.nkc; ++k) {
                const double* r2 = a.Rp + ((int64_t)I.qoff + (int64_t)k * I.n_pad + row) * kM + 8 * ch;
#pragma unroll
                for (int c8 = 0; c8 < 8; ++c8) v8[c8] += __ldcg(r2 + c8);
            }
        }
        double d2[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int col = 8 * ch + c8;
            const double v = v8[c8];
            double rv = 0.0;
            if (row < I.n && col < I.m) {
                const double b = I.B[(int64_t)col * I.ldb + row];
                const double x = I.X[(int64_t)col * I.ldx + row];
                rv = b - I.lam64 * x - v;
            }
            a.R64[vrow * kM + col] = rv;
            d2[c8] = rv * rv;
        }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) d2[c8] += __shfl_xor_sync(0xffffffffu, d2[c8], o);
        if ((lane & 15) == 0)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) wsumd[w * 16 + 8 * ch + c8] = d2[c8];
        msp::bar_workers<kWorkers>();
        if (w == 0 && lane < 16) {
            double t = 0.0;
            for (int ww = 0; ww < kWorkWarps; ++ww) t += wsumd[ww * 16 + lane];
            a.p_r64[((int64_t)I.boff + item.y) * kM + lane] = t;
        }
    }
}

// ------------------------------------------------- mat-vec steps (S3-S5)

// acc += M[rows 0..127][k] V[k][.] over k tiles [kt0, kt1): M row-major (ld),
// rows >= rows_valid read as zero; V staged in shared memory by absolute k.
__device__ __forceinline__ void mv_stream(float (&acc)[4][16], const float* __restrict__ M, int64_t ld, int rows_valid,
                          int kt0, int kt1, const float* Vs, float* tiles, int tid, int w, int lane) {
    const int nkt = kt1 - kt0;
    auto issue = [&](int kt, int buf) {
        float* dst = tiles + buf * kTileFloats;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = tid + kWorkers * j;
            const int row = e >> 4, g = e & 15;
            const bool ok = row < rows_valid;
            const float* src = ok ? M + (int64_t)row * ld + (int64_t)kt * kKT + 4 * g : M;
            msp::cp_async16(dst + row * kKT + ((g ^ (row & 7)) << 2), src, ok);
        }
    };
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
        if (j < nkt) issue(kt0 + j, j);
        msp::cp_async_commit();
    }
#pragma unroll 1
    for (int i = 0; i < nkt; ++i) {
        if (i + 2 < nkt) issue(kt0 + i + 2, (i + 2) % kMvTiles);
        msp::cp_async_commit();
        msp::cp_async_wait<2>();
        msp::bar_workers<kWorkers>();
        fma_tile(acc, tiles + (i % kMvTiles) * kTileFloats, Vs + (int64_t)(kt0 + i) * kKT * kM, w, lane);
        msp::bar_workers<kWorkers>();
    }
}

// Stage rows [k0, k1) of a [.][16] vector block into Vs (same row indices).
__device__ __forceinline__ void stage_vec(float* Vs, const float* src, int k0, int k1, int tid) {
    msp::bar_workers<kWorkers>();
    for (int e = k0 * 4 + tid; e < k1 * 4; e += kWorkers)
        reinterpret_cast<float4*>(Vs)[e] = reinterpret_cast<const float4*>(src)[e];
    msp::bar_workers<kWorkers>();
}

// ------------------------------------------------------------- the steps

// Contiguous share of `n` items for this block.
__device__ __forceinline__ void my_range(int n, int& i0, int& i1) {
    i0 = (int)((int64_t)n * blockIdx.x / gridDim.x);
    i1 = (int)((int64_t)n * (blockIdx.x + 1) / gridDim.x);
}

// Dynamic item claim for the worker threads: thread 0 takes the next index
// of the step's counter and shares it through `slot`.
__device__ __forceinline__ int claim(int* ctr, int* slot, int tid) {
    if (tid == 0) *slot = atomicAdd(ctr, 1);
    msp::bar_workers<kWorkers>();
    const int it = *(volatile int*)slot;
    msp::bar_workers<kWorkers>();
    return it;
}

// R64 = B (X = 0), partials of |b|^2.
__device__ __forceinline__ void step_init(const BArgs& a, double* wsumd, int tid, int w, int lane) {
    int i0, i1;
    my_range(a.nrows, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 item = a.rows[it];
        const BInst& I = a.inst[item.x];
        const int row = item.y * kRB + (tid >> 1), ch = tid & 1;
        const int64_t vrow = (int64_t)I.voff + row;
        double d[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int col = 8 * ch + c8;
            double b = 0.0;
            if (row < I.n && col < I.m) {
                b = I.B[(int64_t)col * I.ldb + row];
                I.X[(int64_t)col * I.ldx + row] = 0.0;
            }
            a.R64[vrow * kM + col] = b;
            d[c8] = b * b;
        }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int o = 2; o < 32; o <<= 1) d[c8] += __shfl_xor_sync(0xffffffffu, d[c8], o);
        if (lane < 2)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) wsumd[w * 16 + 8 * lane + c8] = d[c8];
        msp::bar_workers<kWorkers>();
        if (w == 0 && lane < 16) {
            double t = 0.0;
            for (int ww = 0; ww < kWorkWarps; ++ww) t += wsumd[ww * 16 + lane];
            a.p_r64[((int64_t)I.boff + item.y) * kM + lane] = t;
            a.p_xx[((int64_t)I.boff + item.y) * kM + lane] = 0.0;
        }
        msp::bar_workers<kWorkers>();
    }
}

// Per instance (one block each): residual norms from the R64 partials, the
// final-tolerance flags, |R64| for the next correction solve, results.
__device__ __forceinline__ void step_check(const BArgs& a, int step, int w, int lane) {
    if (w != 0) return;
    for (int i = blockIdx.x; i < a.count; i += gridDim.x) {
        const BInst& I = a.inst[i];
        const int c = lane & 15;
        double rr = 0.0, xx = 0.0;
        for (int b = 0; b < I.nb; ++b) {
            rr += a.p_r64[((int64_t)I.boff + b) * kM + c];
            xx += a.p_xx[((int64_t)I.boff + b) * kM + c];
        }
        const int gi = i * kM + c;
        if (step == 0 && lane < 16) a.bb[gi] = rr;
        const double bb = (step == 0) ? rr : a.bb[gi];
        if (lane < 16 && c < I.m && !isfinite(rr)) atomicCAS(&a.ierr[i], 0, (int)MSP_ENONFINITE);
        __syncwarp();
        const int e = ld_volatile(&a.ierr[i]);
        // backward-error bound |r| / ((L + lam) |x| + |b|), L <= |A|_2
        const double den = (a.anorm[i] + I.lam64) * sqrt(xx) + sqrt(bb);
        const double be = (c < I.m && den > 0.0 && isfinite(rr)) ? sqrt(rr) / den : 0.0;
        const bool met = a.crit ? sqrt(rr) <= a.tol * den : rr <= a.tol2 * bb;
        const bool f = (c >= I.m) || e != 0 || !(bb > 0.0) || met;
        const double rel = (c < I.m && bb > 0.0 && isfinite(rr)) ? sqrt(rr / bb) : 0.0;
        if (lane < 16) {
            a.fin[gi] = f ? 1 : 0;
            a.scale[gi] = sqrt(rr);
        }
        const unsigned unf = __ballot_sync(0xffffffffu, lane < 16 && !f);
        double mr = (lane < 16) ? rel : 0.0, mb = (lane < 16) ? be : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
            mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (lane == 0) {
            a.rel[i] = mr;
            a.berr[i] = mb;
            if (unf) atomicAdd(&a.ctl->unfinished[step & 1], __popc(unf));
        }
    }
    if (blockIdx.x == 0 && lane == 0) a.ctl->ctrR = 0;
}

// Start of a correction solve: R = R64 / |R64| per column (0 for finished
// columns), X_w = 0, Q = 0, partials of |r|^2.
__device__ __forceinline__ void step_scale(const BArgs& a, int step, float* wsum, double* sd, int tid, int w, int lane) {
    if (blockIdx.x == 0 && tid == 0) {
        a.ctl->active[0] = 0;
        a.ctl->active[1] = 0;
        a.ctl->unfinished[(step + 1) & 1] = 0;
        a.ctl->ctrA = 0;
        a.ctl->ctrG = a.ctl->ctrT1 = a.ctl->ctrT2 = a.ctl->ctrZ = 0;
    }
    int i0, i1;
    my_range(a.nrows, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 item = a.rows[it];
        const BInst& I = a.inst[item.x];
        if (w == 0) {
            const int c = lane & 15, gi = item.x * kM + c;
            const bool act = lane < 16 && !a.fin[gi];
            if (lane < 16) sd[c] = act ? a.scale[gi] : 0.0;
            const unsigned any = __ballot_sync(0xffffffffu, act);
            if (item.y == 0 && lane == 0) {
                a.iact[a.count + item.x] = any ? 1 : 0;    // generation read by step 0's S2
                a.istep[item.x] = any ? 1 : 0;
                if (any) a.isteps[item.x] += 1;
            }
        }
        msp::bar_workers<kWorkers>();
        const int row = item.y * kRB + (tid >> 1), ch = tid & 1;
        const int64_t vrow = (int64_t)I.voff + row;
        float r[8], d[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int col = 8 * ch + c8;
            const double sc = sd[col];
            r[c8] = sc > 0.0 ? (float)(a.R64[vrow * kM + col] / sc) : 0.f;
            d[c8] = r[c8] * r[c8];
        }
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        st4(a.R + vrow * kM + 8 * ch, make_float4(r[0], r[1], r[2], r[3]));
        st4(a.R + vrow * kM + 8 * ch + 4, make_float4(r[4], r[5], r[6], r[7]));
        st4(a.XW + vrow * kM + 8 * ch, z4);
        st4(a.XW + vrow * kM + 8 * ch + 4, z4);
        st4(a.Q + vrow * kM + 8 * ch, z4);
        st4(a.Q + vrow * kM + 8 * ch + 4, z4);
        const double t = colsum_rv(d, wsum, w, lane);
        if (w == 0 && lane < 16) a.p_rr[((int64_t)I.boff + item.y) * kM + lane] = t;
    }
}

// S2 part 1: per instance (one block each, warp 0), the convergence flags of
// its columns from the |r|^2 partials, and the active-column count.
__device__ __forceinline__ void step_flags(const BArgs& a, int t, int lane) {
    const int cur = t & 1;
    for (int i = blockIdx.x; i < a.count; i += gridDim.x) {
        const BInst& I = a.inst[i];
        const int c = lane & 15, gi = i * kM + c;
        double rr = 0.0;
        for (int b = 0; b < I.nb; ++b) rr += a.p_rr[((int64_t)I.boff + b) * kM + c];
        const bool live = lane < 16 && c < I.m && !a.fin[gi];
        if (live && !isfinite(rr)) atomicCAS(&a.ierr[i], 0, (int)MSP_ENONFINITE);
        __syncwarp();
        const bool act = live && ld_volatile(&a.ierr[i]) == 0 && rr > a.rtol2 && t < a.max_outer;
        if (lane < 16) a.act[gi] = act ? 1 : 0;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (lane == 0) {
            a.iact[cur * a.count + i] = m ? 1 : 0;
            if (m) {
                a.iters[i] += 1;
                atomicAdd(&a.ctl->active[cur], __popc(m));
            }
        }
    }
}

// S2 part 2: G = C^T R by 64-column strips of C: the producer streams the
// strip's tiles down all row blocks with the R rows of each; warp w takes
// rows 16w..16w+15 of a tile, a lane two columns x 16 right-hand sides
// (FP32 FMA), and the 8 warps' sums are combined in warp order at the end of
// the strip.
__device__ __noinline__ void consume_G(const BArgs& a, unsigned char* ring, uint64_t* full, uint64_t* empty,
                                       const int2* hdr, uint32_t& kring, float* red, int w, int lane) {
    float acc[2][16];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[q][c] = 0.f;
    int* err = &a.ctl->error;
    const int tid = w * 32 + lane;
    while (true) {
        const int s = (int)(kring % kStages);
        if (!msp::mbar_wait_timed(&full[s], (kring / kStages) & 1u, err)) return;
        const int2 h = hdr[s];
        ++kring;
        if (h.x < 0) {
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&empty[s]);
            return;
        }
        const float* T = reinterpret_cast<const float*>(ring + (size_t)s * kStageBytes);
        const float4* R4 = reinterpret_cast<const float4*>(T + kTileFloats);
#pragma unroll 4
        for (int rr = 0; rr < 16; ++rr) {
            const int r = 16 * w + rr, sw = r & 7;
            const float* Tr = T + r * kKT;
            const float c0 = Tr[(((lane >> 2) ^ sw) << 2) + (lane & 3)];
            const float c1 = Tr[((((lane >> 2) + 8) ^ sw) << 2) + (lane & 3)];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 v = R4[r * 4 + j];
                acc[0][4 * j + 0] = fmaf(c0, v.x, acc[0][4 * j + 0]);
                acc[0][4 * j + 1] = fmaf(c0, v.y, acc[0][4 * j + 1]);
                acc[0][4 * j + 2] = fmaf(c0, v.z, acc[0][4 * j + 2]);
                acc[0][4 * j + 3] = fmaf(c0, v.w, acc[0][4 * j + 3]);
                acc[1][4 * j + 0] = fmaf(c1, v.x, acc[1][4 * j + 0]);
                acc[1][4 * j + 1] = fmaf(c1, v.y, acc[1][4 * j + 1]);
                acc[1][4 * j + 2] = fmaf(c1, v.z, acc[1][4 * j + 2]);
                acc[1][4 * j + 3] = fmaf(c1, v.w, acc[1][4 * j + 3]);
            }
        }
        __syncwarp();
        if (lane == 0) msp::mbar_arrive(&empty[s]);
        if (!(h.y & 1)) continue;
        // ---- strip complete: sum the 8 warps' partials in order
        const int2 item = a.strips[h.x];
        const BInst& I = a.inst[item.x];
        float4* red4 = reinterpret_cast<float4*>(red);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                red4[(w * 64 + lane + 32 * q) * 4 + j] =
                    make_float4(acc[q][4 * j], acc[q][4 * j + 1], acc[q][4 * j + 2], acc[q][4 * j + 3]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[q][c] = 0.f;
        msp::bar_workers<kWorkers>();
        {
            const int j = tid >> 2, qd = tid & 3;
            float4 v = red4[j * 4 + qd];
            for (int ww = 1; ww < kWorkWarps; ++ww) {
                const float4 u = red4[(ww * 64 + j) * 4 + qd];
                v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
            }
            st4(a.G + ((int64_t)I.soff + item.y * kKT + j) * kM + 4 * qd, v);
        }
        msp::bar_workers<kWorkers>();
    }
}

// S3 / S4: Y_out[chunk] = L^{-1} G or L^{-T} Y1 (triangular k range).
template <bool kUpper>
__device__ __noinline__ void step_tri(const BArgs& a, int t, unsigned char* smem, float* red, int* slot,
                                      int tid, int w, int lane) {
    const int cur = t & 1;
    float* tiles = reinterpret_cast<float*>(smem);
    float* Vs = reinterpret_cast<float*>(smem + kVsOffset);
    for (;;) {
        const int it = claim(kUpper ? &a.ctl->ctrT2 : &a.ctl->ctrT1, slot, tid);
        if (it >= a.nchunks) break;
        const int2 item = a.chunks[it];
        const BInst& I = a.inst[item.x];
        if (!ld_volatile(&a.iact[cur * a.count + item.x])) continue;
        const int kt0 = kUpper ? 2 * item.y : 0;
        const int kt1 = kUpper ? I.s_pad / kKT : 2 * (item.y + 1);
        const float* V = (kUpper ? a.Y1 : a.G) + (int64_t)I.soff * kM;
        stage_vec(Vs, V, kt0 * kKT, kt1 * kKT, tid);
        float acc[4][16];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[i][c] = 0.f;
        const float* M = (kUpper ? I.Bu : I.Bl) + (int64_t)item.y * kRB * I.s_pad;
        mv_stream(acc, M, I.s_pad, kRB, kt0, kt1, Vs, tiles, tid, w, lane);
        float out[8];
        reduce_scatter_fma(acc, red, out, w, lane);
        const int ch = lane >> 4;
        float* Y = (kUpper ? a.Y2 : a.Y1) + ((int64_t)I.soff + item.y * kRB + 16 * w + (lane & 15)) * kM + 8 * ch;
        st4(Y, make_float4(out[0], out[1], out[2], out[3]));
        st4(Y + 4, make_float4(out[4], out[5], out[6], out[7]));
        msp::bar_workers<kWorkers>();
    }
}

// S5: Z = (R - C Y2) / lam~ by row blocks, partials of z.r and z.q: the
// producer warp streams the instance's C tiles with Y2 slices through the
// ring; the consumers keep FP32 FMA (the Woodbury form cancels).
__device__ __noinline__ void consume_Z(const BArgs& a, unsigned char* ring, uint64_t* full, uint64_t* empty,
                                       const int2* hdr, uint32_t& kring, float* red, float* wsum, int w,
                                       int lane) {
    float acc[4][16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[i][c] = 0.f;
    int* err = &a.ctl->error;
    while (true) {
        const int s = (int)(kring % kStages);
        if (!msp::mbar_wait_timed(&full[s], (kring / kStages) & 1u, err)) return;
        const int2 h = hdr[s];
        ++kring;
        if (h.x < 0) {
            __syncwarp();
            if (lane == 0) msp::mbar_arrive(&empty[s]);
            return;
        }
        const float* T = reinterpret_cast<const float*>(ring + (size_t)s * kStageBytes);
        fma_tile(acc, T, T + kTileFloats, w, lane);
        __syncwarp();
        if (lane == 0) msp::mbar_arrive(&empty[s]);
        if (!(h.y & 1)) continue;
        const int2 item = a.rows[h.x];
        const BInst& I = a.inst[item.x];
        float out[8];
        reduce_scatter_fma(acc, red, out, w, lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[i][c] = 0.f;
        const int ch = lane >> 4;
        const int64_t vrow = (int64_t)I.voff + item.y * kRB + 16 * w + (lane & 15);
        const float4 r0 = ld4(a.R + vrow * kM + 8 * ch), r1 = ld4(a.R + vrow * kM + 8 * ch + 4);
        const float4 q0 = ld4(a.Q + vrow * kM + 8 * ch), q1 = ld4(a.Q + vrow * kM + 8 * ch + 4);
        const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const float qv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        float z[8], zr[8], zq[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            z[c8] = (rv[c8] - out[c8]) * I.inv_lt;
            zr[c8] = z[c8] * rv[c8];
            zq[c8] = z[c8] * qv[c8];
        }
        st4(a.Z + vrow * kM + 8 * ch, make_float4(z[0], z[1], z[2], z[3]));
        st4(a.Z + vrow * kM + 8 * ch + 4, make_float4(z[4], z[5], z[6], z[7]));
        const double tzr = colsum_rs(zr, wsum, w, lane);
        if (w == 0 && lane < 16) a.p_zr[((int64_t)I.boff + item.y) * kM + lane] = tzr;
        msp::bar_workers<kWorkers>();
        const double tzq = colsum_rs(zq, wsum, w, lane);
        if (w == 0 && lane < 16) a.p_zq[((int64_t)I.boff + item.y) * kM + lane] = tzq;
        msp::bar_workers<kWorkers>();
    }
}

// S6: beta = -alpha z^T q / rz_old (flexible Polak-Ribiere with
// r_new - r_old = -alpha q), P = Z + beta P; rz_new kept for S1.
__device__ __forceinline__ void step_P(const BArgs& a, int t, float* sv, int tid, int w, int lane) {
    const int cur = t & 1, prev = cur ^ 1;
    int i0, i1;
    my_range(a.nrows, i0, i1);
    int cached = -1;
    for (int it = i0; it < i1; ++it) {
        const int2 item = a.rows[it];
        const BInst& I = a.inst[item.x];
        if (!ld_volatile(&a.iact[cur * a.count + item.x])) continue;
        // beta of the instance: once per instance met by this block
        if (item.x != cached || item.y == 0) {
            msp::bar_workers<kWorkers>();     // the previous item's readers of sv are done
            if (w == 0 && lane < 16) {
                const int c = lane, gi = item.x * kM + c;
                double rzn = 0.0, zq = 0.0;
                for (int b = 0; b < I.nb; ++b) {
                    rzn += a.p_zr[((int64_t)I.boff + b) * kM + c];
                    zq += a.p_zq[((int64_t)I.boff + b) * kM + c];
                }
                const double rzo = a.rz[(int64_t)prev * a.count * kM + gi];
                double beta = 0.0;
                if (t > 0 && a.act[gi] && rzo > 0.0 && isfinite(rzo)) beta = -a.alpha[gi] * zq / rzo;
                sv[c] = (float)beta;
                if (item.y == 0) {
                    a.rz[(int64_t)cur * a.count * kM + gi] = rzn;
                    if (a.act[gi] && !(rzn > 0.0)) atomicCAS(&a.ierr[item.x], 0, (int)MSP_ENOTPD);
                }
            }
            cached = item.x;
            msp::bar_workers<kWorkers>();
        }
        const int row = item.y * kRB + (tid >> 1), ch = tid & 1;
        const int64_t vrow = (int64_t)I.voff + row;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int off = 8 * ch + 4 * h;
            const float4 z = ld4(a.Z + vrow * kM + off);
            const float4 p = ld4(a.P + vrow * kM + off);
            st4(a.P + vrow * kM + off,
                make_float4(fmaf(sv[off + 0], p.x, z.x), fmaf(sv[off + 1], p.y, z.y),
                            fmaf(sv[off + 2], p.z, z.z), fmaf(sv[off + 3], p.w, z.w)));
        }
    }
    msp::bar_workers<kWorkers>();
}

// S1: alpha = rz / p^T q, X_w += alpha P, R -= alpha Q, partials of |r|^2.
__device__ __forceinline__ void step_X(const BArgs& a, int t, float* wsum, float* sv, int tid, int w, int lane) {
    const int cur = t & 1;
    if (blockIdx.x == 0 && tid == 0) {
        a.ctl->ctrA = 0;
        a.ctl->ctrG = a.ctl->ctrT1 = a.ctl->ctrT2 = a.ctl->ctrZ = 0;
    }
    int i0, i1;
    my_range(a.nrows, i0, i1);
    int cached = -1;
    for (int it = i0; it < i1; ++it) {
        const int2 item = a.rows[it];
        const BInst& I = a.inst[item.x];
        if (!ld_volatile(&a.iact[cur * a.count + item.x])) continue;
        // alpha of the instance: once per instance met by this block
        if (item.x != cached || item.y == 0) {
            if (w == 0 && lane < 16) {
                const int c = lane, gi = item.x * kM + c;
                double al = 0.0;
                if (a.act[gi]) {
                    double pq = 0.0;
                    for (int b = 0; b < I.nb; ++b) pq += a.p_pq[((int64_t)I.boff + b) * kM + c];
                    const double rz = a.rz[(int64_t)cur * a.count * kM + gi];
                    if (pq > 0.0 && isfinite(pq)) al = rz / pq;
                    else atomicCAS(&a.ierr[item.x], 0, isfinite(pq) ? (int)MSP_ENOTPD : (int)MSP_ENONFINITE);
                }
                sv[c] = (float)al;
                if (item.y == 0) a.alpha[gi] = al;
            }
            cached = item.x;
            msp::bar_workers<kWorkers>();
        }
        const int row = item.y * kRB + (tid >> 1), ch = tid & 1;
        const int64_t vrow = (int64_t)I.voff + row;
        float d[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int off = 8 * ch + 4 * h;
            const float4 p = ld4(a.P + vrow * kM + off);
            const float4 q = ld4(a.Q + vrow * kM + off);
            const float4 x = ld4(a.XW + vrow * kM + off);
            const float4 r = ld4(a.R + vrow * kM + off);
            const float4 xn = make_float4(fmaf(sv[off + 0], p.x, x.x), fmaf(sv[off + 1], p.y, x.y),
                                          fmaf(sv[off + 2], p.z, x.z), fmaf(sv[off + 3], p.w, x.w));
            const float4 rn = make_float4(fmaf(-sv[off + 0], q.x, r.x), fmaf(-sv[off + 1], q.y, r.y),
                                          fmaf(-sv[off + 2], q.z, r.z), fmaf(-sv[off + 3], q.w, r.w));
            st4(a.XW + vrow * kM + off, xn);
            st4(a.R + vrow * kM + off, rn);
            d[4 * h + 0] = rn.x * rn.x;
            d[4 * h + 1] = rn.y * rn.y;
            d[4 * h + 2] = rn.z * rn.z;
            d[4 * h + 3] = rn.w * rn.w;
        }
        const double tr = colsum_rv(d, wsum, w, lane);
        if (w == 0 && lane < 16) a.p_rr[((int64_t)I.boff + item.y) * kM + lane] = tr;
    }
}

// End of a correction solve: X += |R64| X_w, then X = x_hi + x_lo for the
// residual pass.
__device__ __forceinline__ void step_back(const BArgs& a, double* wsumd, int tid, int w, int lane) {
    int i0, i1;
    my_range(a.nrows, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 item = a.rows[it];
        const BInst& I = a.inst[item.x];
        if (!ld_volatile(&a.istep[item.x])) continue;
        const int row = item.y * kRB + (tid >> 1), ch = tid & 1;
        const int64_t vrow = (int64_t)I.voff + row;
        float xh[8], xl[8];
        double d[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int col = 8 * ch + c8;
            double x = 0.0;
            if (row < I.n && col < I.m) {
                double* xp = I.X + (int64_t)col * I.ldx + row;
                x = *xp + a.scale[item.x * kM + col] * (double)a.XW[vrow * kM + col];
                *xp = x;
            }
            xh[c8] = (float)x;
            xl[c8] = (float)(x - (double)xh[c8]);
            d[c8] = x * x;
        }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int o = 2; o < 32; o <<= 1) d[c8] += __shfl_xor_sync(0xffffffffu, d[c8], o);
        if (lane < 2)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) wsumd[w * 16 + 8 * lane + c8] = d[c8];
        msp::bar_workers<kWorkers>();
        if (w == 0 && lane < 16) {
            double t = 0.0;
            for (int ww = 0; ww < kWorkWarps; ++ww) t += wsumd[ww * 16 + lane];
            a.p_xx[((int64_t)I.boff + item.y) * kM + lane] = t;
        }
        msp::bar_workers<kWorkers>();
        st4(a.XH + vrow * kM + 8 * ch, make_float4(xh[0], xh[1], xh[2], xh[3]));
        st4(a.XH + vrow * kM + 8 * ch + 4, make_float4(xh[4], xh[5], xh[6], xh[7]));
        st4(a.XL + vrow * kM + 8 * ch, make_float4(xl[0], xl[1], xl[2], xl[3]));
        st4(a.XL + vrow * kM + 8 * ch + 4, make_float4(xl[4], xl[5], xl[6], xl[7]));
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_batch_solve(BArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float* red = reinterpret_cast<float*>(smem + kRingBytes);
    unsigned char* misc = smem + kRingBytes + kRedBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(misc);
    uint64_t* empty = full + kStages;
    int2* hdr = reinterpret_cast<int2*>(misc + 64);
    float* wsum = reinterpret_cast<float*>(misc + 128);       // 8 x 16 (FP32 or FP64)
    double* wsumd = reinterpret_cast<double*>(misc + 128);
    float* sv = reinterpret_cast<float*>(misc + 1152);        // 16 per-column scalars
    double* sd = reinterpret_cast<double*>(misc + 1280);      // 16 per-column scalars
    int* slot = reinterpret_cast<int*>(misc + 1408);          // claimed item index
    int* sflag = reinterpret_cast<int*>(misc + 1412);         // last-unit flag

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool worker = w < kWorkWarps;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            msp::mbar_init(&full[s], 1);
            msp::mbar_init(&empty[s], kWorkWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    BCtl* ctl = a.ctl;
    uint32_t kring = 0;
    uint64_t t_last = msp::globaltimer_ns();
    const bool timer = blockIdx.x == 0 && tid == 0;
#define MSP_GBAR(cls)                                                                  \
    do {                                                                               \
        if (!msp::grid_barrier(&ctl->bar_word, &ctl->error)) return;   \
        if (ld_volatile(&ctl->error)) return;                                          \
        if (timer) {                                                                   \
            const uint64_t now = msp::globaltimer_ns();                                \
            ctl->t_ns[cls] += now - t_last;                                            \
            t_last = now;                                                              \
        }                                                                              \
    } while (0)

    if (worker) step_init(a, wsumd, tid, w, lane);
    MSP_GBAR(kTCheck);
    for (int step = 0;; ++step) {
        step_check(a, step, w, lane);
        MSP_GBAR(kTCheck);
        const int unf = ld_volatile(&ctl->unfinished[step & 1]);
        if (unf == 0 || step >= a.max_steps) break;
        if (worker) step_scale(a, step, wsum, sd, tid, w, lane);
        MSP_GBAR(kTCheck);
        for (int t = 0;; ++t) {
            if (worker) {
                if (w == 0) step_flags(a, t, lane);
                consume_G(a, ring, full, empty, hdr, kring, red, w, lane);
            } else if (lane == 0) {
                producer<kModeG>(a, ring, full, empty, hdr, kring, &ctl->ctrG, a.iact + ((t + 1) & 1) * a.count);
            }
            MSP_GBAR(kTG);
            if (ld_volatile(&ctl->active[t & 1]) == 0) break;
            if (blockIdx.x == 0 && tid == 0) {
                ctl->active[(t + 1) & 1] = 0;
                ctl->sweepsA += 1;
            }
            if (worker) step_tri<false>(a, t, smem, red, slot, tid, w, lane);
            MSP_GBAR(kTTri);
            if (worker) step_tri<true>(a, t, smem, red, slot, tid, w, lane);
            MSP_GBAR(kTTri);
            if (worker) consume_Z(a, ring, full, empty, hdr, kring, red, wsum, w, lane);
            else if (lane == 0)
                producer<kModeZ>(a, ring, full, empty, hdr, kring, &ctl->ctrZ, a.iact + (t & 1) * a.count);
            MSP_GBAR(kTZ);
            if (worker) step_P(a, t, sv, tid, w, lane);
            MSP_GBAR(kTVec);
            if (worker) consume_A(a, ring, full, empty, hdr, kring, red, wsum, sflag, w, lane);
            else if (lane == 0)
                producer<kModeA>(a, ring, full, empty, hdr, kring, &ctl->ctrA, a.iact + (t & 1) * a.count);
            MSP_GBAR(kTA);
            if (worker) step_X(a, t, wsum, sv, tid, w, lane);
            MSP_GBAR(kTVec);
        }
        if (worker) step_back(a, wsumd, tid, w, lane);
        MSP_GBAR(kTResid);
        if (blockIdx.x == 0 && tid == 0) ctl->sweepsR += 1;
        if (worker)
            consume_R(a, ring, full, empty, hdr, kring, reinterpret_cast<double*>(red), wsumd, sflag, w, lane);
        else if (lane == 0)
            producer<kModeR>(a, ring, full, empty, hdr, kring, &ctl->ctrR, a.istep);
        MSP_GBAR(kTResid);
    }
#undef MSP_GBAR
}

// Copy a rows x cols row-major matrix (lda) into the swizzled tile layout,
// zero-padded: A itself, and the sketch C for the Z step.
__global__ void __launch_bounds__(256) k_pack_tiles(const float* __restrict__ A, int64_t lda, int n,
                                                   int ncols, int nk, float* __restrict__ At) {
    const int tile = blockIdx.x, I = tile / nk, K = tile % nk;
    float* dst = At + (int64_t)tile * kTileFloats;
    const bool vec = (lda % 4 == 0) && (((uintptr_t)A & 15) == 0);
    for (int e = threadIdx.x; e < kRB * 16; e += blockDim.x) {
        const int r = e >> 4, g = e & 15;
        const int64_t gr = (int64_t)I * kRB + r, gc = (int64_t)K * kKT + 4 * g;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr < n) {
            if (vec && gc + 4 <= ncols) {
                v = __ldcs(reinterpret_cast<const float4*>(A + gr * lda + gc));
            } else {
                if (gc + 0 < ncols) v.x = A[gr * lda + gc + 0];
                if (gc + 1 < ncols) v.y = A[gr * lda + gc + 1];
                if (gc + 2 < ncols) v.z = A[gr * lda + gc + 2];
                if (gc + 3 < ncols) v.w = A[gr * lda + gc + 3];
            }
        }
        reinterpret_cast<float4*>(dst)[r * 16 + (g ^ (r & 7))] = v;
    }
}

std::atomic<bool> g_attr_set[64];

}  // namespace

// ------------------------------------------------------------------ host

struct msp_batch_s {
    int count = 0;
    std::vector<msp_instance> inst;
    std::vector<msp_sketch_t*> sk;
    std::vector<msp_factor_t*> f;
    std::vector<BInst> hinst;
    std::vector<int2> rows, strips, chunks, units;
    void* mem = nullptr;
    cudaStream_t stream = nullptr;
    BArgs args{};
    int device = 0;
    int last_max_steps = 0;
    int last_mixed = 1;
    double last_tol = 0.0;
    int last_crit = 0;
    std::vector<int> by_n;      // instances, largest n first
    std::vector<int> dup;       // first identical instance (shared set-up), or -1
    BInst* d_inst = nullptr;    // device copy of hinst
};

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Worker contexts for concurrent set-up: one stream and one host thread each.
msp_status ensure_lanes(msp_ctx* ctx, int want) {
    if (ctx->n_lanes >= want) return MSP_OK;
    msp_ctx** nl = new (std::nothrow) msp_ctx*[want]();
    cudaStream_t* ns = new (std::nothrow) cudaStream_t[want]();
    if (!nl || !ns) {
        delete[] nl;
        delete[] ns;
        return msp_set_error(ctx, MSP_ENOMEM, "batch: host allocation failed");
    }
    for (int i = 0; i < ctx->n_lanes; ++i) {
        nl[i] = ctx->lanes[i];
        ns[i] = ctx->lane_streams[i];
    }
    int made = ctx->n_lanes;
    msp_status st = MSP_OK;
    for (; made < want; ++made) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = msp_set_error(ctx, MSP_ECUDA, "batch: cudaStreamCreate failed");
            break;
        }
        msp_ctx* l = nullptr;
        if (msp_create(&l, ctx->device, s) != MSP_OK) {
            cudaStreamDestroy(s);
            st = msp_set_error(ctx, MSP_ECUDA, "batch: worker context: %s", msp_last_error(nullptr));
            break;
        }
        // the lanes already factor several instances at once: no side
        // streams inside each factor
        l->fac_overlap = false;
        nl[made] = l;
        ns[made] = s;
    }
    delete[] ctx->lanes;
    delete[] ctx->lane_streams;
    ctx->lanes = nl;
    ctx->lane_streams = ns;
    ctx->n_lanes = made;
    return st;
}

msp_status check_instance(msp_ctx* ctx, int k, const msp_instance& I) {
    if (!I.A || !I.B || !I.X)
        return msp_set_error(ctx, MSP_EINVAL, "batch: instance %d has a NULL A, B or X", k);
    if (I.n < 16 || I.n > 65536 || I.lda < I.n || I.ldb < I.n || I.ldx < I.n)
        return msp_set_error(ctx, MSP_EINVAL,
                             "batch: instance %d needs 16 <= n <= 65536 and lda, ldb, ldx >= n", k);
    if (I.m < 1 || I.m > kM)
        return msp_set_error(ctx, MSP_EINVAL, "batch: instance %d needs 1 <= m <= 16 (m = %d)", k, I.m);
    if (!(I.lambda > 0.0) || !std::isfinite(I.lambda) || !(I.lambda0 >= 0.0) || !std::isfinite(I.lambda0))
        return msp_set_error(ctx, MSP_EINVAL, "batch: instance %d needs lambda > 0, lambda0 >= 0", k);
    if (I.s < 16 || I.s > std::min<int64_t>(I.n, MSP_MAX_S) || I.gamma < 1 || I.gamma > MSP_MAX_GAMMA ||
        I.gamma > I.s)
        return msp_set_error(ctx, MSP_EINVAL,
                             "batch: instance %d needs 16 <= s <= min(n, %d), 1 <= gamma <= min(s, %d)", k,
                             MSP_MAX_S, MSP_MAX_GAMMA);
    return MSP_OK;
}

// Units of width ut (tiles): per-instance unit counts, partial-buffer
// offsets and the unit list (largest first; the last unit of a row block may
// be shorter), uploaded with the instance table.
msp_status set_units(msp_ctx* ctx, msp_batch_s* b, int ut) {
    std::vector<std::pair<int, int2>> us;
    int64_t nq = 0;
    for (BInst& H : b->hinst) {
        const int nk = H.n_pad / kKT;
        H.nkc = (nk + ut - 1) / ut;
        H.qoff = (int)nq;
        if (H.nkc > 1) nq += (int64_t)H.nkc * H.n_pad;
    }
    for (int k : b->by_n) {
        const BInst& H = b->hinst[k];
        const int nk = H.n_pad / kKT;
        for (int r = 0; r < H.nb; ++r)
            for (int c = 0; c < H.nkc; ++c)
                us.push_back({std::min(nk, (c + 1) * ut) - c * ut, make_int2(k, r | (c << 16))});
    }
    std::stable_sort(us.begin(), us.end(), [](const std::pair<int, int2>& x, const std::pair<int, int2>& y) {
        return x.first > y.first;
    });
    b->units.clear();
    for (const auto& u : us) b->units.push_back(u.second);
    b->args.ut = ut;
    b->args.nunits = (int)b->units.size();
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync((void*)b->args.units, b->units.data(), sizeof(int2) * b->units.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(b->d_inst, b->hinst.data(), sizeof(BInst) * b->hinst.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
    // pageable sources: the copies complete before the host vectors change
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return MSP_OK;
}

void destroy_parts(msp_batch_s* b) {
    for (size_t k = 0; k < b->f.size(); ++k)
        if (b->dup.empty() || b->dup[k] < 0) msp_factor_destroy(b->f[k]);
    for (size_t k = 0; k < b->sk.size(); ++k)
        if (b->dup.empty() || b->dup[k] < 0) msp_sketch_destroy(b->sk[k]);
    b->f.clear();
    b->sk.clear();
    if (b->mem) cudaFreeAsync(b->mem, b->stream);
    b->mem = nullptr;
}

}  // namespace

extern "C" {

void msp_batch_destroy(msp_batch_t* b) {
    if (!b) return;
    destroy_parts(b);
    delete b;
}

msp_status msp_batch_create(msp_ctx* ctx, int count, const msp_instance* inst, msp_batch_t** out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!out || !inst || count < 1 || count > (1 << 20))
        return msp_set_error(ctx, MSP_EINVAL, "batch: need count >= 1 and non-NULL inst/out");
    *out = nullptr;
    for (int k = 0; k < count; ++k) MSP_TRY(check_instance(ctx, k, inst[k]));
    msp::DeviceGuard guard(ctx->device);
    if (ctx->smem_optin < kSmem)
        return msp_set_error(ctx, MSP_EINVAL, "batch: needs %zu bytes of shared memory per block (device has %zu)",
                             kSmem, ctx->smem_optin);
    msp_batch_s* b = new (std::nothrow) msp_batch_s();
    if (!b) return msp_set_error(ctx, MSP_ENOMEM, "batch: host allocation failed");
    b->count = count;
    b->device = ctx->device;
    b->stream = ctx->stream;
    b->inst.assign(inst, inst + count);
    b->sk.assign(count, nullptr);
    b->f.assign(count, nullptr);
    auto fail = [&](msp_status st) {
        cudaStreamSynchronize(ctx->stream);
        msp_batch_destroy(b);
        return st;
    };

    // ---- set-up of every instance on worker streams (largest first)
    const int nl = std::min(count, 16);
    {
        const msp_status st = ensure_lanes(ctx, nl);
        if (st != MSP_OK) return fail(st);
    }
    cudaEvent_t ev = nullptr;
    MSP_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (cudaEventRecord(ev, ctx->stream) != cudaSuccess) {
        cudaEventDestroy(ev);
        return fail(msp_set_error(ctx, MSP_ECUDA, "batch: cudaEventRecord failed"));
    }
    // instances that differ only in B / X / m share the sketch, the factor
    // and the tiled copies of A and C (the same system with more right-hand
    // sides than one instance holds)
    b->dup.assign(count, -1);
    {
        std::map<std::tuple<const float*, int64_t, int64_t, double, double, int64_t, int, int64_t, int, uint64_t>,
                 int> first;
        for (int k = 0; k < count; ++k) {
            const msp_instance& I = inst[k];
            const auto key = std::make_tuple(I.A, I.n, I.lda, I.lambda, I.lambda0, I.s, I.gamma, I.phi,
                                             I.gamma_phi, I.seed);
            const auto it = first.find(key);
            if (it == first.end()) first.emplace(key, k);
            else b->dup[k] = it->second;
        }
    }
    std::vector<int> order;
    for (int k = 0; k < count; ++k)
        if (b->dup[k] < 0) order.push_back(k);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return inst[x].n * inst[x].s > inst[y].n * inst[y].s; });
    const int nuniq = (int)order.size();
    std::atomic<int> next{0};
    std::atomic<int> bad{-1};
    std::vector<msp_status> lst(nl, MSP_OK);
    std::vector<std::string> lmsg(nl);
    auto work = [&](int li) {
        msp_ctx* L = ctx->lanes[li];
        cudaSetDevice(ctx->device);
        if (cudaStreamWaitEvent(L->stream, ev, 0) != cudaSuccess) {
            lst[li] = msp_set_error(L, MSP_ECUDA, "batch: cudaStreamWaitEvent failed");
            bad = li;
            return;
        }
        while (bad.load() < 0) {
            const int j = next.fetch_add(1);
            if (j >= nuniq) break;
            const int k = order[j];
            const msp_instance& I = inst[k];
            msp_sketch_t* sk = nullptr;
            msp_factor_t* f = nullptr;
            msp_status st = msp_sketch_impl(L, I.A, MSP_F32, I.n, I.lda, I.s, I.gamma, I.seed, false, &sk);
            if (st == MSP_OK) st = msp_nystrom_impl(L, sk, I.lambda, I.lambda0, I.phi, I.gamma_phi, I.seed, &f);
            if (st != MSP_OK) {
                if (sk) msp_sketch_destroy(sk);
                lst[li] = st;
                lmsg[li] = std::string("instance ") + std::to_string(k) + ": " + L->last_error;
                bad = li;
                break;
            }
            b->sk[k] = sk;
            b->f[k] = f;
        }
        if (cudaStreamSynchronize(L->stream) != cudaSuccess && lst[li] == MSP_OK) {
            lst[li] = MSP_ECUDA;
            lmsg[li] = "worker stream failed";
            bad = li;
        }
    };
    {
        std::vector<std::thread> th;
        th.reserve(nl);
        for (int li = 0; li < nl; ++li) th.emplace_back(work, li);
        for (auto& t : th) t.join();
    }
    cudaEventDestroy(ev);
    if (bad.load() >= 0) {
        const int li = bad.load();
        return fail(msp_set_error(ctx, lst[li] != MSP_OK ? lst[li] : MSP_ECUDA, "batch: %s", lmsg[li].c_str()));
    }
    // handles are freed on the main stream from now on (worker work is complete)
    for (int k = 0; k < count; ++k) {
        if (b->dup[k] >= 0) {
            b->sk[k] = b->sk[b->dup[k]];
            b->f[k] = b->f[b->dup[k]];
            continue;
        }
        b->sk[k]->stream = ctx->stream;
        b->f[k]->stream = ctx->stream;
    }

    // ---- layout
    int64_t nv = 0, ns = 0, nbt = 0, at = 0, nq = 0;
    b->hinst.resize(count);
    for (int k = 0; k < count; ++k) {
        const msp_instance& I = inst[k];
        BInst& H = b->hinst[k];
        H.n = (int)I.n;
        H.n_pad = (int)round_up(I.n, kRB);
        H.s_pad = (int)b->sk[k]->s_pad;
        H.m = I.m;
        H.nb = H.n_pad / kRB;
        H.voff = (int)nv;
        H.soff = (int)ns;
        H.boff = (int)nbt;
        H.nkc = (H.n_pad / kKT + kUtMin - 1) / kUtMin;   // the most units (smallest width)
        H.qoff = (int)nq;
        H.lam = (float)I.lambda;
        H.lam64 = I.lambda;
        H.inv_lt = (float)(1.0 / b->f[k]->lam_tilde);
        H.ldb = I.ldb;
        H.ldx = I.ldx;
        H.B = I.B;
        H.X = I.X;
        nv += H.n_pad;
        ns += H.s_pad;
        nbt += H.nb;
        if (H.nkc > 1) nq += (int64_t)H.nkc * H.n_pad;
        if (b->dup[k] < 0) at += (int64_t)H.n_pad * H.n_pad;
    }
    if (nv * kM >= (1ll << 31) || nq * kM >= (1ll << 31) || nbt >= (1 << 30))
        return fail(msp_set_error(ctx, MSP_EINVAL, "batch: total size too large"));
    // row items: largest instance first (dynamic scheduling then balances)
    std::vector<int> by_n(count);
    for (int k = 0; k < count; ++k) by_n[k] = k;
    std::stable_sort(by_n.begin(), by_n.end(), [&](int x, int y) { return inst[x].n > inst[y].n; });
    for (int k : by_n)
        for (int r = 0; r < b->hinst[k].nb; ++r) b->rows.push_back(make_int2(k, r));
    for (int k : by_n)
        for (int s = 0; s < b->hinst[k].s_pad / kKT; ++s) b->strips.push_back(make_int2(k, s));
    for (int k : by_n)
        for (int s = 0; s < b->hinst[k].s_pad / kRB; ++s) b->chunks.push_back(make_int2(k, s));
    b->by_n = by_n;
    // room for the units list at the smallest width
    size_t max_units = 0;
    for (const BInst& H : b->hinst) max_units += (size_t)H.nb * H.nkc;

    const int cnt = count;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_at = take((size_t)at * 4);
    int64_t ct_total = 0;
    for (int k = 0; k < count; ++k)
        if (b->dup[k] < 0) ct_total += (int64_t)b->hinst[k].n_pad * b->hinst[k].s_pad;
    const size_t o_ct = take((size_t)ct_total * 4);
    const size_t o_inst = take(sizeof(BInst) * cnt);
    const size_t o_rows = take(sizeof(int2) * b->rows.size());
    const size_t o_strips = take(sizeof(int2) * b->strips.size());
    const size_t o_chunks = take(sizeof(int2) * b->chunks.size());
    const size_t o_units = take(sizeof(int2) * max_units);
    const size_t o_vec = off;
    const size_t vbytes = (size_t)nv * kM * 4;
    size_t o_v[7];
    for (int q = 0; q < 7; ++q) o_v[q] = take(vbytes);
    const size_t o_r64 = take((size_t)nv * kM * 8);
    const size_t sbytes = (size_t)ns * kM * 4;
    const size_t o_g = take(sbytes), o_y1 = take(sbytes), o_y2 = take(sbytes);
    const size_t pbytes = (size_t)nbt * kM * 8;
    size_t o_p[6];
    for (int q = 0; q < 6; ++q) o_p[q] = take(pbytes);
    const size_t cbytes = (size_t)cnt * kM * 8;
    const size_t o_bb = take(cbytes), o_sc = take(cbytes), o_al = take(cbytes), o_rz = take(2 * cbytes);
    const size_t o_act = take((size_t)cnt * kM * 4), o_fin = take((size_t)cnt * kM * 4);
    const size_t o_iact = take((size_t)cnt * 8);
    const size_t o_istep = take((size_t)cnt * 4), o_iters = take((size_t)cnt * 4);
    const size_t o_ierr = take((size_t)cnt * 4), o_isteps = take((size_t)cnt * 4);
    const size_t o_rel = take((size_t)cnt * 8), o_berr = take((size_t)cnt * 8);
    const size_t o_anorm = take((size_t)cnt * 8);
    int64_t nmax = 0;
    for (int k = 0; k < count; ++k) nmax = std::max<int64_t>(nmax, inst[k].n);
    const size_t o_nwork = take((size_t)nmax * 24);
    const size_t o_qp = take((size_t)std::max<int64_t>(nq, 1) * kM * 4);
    const size_t o_rp = take((size_t)std::max<int64_t>(nq, 1) * kM * 8);
    const size_t o_rbcnt = take((size_t)nbt * 4);
    const size_t o_ctl = take(sizeof(BCtl));
    const size_t total = off;
    if (cudaMallocAsync(&b->mem, total, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        b->mem = nullptr;
        return fail(msp_set_error(ctx, MSP_ENOMEM, "batch: device allocation of %zu bytes failed", total));
    }
    char* base = (char*)b->mem;
    int64_t ta = 0, tc = 0;
    for (int k = 0; k < count; ++k) {
        BInst& H = b->hinst[k];
        if (b->dup[k] >= 0) {
            H.At = b->hinst[b->dup[k]].At;
            H.Ct = b->hinst[b->dup[k]].Ct;
        } else {
            H.At = (const float*)(base + o_at) + ta;
            H.Ct = (const float*)(base + o_ct) + tc;
            tc += (int64_t)H.n_pad * H.s_pad;
            ta += (int64_t)H.n_pad * H.n_pad;
        }
        H.C = (const float*)b->sk[k]->C;
        H.Bl = (const float*)b->f[k]->B;
        H.Bu = (const float*)b->f[k]->Bt;
    }
    // A -> tiles
    for (int k = 0; k < count; ++k) {
        if (b->dup[k] >= 0) continue;
        const BInst& H = b->hinst[k];
        const int nk = H.n_pad / kKT;
        const int tiles = H.nb * nk;
        k_pack_tiles<<<tiles, 256, 0, ctx->stream>>>(inst[k].A, inst[k].lda, H.n, H.n, nk, (float*)H.At);
        if (cudaGetLastError() != cudaSuccess) return fail(msp_set_error(ctx, MSP_ECUDA, "batch: pack launch failed"));
        ++ctx->launches;
        const int nkc = H.s_pad / kKT;
        k_pack_tiles<<<H.nb * nkc, 256, 0, ctx->stream>>>(H.C, H.s_pad, H.n, H.s_pad, nkc, (float*)H.Ct);
        if (cudaGetLastError() != cudaSuccess) return fail(msp_set_error(ctx, MSP_ECUDA, "batch: pack launch failed"));
        ++ctx->launches;
    }
    auto h2d = [&](size_t o, const void* src, size_t bytes) {
        return cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
    };
    if (h2d(o_inst, b->hinst.data(), sizeof(BInst) * cnt) != cudaSuccess ||
        h2d(o_rows, b->rows.data(), sizeof(int2) * b->rows.size()) != cudaSuccess ||
        h2d(o_strips, b->strips.data(), sizeof(int2) * b->strips.size()) != cudaSuccess ||
        h2d(o_chunks, b->chunks.data(), sizeof(int2) * b->chunks.size()) != cudaSuccess ||
        cudaMemsetAsync(base + o_vec, 0, total - o_vec, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(msp_set_error(ctx, MSP_ECUDA, "batch: descriptor upload failed"));
    }
    BArgs& A = b->args;
    A.inst = (const BInst*)(base + o_inst);
    A.count = cnt;
    A.nrows = (int)b->rows.size();
    A.nstrips = (int)b->strips.size();
    A.nchunks = (int)b->chunks.size();
    A.rows = (const int2*)(base + o_rows);
    A.strips = (const int2*)(base + o_strips);
    A.chunks = (const int2*)(base + o_chunks);
    A.units = (const int2*)(base + o_units);
    A.Qp = (float*)(base + o_qp);
    A.Rp = (double*)(base + o_rp);
    A.rbcnt = (int*)(base + o_rbcnt);
    b->d_inst = (BInst*)(base + o_inst);
    float** vp[7] = {&A.P, &A.Q, &A.R, &A.Z, &A.XW, &A.XH, &A.XL};
    for (int q = 0; q < 7; ++q) *vp[q] = (float*)(base + o_v[q]);
    A.R64 = (double*)(base + o_r64);
    A.G = (float*)(base + o_g);
    A.Y1 = (float*)(base + o_y1);
    A.Y2 = (float*)(base + o_y2);
    double** pp[6] = {&A.p_pq, &A.p_rr, &A.p_zr, &A.p_zq, &A.p_r64, &A.p_xx};
    for (int q = 0; q < 6; ++q) *pp[q] = (double*)(base + o_p[q]);
    A.bb = (double*)(base + o_bb);
    A.scale = (double*)(base + o_sc);
    A.alpha = (double*)(base + o_al);
    A.rz = (double*)(base + o_rz);
    A.act = (int*)(base + o_act);
    A.fin = (int*)(base + o_fin);
    A.iact = (int*)(base + o_iact);
    A.istep = (int*)(base + o_istep);
    A.iters = (int*)(base + o_iters);
    A.ierr = (int*)(base + o_ierr);
    A.isteps = (int*)(base + o_isteps);
    A.rel = (double*)(base + o_rel);
    A.berr = (double*)(base + o_berr);
    A.anorm = (const double*)(base + o_anorm);
    A.ctl = (BCtl*)(base + o_ctl);
    // L <= |A_k|_2 for the backward-error rule (one pass over each A)
    for (int k = 0; k < count; ++k) {
        double* dst = (double*)(base + o_anorm) + k;
        if (b->dup[k] >= 0) {
            MSP_CUDA_TRY(ctx, cudaMemcpyAsync(dst, (double*)(base + o_anorm) + b->dup[k], 8,
                                              cudaMemcpyDeviceToDevice, ctx->stream));
            continue;
        }
        const msp_status st = msp_norm_lb_launch(ctx, inst[k].A, MSP_F32, inst[k].n, inst[k].lda,
                                                 (double*)(base + o_nwork), dst);
        if (st != MSP_OK) return fail(st);
    }
    {
        // default width: the widest whose units still number 8 per SM
        int ut = kUtMin;
        for (int cand : {256, 128, 64, 32, 16}) {
            size_t nu = 0;
            for (const BInst& H : b->hinst) nu += (size_t)H.nb * ((H.n_pad / kKT + cand - 1) / cand);
            if (nu >= (size_t)8 * ctx->num_sms) {
                ut = cand;
                break;
            }
        }
        const msp_status st = set_units(ctx, b, ut);
        if (st != MSP_OK) return fail(st);
    }
    // the host copies above are from pageable memory: complete before return
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *out = b;
    return MSP_OK;
}

msp_status msp_batch_solve(msp_ctx* ctx, msp_batch_t* b, const msp_opts* opts, msp_info* infos) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!b) return msp_set_error(ctx, MSP_EINVAL, "batch_solve: batch is NULL");
    if (b->device != ctx->device) return msp_set_error(ctx, MSP_EINVAL, "batch_solve: batch is on another device");
    msp_opts o;
    if (opts) o = *opts; else msp_default_opts(&o);
    if (!(o.tol > 0.0) || o.max_outer < 1 || o.max_refine < 0)
        return msp_set_error(ctx, MSP_EINVAL, "batch_solve: bad options");
    if (o.precision != MSP_PREC_MIXED && o.precision != MSP_PREC_FP32)
        return msp_set_error(ctx, MSP_EINVAL, "batch_solve: precision must be MSP_PREC_MIXED or MSP_PREC_FP32");
    msp::DeviceGuard guard(ctx->device);
    const bool mixed = o.precision == MSP_PREC_MIXED;
    if (o.criterion != MSP_STOP_RESIDUAL && o.criterion != MSP_STOP_BACKWARD)
        return msp_set_error(ctx, MSP_EINVAL, "batch_solve: unknown criterion %d", o.criterion);
    BArgs a = b->args;
    a.crit = o.criterion;
    a.tol = o.tol;
    a.tol2 = o.tol * o.tol;
    const double rt = mixed ? std::max(o.refine_tol, o.tol) : o.tol;
    a.rtol2 = rt * rt;
    a.max_outer = o.max_outer;
    a.max_steps = mixed ? o.max_refine + 1 : 1;
    b->last_max_steps = a.max_steps;
    b->last_mixed = mixed ? 1 : 0;
    b->last_tol = o.tol;
    b->last_crit = o.criterion;
    // per-solve state: control block and per-instance counters
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(a.ctl, 0, sizeof(BCtl), ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(a.iters, 0, (size_t)a.count * 4, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(a.ierr, 0, (size_t)a.count * 4, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(a.isteps, 0, (size_t)a.count * 4, ctx->stream));
    // unit counters (left at zero by a completed pass; cleared in case the
    // last solve stopped inside one)
    MSP_CUDA_TRY(ctx, cudaMemsetAsync(a.rbcnt, 0, (size_t)(b->hinst.back().boff + b->hinst.back().nb) * 4,
                                      ctx->stream));
    const int d = ctx->device;
    if (d >= 0 && d < 64 && !g_attr_set[d].load()) {
        MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmem));
        g_attr_set[d] = true;
    }
    int per_sm = 0;
    MSP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_solve, kThreads, kSmem));
    if (per_sm < 1) return msp_set_error(ctx, MSP_ECUDA, "batch_solve: kernel does not fit on an SM");
    const int grid = ctx->num_sms;
    void* args[] = {&a};
    MSP_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_batch_solve, dim3(grid), dim3(kThreads), args,
                                                  kSmem, ctx->stream));
    ++ctx->launches;
    if (!infos) return MSP_OK;
    return msp_batch_info(ctx, b, infos);
}

msp_status msp_batch_info(msp_ctx* ctx, const msp_batch_t* b, msp_info* infos) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!b || !infos) return msp_set_error(ctx, MSP_EINVAL, "batch_info: NULL argument");
    msp::DeviceGuard guard(ctx->device);
    const int cnt = b->count;
    std::vector<int> iters(cnt), ierr(cnt), steps(cnt);
    std::vector<double> rel(cnt), berr(cnt), anorm(cnt);
    BCtl ctl;
    const BArgs& a = b->args;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(berr.data(), a.berr, cnt * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(anorm.data(), a.anorm, cnt * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(iters.data(), a.iters, cnt * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(ierr.data(), a.ierr, cnt * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(steps.data(), a.isteps, cnt * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(rel.data(), a.rel, cnt * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(&ctl, a.ctl, sizeof ctl, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    msp_status first = MSP_OK;
    for (int k = 0; k < cnt; ++k) {
        msp_info& I = infos[k];
        std::memset(&I, 0, sizeof I);
        // batch-wide device-timer split of the one launch (same in every entry)
        I.gemv_launches = ctl.sweepsA;
        I.resid_launches = ctl.sweepsR;
        I.gemv_ms = 1e-6 * (double)ctl.t_ns[kTA];
        I.level2_ms = 1e-6 * (double)(ctl.t_ns[kTG] + ctl.t_ns[kTTri] + ctl.t_ns[kTZ] + ctl.t_ns[kTVec]);
        I.resid_ms = 1e-6 * (double)ctl.t_ns[kTResid];
        I.outer_iters = iters[k];
        I.refine_steps = steps[k];
        I.rel_resid = rel[k];
        I.backward_err = berr[k];
        I.norm_lb = anorm[k];
        I.lambda_tilde = b->f[k]->lam_tilde;
        I.shift = b->f[k]->shift;
        I.shift_retries = b->f[k]->retries;
        msp_status st = (msp_status)ierr[k];
        if (st == MSP_OK && ctl.error) st = (msp_status)ctl.error;
        const double achieved = b->last_crit == MSP_STOP_BACKWARD ? berr[k] : rel[k];
        if (st == MSP_OK && b->last_mixed && !(achieved <= b->last_tol)) st = MSP_ENOCONV;
        I.status = st;
        if (first == MSP_OK && st != MSP_OK) first = st;
    }
    if (ctl.error)
        return msp_set_error(ctx, (msp_status)ctl.error, "batch_solve: device error %d (wait limit or fault)",
                             ctl.error);
    if (first != MSP_OK)
        return msp_set_error(ctx, first, "batch_solve: at least one instance ended with status %d", (int)first);
    return MSP_OK;
}

msp_status msp_batch_stats(msp_ctx* ctx, const msp_batch_t* b, double* stats) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!b || !stats) return msp_set_error(ctx, MSP_EINVAL, "batch_stats: NULL argument");
    msp::DeviceGuard guard(ctx->device);
    BCtl ctl;
    MSP_CUDA_TRY(ctx, cudaMemcpyAsync(&ctl, b->args.ctl, sizeof ctl, cudaMemcpyDeviceToHost, ctx->stream));
    MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t dense = 0;
    for (const BInst& H : b->hinst) dense += (int64_t)H.n_pad * H.n_pad;
    stats[0] = (double)ctl.sweepsA;
    stats[1] = (double)ctl.sweepsR;
    stats[2] = (double)ctl.tilesA * kTileBytes;
    stats[3] = (double)ctl.tilesR * kTileBytes;
    for (int c = 0; c < kTimerClasses; ++c) stats[4 + c] = 1e-6 * (double)ctl.t_ns[c];
    stats[11] = (double)dense * 4.0;
    stats[13] = (double)ctl.bytesG;
    stats[14] = (double)ctl.bytesZ;
    stats[15] = (double)b->args.ut;
    int64_t nn = 0;
    for (const BInst& H : b->hinst) nn += (int64_t)H.n * H.n;
    stats[12] = (double)nn * 4.0;
    return MSP_OK;
}

msp_status msp_batch_autotune(msp_ctx* ctx, msp_batch_t* b, int* unit_tiles) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!b || !unit_tiles) return msp_set_error(ctx, MSP_EINVAL, "batch_autotune: NULL argument");
    msp::DeviceGuard guard(ctx->device);
    const int want = *unit_tiles;
    if (want > 0) {
        if (want < kUtMin || (want & (want - 1)))
            return msp_set_error(ctx, MSP_EINVAL, "batch_autotune: unit width must be a power of two >= %d",
                                 kUtMin);
        return set_units(ctx, b, want);
    }
    // time the A passes of a fixed number of level-1 iterations at each width
    msp_opts o;
    msp_default_opts(&o);
    o.max_refine = 0;
    o.refine_tol = 1e-300;
    o.tol = 1e-300;
    o.max_outer = 12;
    int nk_max = 1;
    for (const BInst& H : b->hinst) nk_max = std::max(nk_max, H.n_pad / kKT);
    double best = 0.0;
    int best_ut = b->args.ut;
    for (int ut = kUtMin; ut < 2 * nk_max && ut <= 1024; ut *= 2) {
        MSP_TRY(set_units(ctx, b, ut));
        double st[16];
        for (int rep = 0; rep < 2; ++rep) {     // the first run warms caches and clocks
            const msp_status s = msp_batch_solve(ctx, b, &o, nullptr);
            if (s != MSP_OK) return s;
        }
        MSP_TRY(msp_batch_stats(ctx, b, st));
        const double rate = st[4] > 0.0 ? st[2] / st[4] : 0.0;     // bytes per ms of A pass
        if (rate > best) {
            best = rate;
            best_ut = ut;
        }
    }
    MSP_TRY(set_units(ctx, b, best_ut));
    *unit_tiles = best_ut;
    return MSP_OK;
}

msp_status msp_solve_batched(msp_ctx* ctx, int count, const msp_instance* inst, const msp_opts* opts,
                             msp_info* infos) {
    msp_batch_t* b = nullptr;
    MSP_TRY(msp_batch_create(ctx, count, inst, &b));
    std::vector<msp_info> tmp;
    msp_info* dst = infos;
    if (!dst) {
        tmp.resize(count);
        dst = tmp.data();
    }
    const msp_status st = msp_batch_solve(ctx, b, opts, dst);
    cudaStreamSynchronize(ctx->stream);
    msp_batch_destroy(b);
    return st;
}

}  // extern "C"
