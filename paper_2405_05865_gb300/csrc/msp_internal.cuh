// Internal declarations shared by the CUDA translation units of libmsp.
// Nothing here is part of the public ABI (include/msp.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "msp.h"

#define MSP_MAX_GAMMA 64
#define MSP_MAX_S 1024          // batched, general and FP64 sketches
#define MSP_MAX_S_SINGLE 2048   // FP32 sketches of a single system (msp_sketch)
#define MSP_S_ALIGN 128

// ------------------------------------------------------------------ handles

struct msp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string last_error;
    // device control block: barrier words, flags, scalars (see CtlBlock)
    void* ctl = nullptr;
    // pinned host mirror for flag reads
    void* host_flags = nullptr;
    // grow-only scratch for solves and staging of host arguments
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    void* stage = nullptr;       // device staging for host A / b / x
    size_t stage_bytes = 0;
    int64_t launches = 0;        // kernels launched by this context
    // CUDA-event pool for opts.profile (pairs), created lazily
    cudaEvent_t* events = nullptr;
    int n_events = 0;
    // worker contexts (own streams) for concurrent batch set-up, created lazily
    cudaStream_t copy_stream = nullptr;   // host-to-device copies overlapped with compute
    // side streams of the recursive Cholesky, one per recursion depth, and
    // their fork/join events (created once, lazily; an event is re-recorded
    // only after every wait on its previous record has been enqueued)
    cudaStream_t fac_side[8] = {};
    cudaEvent_t fac_ev[8][2] = {};
    // side stream and fork/join events of the sketch's row statistics
    // (created once, lazily)
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t aux_ev[2] = {};
    bool fac_overlap = true;     // false: the factor's products stay on the main stream
    bool gram_tc = true;         // M2 Gram on the tensor cores (false: FP32 pipe, compensated)
    bool factor_ff = true;       // Cholesky of an FP32 factor in float-float (false: FP64)
    bool sketch_sym = true;      // FP32 sketch pass by the symmetric one-pass kernel
    // level-1 iterations of msp_solve replayed as a CUDA graph (capture
    // stream, cached executable, its key and profiling event nodes)
    bool l1_graphs = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t l1_graph = nullptr;
    cudaGraphExec_t l1_exec = nullptr;
    unsigned char l1_key[512] = {};
    size_t l1_key_len = 0;
    cudaGraphNode_t l1_ev_nodes[2] = {};
    int l1_kernels = 0;
    int64_t l1_graph_iters = 0;  // level-1 iterations replayed from the graph
    // the float-float Cholesky inverse of one factor attempt as a CUDA graph
    // (its buffers are scratch, so the executable serves every factor of a
    // size until the scratch moves)
    cudaGraph_t fac_graph = nullptr;
    cudaGraphExec_t fac_exec = nullptr;
    unsigned char fac_key[64] = {};
    size_t fac_key_len = 0;
    int fac_kernels = 0;
    int hutch_terms = 2;         // tensor-core Hutchinson: 2 = two FP16 terms, 3 = three BF16 terms
    msp_ctx** lanes = nullptr;
    cudaStream_t* lane_streams = nullptr;
    int n_lanes = 0;
};

// Launch accounting / optional event timing of one launch site class.
struct ProfSlot {
    double ms = 0.0;
    int launches = 0;
};

struct msp_sketch_s {
    int64_t n = 0, s = 0, s_pad = 0;
    int gamma = 0;
    msp_dtype dtype = MSP_F32;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;   // stream of the creating context (frees)
    int32_t* idx = nullptr;      // n x gamma, columns of Pi per row (sorted)
    int8_t* sgn = nullptr;       // n x gamma
    int32_t* csr_ptr = nullptr;  // s_pad + 1, Pi^T rows (= sketch columns)
    int32_t* csr_ent = nullptr;  // n*gamma entries (j << 1) | negative
    void* C = nullptr;           // n x s_pad, dtype
    float* packed = nullptr;     // FP32 A: upper 128 x 128 tiles (see symv.cu)
    const void* A_src = nullptr; // the A the sketch (and packed copy) came from
    // norm bound of A_src for the backward-error rule: row sums, their
    // rounding bounds and row squares (3 n), then the bound (see norms.cu)
    double* stats = nullptr;
};

struct msp_factor_s {
    const msp_sketch_s* sk = nullptr;
    int64_t s = 0, s_pad = 0, phi = 0;
    double lambda = 0, lambda0 = 0, lam_tilde = 0, shift = 0;
    int retries = 0;
    msp_dtype dtype = MSP_F32;
    cudaStream_t stream = nullptr;
    void* W = nullptr;          // s_pad x s_pad, dtype (working copy)
    void* B = nullptr;          // L^{-1}, s_pad x s_pad, dtype (lower)
    void* Bt = nullptr;         // (L^{-1})^T, dtype (upper)
    double* W64 = nullptr;      // s_pad x s_pad
    double* M2 = nullptr;       // s_pad x s_pad, before shift
    double* Linv64 = nullptr;   // s_pad x s_pad
    // storage of the level-2 data C and W: MSP_F32 (the sketch's C and W
    // above) or MSP_BF16 (Cb, Wb: BF16 roundings; W, M2 and L^{-1} are then
    // formed from the rounded C, so that M = Cb W^{-1} Cb^T + lambda~ I is the
    // preconditioner the level-2 iteration applies)
    msp_dtype data = MSP_F32;
    void* Cb = nullptr;         // n x s_pad BF16
    void* Wb = nullptr;         // s_pad x s_pad BF16
};

// Device control block layout (one per context).
struct CtlBlock {
    unsigned int bar_word;      // grid barrier: generation << 16 | arrivals
    unsigned int bar_spare;
    unsigned int last_block_counter;
    int done;           // level-1 solve converged
    int error;          // msp_status-like error code set on device
    int iters;          // level-1 iterations completed
    int inner_iters;    // level-2 iterations accumulated
    int pad0;
    double alpha;       // level-1 step
    double rz;          // r^T z of the level-1 iteration
    double rr;          // |r|^2
    double bb;          // |rhs|^2
    double tol2;        // tol^2 |rhs|^2
    double pq;
    double beta;
    double scratch[8];
};

// ------------------------------------------------------------------ errors

msp_status msp_set_error(msp_ctx* ctx, msp_status st, const char* fmt, ...);

#define MSP_CUDA_TRY(ctx, call)                                                  \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess) {                                                 \
            return msp_set_error((ctx), _e == cudaErrorMemoryAllocation          \
                                            ? MSP_ENOMEM : MSP_ECUDA,            \
                                 "%s:%d: %s: %s", __FILE__, __LINE__, #call,     \
                                 cudaGetErrorString(_e));                        \
        }                                                                        \
    } while (0)

#define MSP_TRY(expr)                                                            \
    do {                                                                         \
        msp_status _s = (expr);                                                  \
        if (_s != MSP_OK) return _s;                                             \
    } while (0)

#define MSP_CHECK_LAUNCH(ctx)                                                    \
    do {                                                                         \
        ++(ctx)->launches;                                                       \
        MSP_CUDA_TRY(ctx, cudaGetLastError());                                   \
    } while (0)

// ------------------------------------------------------------------ memory

msp_status msp_alloc(msp_ctx* ctx, void** p, size_t bytes);
void msp_free(void* p);
msp_status msp_scratch(msp_ctx* ctx, size_t bytes, void** out);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline size_t dtype_size(msp_dtype t) { return t == MSP_F64 ? 8 : 4; }

// ------------------------------------------------------ device primitives

namespace msp {

// Switch to a device for the duration of a call (restores the caller's).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// SplitMix64 finaliser and the counter-based draw described in msp.h.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t draw(uint64_t seed, uint32_t stream, uint64_t row,
                                         uint32_t q) {
    uint64_t k = ((uint64_t)stream << 56) | (row << 8) | (uint64_t)q;
    return mix64(seed + (k + 1ull) * 0x9E3779B97F4A7C15ull);
}

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wall-clock limit of every device-side wait (ns).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Limit of the grid-wide barriers below, per translation unit (default
// kWaitLimitNs); a unit may let callers lower it (msp_set_grid_wait_limit).
// Read as volatile: the device code never writes it, and a plain read of an
// internal-linkage variable may be folded to its initial value.
static __device__ unsigned long long g_grid_wait_limit_ns = kWaitLimitNs;

__device__ inline unsigned long long grid_wait_limit_ns() {
    return *reinterpret_cast<volatile unsigned long long*>(&g_grid_wait_limit_ns);
}

// Grid-wide barrier for a cooperative (co-resident) launch. One word holds
// the arrival count (low 16 bits) and the generation (high 16 bits): thread
// 0 of every block arrives with one acq_rel atomic add, the last arrival
// adds 2^16 - G (count back to zero, generation + 1) with release
// semantics, the others poll the word with acquire loads until the
// generation moves. One round trip to L2 per arrival (no separate read of
// the generation) and no fence after the wait (the acquire load orders the
// block's later reads); the block barriers on both sides carry the order to
// the other threads. Bounded in wall-clock time: on timeout it records
// MSP_ETIMEOUT in *err and returns false. All blocks must call it equally
// often; at most 65535 blocks.
__device__ inline bool grid_barrier(unsigned int* word, int* err) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        __threadfence();
        unsigned int old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(word) : "memory");
        if ((old & 0xFFFFu) == nb - 1) {
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(word), "r"(0x10000u - nb) : "memory");
        } else {
            const uint64_t t0 = globaltimer_ns();
            const unsigned long long limit = grid_wait_limit_ns();
            unsigned int cur;
            int spins = 0;
            while (true) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(word) : "memory");
                if ((cur ^ old) >> 16) break;
                // the clock after every unsuccessful poll (one register read)
                if (globaltimer_ns() - t0 > limit) {
                    atomicExch(err, (int)MSP_ETIMEOUT);
                    ok = 0;
                    break;
                }
                if (++spins > 16) __nanosleep(40);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace msp

// ------------------------------------------------- cross-unit entry points

// sketch.cu
msp_status msp_pattern_launch(msp_ctx* ctx, int64_t n, int64_t rows, int gamma,
                              uint64_t seed, int stream, int32_t* idx, int8_t* sgn,
                              int32_t* counts);
msp_status msp_build_csr(msp_ctx* ctx, int64_t n, int64_t rows, int gamma,
                         const int32_t* idx, const int8_t* sgn, int32_t* ptr,
                         int32_t* ent);
msp_status msp_sketch_apply(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n,
                            int64_t lda, int64_t s_pad, const int32_t* ptr,
                            const int32_t* ent, int gamma, void* C);
// C = A Pi for an m x n A (rows of C follow the rows of A).
msp_status msp_sketch_apply_rows(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t m, int64_t n,
                                 int64_t lda, int64_t s_pad, const int32_t* ptr,
                                 const int32_t* ent, int gamma, void* C);
// tab[c * (nch + 1) + t] = first entry of column c with row >= t J
msp_status msp_chunk_starts(msp_ctx* ctx, const int32_t* ptr, const int32_t* ent, int64_t s_pad, int J, int nch,
                            int32_t* tab);
// One pass over a symmetric FP32 A (device, 16-byte aligned, lda % 4 == 0,
// n >= 32, s_pad <= 2048): C = A Pi, and optionally the packed upper tiles.
bool msp_sketch_sym_ok(const void* A, int64_t n, int64_t lda, int64_t s_pad, int gamma);
msp_status msp_sketch_sym_pass(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t s_pad,
                               const int32_t* ptr, const int32_t* ent, int gamma, float* C, float* packed);
// The same pass for the 32-row blocks [ib0, ib1) of C only (clamped to the
// blocks up to the last tile column): each block reads the column block
// A[:, 32 ib .. 32 ib + 32), which must be complete. Launches over
// consecutive ranges, in order on one stream, form the whole pass.
msp_status msp_sketch_sym_blocks(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, int64_t s_pad,
                                 const int32_t* ptr, const int32_t* ent, int gamma, float* C, float* packed,
                                 int64_t ib0, int64_t ib1);
// the norm bound from row statistics already in work (3 n doubles)
msp_status msp_norm_lb_finish(msp_ctx* ctx, double* work, int64_t n, double* out_dev);
msp_status msp_gather_rows(msp_ctx* ctx, msp_dtype dt, int64_t rows_out, int64_t width,
                           const int32_t* ptr, const int32_t* ent, const void* in,
                           int64_t ld_in, double scale, void* out, int64_t ld_out);

// api.cu: sketch (pack = also build the packed upper tiles of an FP32 A for
// the single-RHS A pass) and Nystrom factor, without argument re-checks of
// the handles
// host_chunks != NULL: A is the device staging buffer (ld n) and host_chunks
// the host matrix (ld lda); the copy runs in row chunks overlapped with the
// sketch and the packing
msp_status msp_sketch_impl(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n, int64_t lda,
                           int64_t s, int gamma, uint64_t seed, bool pack, msp_sketch_s** out,
                           const void* host_chunks = nullptr);
msp_status msp_nystrom_impl(msp_ctx* ctx, const msp_sketch_s* sk, double lambda, double lambda0,
                            int64_t phi, int gamma_phi, uint64_t seed, msp_factor_s** out,
                            msp_dtype data = MSP_F32);

// norms.cu: L <= |A|_2 into *out_dev; work holds 3n doubles
msp_status msp_norm_lb_launch(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n, int64_t lda,
                              double* work, double* out_dev);

// gram_tc.cu: M2 = X^T X + lam W (W null: + lam I) on the tensor cores
// (two FP16 terms per entry, FP64 across K slices); MSP_EINVAL when the
// tensor-core path is unavailable
msp_status msp_gram_tc(msp_ctx* ctx, const float* X, int64_t K, int64_t ld, int64_t s, int64_t s_pad,
                       const float* W, double lam, double* M2);
bool msp_gram_tc_ok(int64_t s_pad);

// factor.cu
msp_status msp_build_factor(msp_ctx* ctx, msp_factor_s* f, const void* Ct, int64_t phi_rows);
// G64 = X^T X + diag I (FP64, pad identity); M^{-1} of an SPD FP64 matrix;
// C = X^T Y (FP32, compensated) -- see factor.cu
msp_status msp_gram64(msp_ctx* ctx, const float* X, int64_t rows, int64_t ld, int64_t s, int64_t sp,
                      double diag, double* G64);
msp_status msp_spd_inverse(msp_ctx* ctx, const double* M64, int64_t s, int64_t sp, double* Linv64,
                           double* Minv, double* shift, int* retries);
msp_status msp_gemm_tn(msp_ctx* ctx, const float* X, int64_t ldx, int64_t ncx, const float* Y, int64_t ldy,
                       int64_t ncy, int64_t K, int64_t nx_pad, int64_t ny_pad, float* C);
// (X^T X + diag I)^{-1} as a dense FP64 s_pad x s_pad matrix (see factor.cu)
msp_status msp_gram_inverse(msp_ctx* ctx, const float* X, int64_t rows, int64_t s, int64_t sp,
                            double diag, double* G64, double* Linv64, double* Minv,
                            double* shift, int* retries);

// symv.cu
int64_t msp_packed_tiles(int64_t n);
msp_status msp_pack_upper(msp_ctx* ctx, const float* A, int64_t lda, int64_t n, float* packed);
msp_status msp_pack_upper_rows(msp_ctx* ctx, const float* A, int64_t lda, int64_t n, int64_t I0, int64_t I1,
                               float* packed);
// fill the strictly lower 128-tiles of tile rows [I0, I1) from the upper ones
msp_status msp_mirror_lower_rows(msp_ctx* ctx, float* A, int64_t lda, int64_t n, int64_t I0, int64_t I1);
msp_status msp_mirror_lower_cols(msp_ctx* ctx, float* A, int64_t lda, int64_t n, int64_t J0, int64_t J1);
msp_status msp_symv_packed(msp_ctx* ctx, const float* packed, int64_t n, float lam, const float* p,
                           float* part, double* dpart, int grid);

// krylov.cu
msp_status msp_grid_wait_limit_krylov(msp_ctx* ctx, unsigned long long ns);
// prof: null, or two slots (A-pass GEMV, level-2 kernel) to accumulate
// event-timed durations into (opts->profile).
// packed: null (dense A pass over A) or the sketch's packed upper tiles.
msp_status msp_krylov_solve(msp_ctx* ctx, const msp_factor_s* f, const void* A,
                            msp_dtype dt, int64_t n, int64_t lda, double lambda,
                            const void* rhs, void* sol, double tol_rel, int max_outer,
                            const msp_opts* o, int* iters, int* inner_iters,
                            ProfSlot* prof, const float* packed);
// compensated: double-double accumulation (k_matvec64_dd), for residuals
// below the FP64 accumulation floor
msp_status msp_matvec64(msp_ctx* ctx, const void* A, msp_dtype dt, int64_t n,
                        int64_t lda, double lambda, const double* x, const double* b,
                        double* out, double* norm2_out_dev, bool compensated = false);

// Event timing helper: with `on`, records an event pair around each timed
// launch; finish() sums the elapsed times (after a stream sync). An entry is
// a (begin, end) pair of indices into the context's event pool; entries of a
// graph's event-record nodes may share an event (one event ends a launch and
// begins the next).
struct Profiler {
    msp_ctx* ctx = nullptr;
    bool on = false;
    int used = 0;                  // entries
    int next_ev = 0;               // events handed out from the pool
    bool open = false;             // begin() recorded, end() not yet
    int slot_of[4096];
    int ev_b[4096], ev_e[4096];
    msp_status begin(int slot);
    msp_status end();
    // the next event of the pool (false once it is used up)
    bool take(cudaEvent_t* ev, int* idx);
    // an entry of two events taken before
    void add(int slot, int b, int e);
    // adds the entries [harvested, upto) to the slots; their events must
    // have completed (the host may call it while later work runs)
    int harvested = 0;
    msp_status harvest(ProfSlot* slots, int nslots, int upto);
    // syncs, then sums the first `keep` entries (all when keep < 0)
    msp_status finish(ProfSlot* slots, int nslots, int keep = -1);
};
msp_status msp_profiler_reserve(msp_ctx* ctx, int pairs);
// frees the context's level-1 graph (deferred by CUDA while replays run)
void msp_l1_graph_release(msp_ctx* ctx);
// frees the context's factor graph
void msp_fac_graph_release(msp_ctx* ctx);
msp_status msp_norm2(msp_ctx* ctx, const double* v, int64_t n, double* out_dev);
msp_status msp_scale_cast(msp_ctx* ctx, const double* src, const double* nrm2, int64_t n,
                          msp_dtype dt, void* dst);
msp_status msp_axpy_back(msp_ctx* ctx, double* x, const void* d, msp_dtype dt, const double* nrm2,
                         int64_t n, int accumulate);
msp_status msp_solve_m1_impl(msp_ctx* ctx, const msp_factor_s* f, const void* r, void* w,
                             const msp_opts* o, int* inner_iters);
