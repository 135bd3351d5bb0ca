/*
 * msp.h -- C ABI of the GB300 (sm_103a) implementation of two-level
 * Multi-level Sketched Preconditioning (MSP) for the regularised PSD system
 *
 *     (A + lambda I) x = b,     A in S_n^+ dense, lambda > 0,
 *
 * from Derezinski, Musco and Yang, "Faster Linear Systems and Matrix Norm
 * Approximation via Multi-level Sketched Preconditioning" (arXiv 2405.05865),
 * Section 4 (Algorithm 1 with SolveM1 of Algorithm 2, Theorem 4.2).
 *
 * Conventions for every entry point
 *   - Matrices are dense row-major with a leading dimension in elements.
 *     A is symmetric, so row-major and column-major storage coincide.
 *   - Array arguments are DEVICE pointers unless the entry point says that it
 *     also accepts host memory. The library never frees caller memory and
 *     keeps no pointer to it after the call returns.
 *   - Work is issued on the context's stream. Entry points that return
 *     scalars (iteration counts, status) synchronise that stream before they
 *     return; the others are asynchronous with respect to the host.
 *   - Handles (msp_ctx, msp_sketch_t, msp_factor_t) own device memory
 *     allocated by the library; release them with the matching *_destroy.
 *     A factor keeps a reference to its sketch: destroy the factor first.
 *   - Errors: every entry point returns an msp_status. MSP_OK is 0. On any
 *     other value a message is available from msp_last_error(ctx). The
 *     library never aborts, traps or prints. Device-side loops carry
 *     iteration and wall-clock limits and report MSP_ETIMEOUT instead of
 *     hanging.
 *   - Determinism: the same seed gives bit-identical sketch patterns; all
 *     reductions use a fixed order, so repeated calls give identical results
 *     on the same device.
 */
#ifndef MSP_H
#define MSP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSP_API __attribute__((visibility("default")))
#else
#define MSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSP_F64 = 0,   /* IEEE binary64 */
    MSP_F32 = 1,   /* IEEE binary32 */
    MSP_BF16 = 2   /* bfloat16 (8-bit significand, binary32 range); storage
                      of preconditioner data (msp_nystrom_ex) and of A for
                      msp_sketch / msp_matvec_f64 */
} msp_dtype;

typedef enum {
    MSP_OK = 0,
    MSP_EINVAL = 1,      /* bad argument (size, pointer, dtype, option)       */
    MSP_ENOMEM = 2,      /* device allocation failed                          */
    MSP_ECUDA = 3,       /* a CUDA runtime call failed                        */
    MSP_ENOTPD = 4,      /* M2 not positive definite after all shift retries,
                            or p^T (A + lam I) p <= 0 in the outer iteration  */
    MSP_ENOCONV = 5,     /* iteration cap reached before the tolerance; the
                            best iterate is returned and msp_info is filled   */
    MSP_ENONFINITE = 6,  /* NaN/Inf in the input or in the iteration          */
    MSP_ETIMEOUT = 7     /* a device-side wait exceeded its wall-clock limit  */
} msp_status;

/* Arithmetic of the Krylov levels (the level-1 outer iteration and the
 * level-2 SolveM1 iteration).
 *   MSP_PREC_FP64  : FP64 A, FP64 sketch data and vectors. The solve runs
 *                    to tol; when its recurrence residual has drifted from
 *                    the true one, further steps correct x from the FP64
 *                    residual (at most max_refine), each asked for the
 *                    remaining factor only.
 *   MSP_PREC_FP32  : FP32 A and sketch data, FP32 vectors, FP64 dot
 *                    products; no refinement ("plain FP32").
 *   MSP_PREC_MIXED : the FP32 solve wrapped in FP64 iterative refinement:
 *                    r = b - (A + lam I) x with FP64 accumulation, solve
 *                    for the correction in FP32, x += d (FP64 x). */
typedef enum {
    MSP_PREC_FP64 = 0,
    MSP_PREC_FP32 = 1,
    MSP_PREC_MIXED = 2
} msp_precision;

typedef struct msp_ctx msp_ctx;
typedef struct msp_sketch_s msp_sketch_t;
typedef struct msp_factor_s msp_factor_t;

/* Solver options. Zero-initialise and call msp_default_opts() to get the
 * defaults listed beside each field. */
typedef struct {
    double tol;           /* stop when |b - (A+lam I)x|_2 <= tol |b|_2, the form of
                             Theorem 1.2 (implies normwise backward error <= tol).
                             Default 1e-10.                                      */
    int max_outer;        /* cap on level-1 iterations per Krylov solve. 2000.   */
    int max_refine;       /* cap on FP64 refinement steps (MIXED, FP64). 20.      */
    double refine_tol;    /* MIXED: each FP32 correction solve stops at relative
                             residual refine_tol. Default 1e-6.                  */
    double inner_tol;     /* level-2 (SolveM1) solve stops at
                             |res| <= inner_tol |C^T r|. Default 1e-6.           */
    int max_inner;        /* cap on level-2 iterations per SolveM1. 50.
                             0 selects the direct level 2: y = M2^{-1} C^T r with
                             no correction steps, exact when M2 is the level-2
                             operator itself (phi = 0, Phi = I).                 */
    int precision;        /* msp_precision. Default MSP_PREC_MIXED.              */
    int check_every;      /* level-1 iterations between host checks of the
                             device-side convergence flag. Default 8.            */
    int profile;          /* 1: time every A-pass and level-2 launch with CUDA
                             events on the context stream (msp_info *_ms);
                             launches queued after the device flagged
                             convergence (they return at once) are not
                             counted. Default 0.                                 */
    int criterion;        /* stopping rule of the solve (the last refinement
                             step in MSP_PREC_MIXED), msp_criterion. Default
                             MSP_STOP_RESIDUAL.                                  */
    int level2_iters;     /* msp_general_solve only: PCG steps of the level-2
                             solve in each SolveM1 (Algorithm 4). Default 8.     */
    int level3_iters;     /* msp_general_solve only: PCG steps of each of the
                             two level-3 solves in SolveM2 (Algorithm 5).
                             Default 8.                                          */
} msp_opts;

/* Stopping rules.
 *   MSP_STOP_RESIDUAL : |b - (A + lam I) x| <= tol |b| (relative residual).
 *   MSP_STOP_BACKWARD : |b - (A + lam I) x| <= tol ((L + lam) |x| + |b|)
 *                       with L <= |A|_2 the certified lower bound of
 *                       msp_norm_lower_bound, so the normwise backward error
 *                       |r| / (|A + lam I|_2 |x| + |b|) (Rigal-Gaches) is at
 *                       most tol. Always satisfied when the residual rule is. */
typedef enum {
    MSP_STOP_RESIDUAL = 0,
    MSP_STOP_BACKWARD = 1
} msp_criterion;

typedef struct {
    int outer_iters;      /* total level-1 iterations (all refinement steps)     */
    int inner_iters;      /* total level-2 iterations                            */
    int refine_steps;     /* FP64 refinement steps taken (MIXED)                 */
    int shift_retries;    /* Cholesky retries with a stabilising shift           */
    double rel_resid;     /* final |b - (A+lam I)x| / |b| (FP64 accumulation)    */
    double lambda_tilde;  /* lambda + lambda_0 used by the preconditioner        */
    double shift;         /* stabilising shift added to M2 (0 if none)           */
    int status;           /* msp_status of the solve                             */
    /* with opts.profile = 1: summed CUDA-event durations (ms) and launch counts */
    int gemv_launches;    /* q = (A + lam I) p passes (level 1)                  */
    int level2_launches;  /* persistent level-1 update + SolveM1 kernels         */
    int resid_launches;   /* FP64 residual passes (refinement)                   */
    int level1_graph_iters; /* level-1 iterations run as CUDA-graph replays      */
    double gemv_ms;
    double level2_ms;
    double resid_ms;
    double backward_err;  /* |r| / ((L + lam) |x| + |b|) at the end: an upper
                             bound on the normwise backward error            */
    double norm_lb;       /* L, the lower bound of |A|_2 used (0 if not formed) */
} msp_info;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t; NULL means the legacy default stream). */
MSP_API msp_status msp_create(msp_ctx** out, int device, void* stream);
MSP_API void msp_destroy(msp_ctx* ctx);
MSP_API const char* msp_last_error(const msp_ctx* ctx);
MSP_API void msp_default_opts(msp_opts* opts);
/* Library version string, e.g. "msp-gb300 0.1 sm_103a". */
MSP_API const char* msp_version(void);
/* Number of CUDA kernels this context has launched since it was created. */
MSP_API int64_t msp_launch_count(const msp_ctx* ctx);

/* ------------------------------------------------- a1: sketch index draw */

/* Definition 2.1 (sparse embedding matrix, Section 2): the pattern of an
 * `rows` x n matrix with `gamma` nonzeros +-1/sqrt(gamma) per column, the
 * gamma row indices of each column drawn uniformly without replacement and
 * the signs independently. Column j of the embedding is written as
 *   idx[j*gamma + q] (int32, ascending in q) and sgn[j*gamma + q] (+1/-1, int8).
 * For the sketch S of Algorithm 1, Pi = S^T is n x s and idx[j*gamma..] are
 * the columns of Pi's row j.
 * Draws: counter-based SplitMix64 (Steele, Lea, Flood 2014) with counter
 * (stream << 56) | (j << 8) | q, Floyd's sampling, sign from the top bit of
 * the draw on stream+1. stream 0 is S, stream 2 is Phi.
 * Requires 1 <= gamma <= min(rows, 64), n < 2^30, rows < 2^30.
 * idx, sgn: device arrays of n*gamma elements, caller-owned. */
MSP_API msp_status msp_sketch_pattern(msp_ctx* ctx, int64_t n, int64_t rows, int gamma,
                              uint64_t seed, int stream, int32_t* idx, int8_t* sgn);

/* ---------------------------------------------- a1-a2: the sketch C = A Pi */

/* Algorithm 1, steps 2-3: draw S (s x n, gamma nonzeros per column, seed
 * `seed`, stream 0) and compute C = A S^T (n x s) in one pass over A.
 * A: device, n x n, leading dimension lda >= n, dtype MSP_F32 or MSP_F64.
 * The C of the handle has the dtype of A. s is padded internally to a
 * multiple of 128 with zero columns (sizes reported by msp_sketch_info).
 * For the solves that follow, the handle also keeps what they need of A:
 * for an FP32 A its upper 128 x 128 tiles, packed (about n^2 / 2 * 4 bytes
 * of device memory; A is taken as symmetric), and the row statistics of the
 * lower bound of |A|_2 used by the backward-error rule (3n doubles). A
 * solve given the same A pointer uses them, so A must not change between
 * this call and those solves.
 * Requires 1 <= gamma <= min(s, 64), s <= n, and 16 <= s <= 2048 for an FP32
 * A (16 <= s <= 1024 for an FP64 A). */
MSP_API msp_status msp_sketch(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                      int64_t lda, int64_t s, int gamma, uint64_t seed,
                      msp_sketch_t** out);
MSP_API void msp_sketch_destroy(msp_sketch_t* sk);
/* n, s, padded s (the leading dimension of C), gamma, dtype. */
MSP_API msp_status msp_sketch_info(const msp_sketch_t* sk, int64_t* n, int64_t* s,
                           int64_t* s_pad, int* gamma, int* dtype);
/* Copy C (n x s, row-major, ldc >= s, dtype of the sketch) into a caller
 * device buffer. */
MSP_API msp_status msp_sketch_get_C(msp_ctx* ctx, const msp_sketch_t* sk, void* C, int64_t ldc);

/* ------------------------------------------- a3-a5: Nystrom core and M2 */

/* Algorithm 1, steps 3-4: W = S C (s x s, symmetrised), lambda~ = lambda +
 * lambda0, C~ = Phi C with Phi a phi x n sparse embedding (gamma_phi
 * nonzeros per column, stream 2), M2 = C~^T C~ + lambda~ W, and the FP64
 * Cholesky factor M2 + nu I = L L^T (FP64 data: nu = 0 first, on failure
 * nu = s 2^-52 |M2|_F; FP32 data: nu = 2^-24 |M2|_F from the start, the
 * rounding level of the data; then times 100 per retry, at most 4 retries,
 * else MSP_ENOTPD). The level-2 preconditioner is applied as
 * M2^{-1} v = L^{-T} (L^{-1} v) with L^{-1} stored explicitly
 * ("pre-compute M2^{-1} exactly", Section 4, Part 3).
 * phi == 0 selects Phi = I_n (C~ = C, M2 = C^T C + lambda~ W exactly: the
 * perfect embedding; the level-2 solve then converges in a few steps).
 * C~^T C~ is accumulated in the working precision; M2 only preconditions the
 * level-2 solve, whose operator C^T C + lambda~ W is always applied in the
 * working precision.
 * Requires lambda > 0, lambda0 >= 0, 0 <= phi, gamma_phi <= min(phi,255). */
MSP_API msp_status msp_nystrom(msp_ctx* ctx, const msp_sketch_t* sk, double lambda,
                       double lambda0, int64_t phi, int gamma_phi, uint64_t seed,
                       msp_factor_t** out);
/* How msp_sketch reads an FP32 A in device memory (16-byte aligned, lda a
 * multiple of 4, n >= 32; other FP32 inputs take the row-wise passes):
 * on = 1 (default): one pass over A that forms C = A Pi as A^T Pi (A is
 * symmetric by this call's contract) from 32-column blocks of A staged by
 * TMA in chunks of 512 rows, and stores the packed upper tiles from the
 * same staged blocks; on = 0: the row-wise C pass, then the packing as a
 * pass of its own. The row statistics of the norm bound are a pass of their
 * own either way. Both give C within the same rounding bound. Not part of
 * the method (it selects an implementation). */
MSP_API msp_status msp_set_sketch_one_pass(msp_ctx* ctx, int on);

/* Where msp_nystrom forms the Gram C~^T C~ of an FP32 sketch: on = 1
 * (default): on the tensor cores (tcgen05, TMA-staged): every entry of C~ is
 * split into two FP16 terms of q c (q a power of two with q max|c| <= 2^14),
 * the three largest of the four term products are accumulated in FP32 in
 * tensor memory over slices of at most 2048 rows, and the slices are added in
 * FP64 (error about 2^-22 of |C~|^T|C~| per entry); on = 0: on the FP32
 * pipe with compensated (TwoSum) sums. Not part of the method (the paper
 * has no counterpart; it selects an implementation). */
MSP_API msp_status msp_set_gram_tensor_cores(msp_ctx* ctx, int on);

/* How msp_nystrom factors M2 + nu I of an FP32 sketch (Algorithm 1, step 4:
 * the Cholesky factor and its inverse, the triangular factor the level-2
 * kernel applies as B = L^{-1} and B^T in FP32): on = 1 (default): in
 * float-float arithmetic on the FP32 pipe (pairs of floats, products by FMA,
 * sums by TwoSum, about 2^-46 relative per operation) on M2 scaled by a
 * power of four; its backward error, a small multiple of s 2^-46 |M2|, stays
 * far below the shift nu = 2^-24 |M2|_F the FP32 data needs, and the result
 * is rounded to FP32. on = 0: in FP64. FP64 sketches always use FP64. Not
 * part of the method (it selects an implementation). */
MSP_API msp_status msp_set_factor_float_float(msp_ctx* ctx, int on);

/* How msp_solve issues its level-1 iterations (Algorithm 2's outer loop:
 * the A pass, then the level-2 kernel with the step, SolveM1 and the new
 * direction): on = 1 (default): the two launches of one iteration are
 * captured once into a CUDA graph (with event-record nodes when
 * opts.profile = 1) and replayed check_every times between host reads of
 * the device convergence flag; the executable is kept by the context and
 * rebuilt when the solve's arguments or buffers change. on = 0: two stream
 * launches per iteration. The same kernels run in the same order with the
 * same arguments, so both give the same x bit for bit; where a capture is
 * not possible the solve launches on the stream (msp_info.level1_graph_iters
 * counts the replayed iterations). Not part of the method (it selects how
 * the launches are issued). */
MSP_API msp_status msp_set_level1_graphs(msp_ctx* ctx, int on);

/* msp_nystrom with the storage of the level-2 data chosen (Algorithm 1 steps
 * 3-4 and Algorithm 2 with reduced-precision preconditioner data; the paper
 * works in exact arithmetic, Section 2). data = MSP_F32 is msp_nystrom.
 * data = MSP_BF16 (FP32 sketch only): C is rounded to BF16 first, and W,
 * C~ and M2 are formed from the rounded C (FP32 and FP64 accumulation), so
 * that M = Cb W^{-1} Cb^T + lambda~ I is exactly the SPD preconditioner the
 * level-2 iteration applies; the level-2 kernel then streams Cb and Wb (BF16,
 * half the bytes of C) with FP32 accumulation, and L^{-1} stays FP32. The
 * outer level-1 iteration still applies the FP32 A, so the refined solution
 * is unchanged in accuracy; only the preconditioner (and so the iteration
 * count) differs. MSP_EINVAL for other data types. */
MSP_API msp_status msp_nystrom_ex(msp_ctx* ctx, const msp_sketch_t* sk, double lambda, double lambda0,
                                  int64_t phi, int gamma_phi, uint64_t seed, msp_dtype data,
                                  msp_factor_t** out);
MSP_API void msp_factor_destroy(msp_factor_t* f);
/* Copies of the factor's pieces into caller device buffers (FP64, row-major,
 * leading dimension s): W, M2 (before the shift), L^{-1} (lower triangle).
 * Any pointer may be NULL. lam_tilde/shift/retries may be NULL. */
MSP_API msp_status msp_factor_get(msp_ctx* ctx, const msp_factor_t* f, double* W,
                          double* M2, double* Linv, double* lam_tilde,
                          double* shift, int* retries);

/* Apply the level-1 preconditioner once: w = SolveM1(r) (Algorithm 2), i.e.
 * w ~ M^{-1} r with M = C W^{-1} C^T + lambda~ I via
 * M^{-1} = (1/lambda~)(I - C (C^T C + lambda~ W)^{-1} C^T) (Eq. M_inverse),
 * the level-2 system solved by PCG preconditioned with M2^{-1}.
 * r, w: device vectors of n elements in the sketch's dtype. inner_iters may
 * be NULL. */
MSP_API msp_status msp_solve_m1(msp_ctx* ctx, const msp_factor_t* f, const void* r,
                        void* w, const msp_opts* opts, int* inner_iters);

/* ------------------------------------------------ a6-a8: the MSP solve */

/* Algorithm 1 step 5: solve (A + lambda I) x = b by the level-1 iteration
 * (flexible PCG, equal to Algorithm 6 in exact arithmetic, Section 6) with
 * SolveM1 as the preconditioner; in MSP_PREC_MIXED the solve is wrapped in
 * FP64 iterative refinement.
 * A: device, n x n, lda >= n; FP64 with MSP_PREC_FP64, FP32 otherwise; it
 *    must be the matrix the factor was built from.
 * b, x: device FP64 vectors of n elements (x is overwritten; no initial
 *    guess). info may be NULL.
 * Returns MSP_ENOCONV (with x the last iterate) if the caps are reached. */
MSP_API msp_status msp_solve(msp_ctx* ctx, const msp_factor_t* f, const void* A,
                     msp_dtype dtype, int64_t n, int64_t lda, double lambda,
                     const double* b, double* x, const msp_opts* opts,
                     msp_info* info);
/* Wall-clock limit of the grid-wide barriers of the level-1 / level-2
 * kernels (msp_solve, msp_solve_refined, msp_solve_many, msp_solve_m1) on
 * the context's device, in seconds; 0 restores the default of 2 s. A block
 * that waits longer gives up and the call returns MSP_ETIMEOUT (the context
 * stays usable: every solve resets its control block). Meant for tests of
 * that error path and for callers that want a solve that cannot stall for
 * long; a limit below a barrier's normal duration (a few microseconds) makes
 * every solve fail. Not part of the method (the paper has no counterpart).
 * MSP_EINVAL outside [0, 60]. */
MSP_API msp_status msp_set_grid_wait_limit(msp_ctx* ctx, double seconds);

/* msp_solve with a separate matrix for the FP64 refinement residual. The
 * paper works in exact arithmetic (Section 2); here the problem is a matrix
 * given in FP64 whose FP32 rounding the level-1 iteration applies. A (FP32,
 * the matrix the factor was built from) drives the level-1 iteration;
 * A_res (device, n x n, ld_res >= n, MSP_F64 or MSP_F32) is the problem
 * itself: every refinement step forms r = b - (A_res + lambda I) x with FP64
 * accumulation, and the backward-error rule takes its norm bound from A_res.
 * Refinement converges while rho = |(A + lambda I)^{-1} (A - A_res)| < 1,
 * the FP32 rounding of A_res being small next to lambda + lambda_min.
 * A_res == A is msp_solve. Other arguments and errors as msp_solve. */
MSP_API msp_status msp_solve_refined(msp_ctx* ctx, const msp_factor_t* f, const void* A,
                                     msp_dtype dtype, int64_t n, int64_t lda, const void* A_res,
                                     msp_dtype res_dtype, int64_t ld_res, double lambda,
                                     const double* b, double* x, const msp_opts* opts,
                                     msp_info* info);
/* Several right-hand sides with one factor: column j of B (device FP64,
 * column-major n x m, ldb >= n) is solved exactly as msp_solve would into
 * column j of X (ldx >= n), one after another; infos (host, may be NULL)
 * receives m msp_info. Returns MSP_ENOCONV if any column hit its caps (all
 * columns are still solved), another error at the first failing column. */
MSP_API msp_status msp_solve_many(msp_ctx* ctx, const msp_factor_t* f, const void* A, msp_dtype dtype,
                                  int64_t n, int64_t lda, double lambda, const double* B, int64_t ldb,
                                  double* X, int64_t ldx, int64_t m, const msp_opts* opts,
                                  msp_info* infos);

/* The whole of Algorithm 1 in one call: sketch, Nystrom factor, solve.
 * A, b and x may each be device or host memory (host buffers are staged
 * through device buffers owned by the context; pinned host memory is
 * fastest). A host A is copied in row chunks on a copy stream of the
 * context, overlapped with the sketch and the packing; of a host FP32 A only
 * the upper triangle (with the diagonal) is read -- A is symmetric, as the
 * packed A pass already assumes -- and the lower triangle is mirrored on the
 * device. Parameters as for msp_sketch / msp_nystrom / msp_solve. */
MSP_API msp_status msp_solve_full(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                          int64_t lda, double lambda, const double* b, double* x,
                          int64_t s, int gamma, double lambda0, int64_t phi,
                          int gamma_phi, uint64_t seed, const msp_opts* opts,
                          msp_info* info);

/* ------------------------------------------------------ a9: batching */

/* One instance of a batch: (A + lambda I) X = B with m right-hand sides,
 * each column an independent solve of Algorithm 1 (Section 4) sharing the
 * instance's sketch and Nystrom factor. Columns are not coupled (no block
 * Krylov method): each has its own level-1 scalars, so a column's result
 * equals that of a single-RHS solve up to rounding. */
typedef struct {
    const float* A;      /* device FP32 n x n row-major, lda >= n, symmetric   */
    int64_t n;           /* 16 <= n <= 65536                                   */
    int64_t lda;
    double lambda;       /* > 0                                                */
    double lambda0;      /* >= 0 (lambda~ = lambda + lambda0)                  */
    const double* B;     /* device FP64 n x m column-major, ldb >= n           */
    int64_t ldb;
    double* X;           /* device FP64 n x m column-major, ldx >= n (output)  */
    int64_t ldx;
    int m;               /* 1 <= m <= 16                                       */
    int gamma;           /* nonzeros per column of S (msp_sketch)              */
    int64_t s;           /* sketch size, 16 <= s <= min(n, 1024)               */
    int64_t phi;         /* level-2 embedding rows; 0 = Phi = I (msp_nystrom)  */
    int gamma_phi;
    int pad_;
    uint64_t seed;
} msp_instance;

typedef struct msp_batch_s msp_batch_t;

/* Set up a batch (Algorithm 1 steps 1-4 for every instance): sketch, W, M2
 * and its factor per instance, built concurrently on worker streams owned by
 * the context, and a copy of each A re-laid out as the tiles the batched A
 * pass streams. The preconditioner is applied directly at level 2
 * (y = M2^{-1} C^T r, as with opts.max_inner = 0). The A, B and X buffers
 * named by `inst` must stay valid and unchanged in size for the life of the
 * batch; B and X are read and written by msp_batch_solve, and A's contents
 * are copied here (later changes to A are not seen). Requires count >= 1 and
 * every instance valid; the whole batch fails on the first bad instance.
 * Instances that name the same A pointer, n, lda, lambda, lambda0, s,
 * gamma, phi, gamma_phi and seed are one system with more right-hand sides:
 * they share one sketch, factor and tiled copy of A (set up once), so a
 * system with more than 16 right-hand sides is solved as several such
 * instances in one launch. Destroy every batch before its context. */
MSP_API msp_status msp_batch_create(msp_ctx* ctx, int count, const msp_instance* inst,
                                    msp_batch_t** out);
MSP_API void msp_batch_destroy(msp_batch_t* batch);

/* Solve every column of every instance (Algorithm 1 step 5 with FP64
 * refinement in MSP_PREC_MIXED) in ONE persistent cooperative kernel launch
 * on the context's stream: the level-1 iteration, the direct level 2, the
 * FP64-accurate residual and every convergence decision run on the device,
 * with no host synchronisation. X is overwritten (no initial guess).
 * opts: tol, criterion (per column), max_outer (per correction solve),
 * max_refine, refine_tol, precision (MSP_PREC_MIXED or MSP_PREC_FP32); other
 * fields are ignored. The residual of the refinement is float-float: x is
 * split into an FP32 pair (48 bits), products are exact (FMA) and sums are
 * kept as FP32 pairs (TwoSum), so it carries an error of a few
 * 2^-48 |(|A| |x|)|; with MSP_STOP_RESIDUAL and a tol below that level
 * relative to |b| a column ends with MSP_ENOCONV. MSP_STOP_BACKWARD, whose
 * threshold scales with |A| |x|, is not limited by it.
 * infos: NULL makes the call asynchronous (and capturable in a CUDA graph on
 * the context's stream); otherwise `count` entries are filled after a
 * stream synchronisation, as msp_batch_info does. The returned status is the
 * first non-OK instance status (MSP_ENOCONV when only caps were hit). */
MSP_API msp_status msp_batch_solve(msp_ctx* ctx, msp_batch_t* batch, const msp_opts* opts,
                                   msp_info* infos);

/* Per-instance results of the last msp_batch_solve (synchronises the
 * context's stream): outer_iters = level-1 iterations in which the instance
 * had an unconverged column, refine_steps, rel_resid = the largest
 * |b_j - (A + lambda I) x_j| / |b_j| over its columns, backward_err = the
 * largest |r_j| / ((L + lambda) |x_j| + |b_j|), norm_lb = L, lambda_tilde,
 * shift, shift_retries, status. gemv_launches / resid_launches count the
 * batch's A passes and residual passes and gemv_ms / level2_ms / resid_ms
 * split the launch's device time (the same in every entry). */
MSP_API msp_status msp_batch_info(msp_ctx* ctx, const msp_batch_t* batch, msp_info* infos);

/* Counters of the last msp_batch_solve (synchronises the context's stream),
 * written to stats[0..15]: [0] level-1 A passes, [1] residual passes,
 * [2] bytes of A streamed by the level-1 passes, [3] by the residual passes
 * (instances whose columns had all converged are skipped), [4..10] device-
 * timer milliseconds of the A passes, G = C^T R, the two triangular
 * applications of L^{-1}, Z = (R - C Y) / lambda~, the vector updates (P,
 * X, R), the residual passes with the X update, and the convergence checks,
 * [11] bytes of one full pass over every tiled A (sum of n_pad^2 * 4),
 * [12] sum of n^2 * 4, [13] bytes of C read by G, [14] by Z, [15] the unit
 * width in tiles. The times are read by one block between grid barriers, so
 * each class includes its barrier. */
MSP_API msp_status msp_batch_stats(msp_ctx* ctx, const msp_batch_t* batch, double* stats);

/* Width of the work units of the batched A passes, the tile shape choice of
 * the batched kernel: a unit is one 128-row block of an A times at most
 * `*unit_tiles` x 64 columns. *unit_tiles > 0 (a power of two >= 16) sets
 * it; *unit_tiles == 0 times the A passes of 12 level-1 iterations at every
 * width from 16 tiles to a whole row and keeps the fastest, returned in
 * *unit_tiles. The timing runs overwrite the X buffers of the batch. A new
 * batch starts with the widest unit that still gives 8 units per SM. */
MSP_API msp_status msp_batch_autotune(msp_ctx* ctx, msp_batch_t* batch, int* unit_tiles);

/* msp_batch_create + msp_batch_solve + msp_batch_destroy. */
MSP_API msp_status msp_solve_batched(msp_ctx* ctx, int count, const msp_instance* inst,
                                     const msp_opts* opts, msp_info* infos);

/* ------------------------------------------------ a10: Schatten-1 norm */

/* Schatten-p norm |A|_p = (sum_i sigma_i^p)^{1/p} of a PSD matrix A
 * (Section 3.2, the norm estimators built on stochastic trace estimation).
 * Only p = 1 is implemented: for PSD A, |A|_1 = tr(A), estimated by
 * Hutchinson's estimator (1/m) sum_j g_j^T A g_j with m = `probes` Rademacher
 * probes (row i of probe j negative iff the top bit of
 * draw(seed, 7 + 2 (j / 256), i, j mod 256) is set). A: device FP32,
 * row-major n x n, lda >= n, symmetric; each of its tiles on one side of
 * the diagonal is read once per group of up to 256 probes (rows 16-byte
 * aligned, i.e. lda % 4 == 0 and A 16-byte aligned: on the tensor cores,
 * by TMA; otherwise packed first and on the FP32 pipe).
 * probes: a multiple of 64 in [64, 4096]. Outputs (host scalars, any may be
 * NULL): norm = the estimate of |A|_1, norm_pow = |A|_1^p (the same for
 * p = 1), std_err = sample standard deviation of the q_j / sqrt(m).
 * Other p return MSP_EINVAL (they need shifted MSP solves). */
MSP_API msp_status msp_schatten(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                                int64_t lda, double p, int64_t probes, uint64_t seed,
                                double* norm, double* norm_pow, double* std_err);

/* The per-probe quadratic forms q_j = g_j^T A g_j of msp_schatten (device
 * FP64 array of `probes`). Tensor-core path: every entry of A split into
 * 16-bit terms (msp_set_hutchinson_terms), products with the +-1 probes
 * accumulated in FP32 over a row block of 128 rows, then FP32 sums over 32
 * rows and FP64 beyond. Other path: 128-term FP32 tile products combined
 * in FP64. Returns after synchronising the stream (a device-side wait that
 * gave up is reported as MSP_ETIMEOUT). */
MSP_API msp_status msp_hutchinson(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                                  int64_t lda, int64_t probes, uint64_t seed, double* q);

/* 16-bit terms per FP32 entry of A in the tensor-core Hutchinson product of
 * this context: 2 (default) = two FP16 terms of s a, s a power of two with
 * s max_k a_kk <= 2^14, so that every |2 s a_ij| stays inside the FP16 range
 * when A is PSD; hi + lo carry 22 significant bits (error <= 2^-22 |a|, or
 * 2^-25 / s absolute for the smallest entries). A matrix with an entry
 * beyond that range (not PSD) is detected and recomputed with 3 terms.
 * 3 = three BF16 terms, which hold the whole FP32 significand (exact), at
 * half again the tensor-core work and shared-memory traffic. MSP_EINVAL for
 * other values. */
MSP_API msp_status msp_set_hutchinson_terms(msp_ctx* ctx, int terms);

/* ------------------------------------------ effective dimension d_lambda */

/* d_lambda = tr(A (A + lambda I)^{-1}) = sum_i sigma_i / (sigma_i + lambda)
 * (Section 2, the quantity of Lemma 2.1 that sets the sketch size in the
 * kernel ridge regression analysis), estimated as
 * n - lambda (1/m) sum_j g_j^T (A + lambda I)^{-1} g_j over m = `probes`
 * Rademacher probes (the probes of msp_schatten with `seed`), the solves run
 * as one batch (msp_batch_create with every instance naming A, so the
 * sketch of size s and gamma, seed `seed`, the factor and the tiled copy of
 * A are built once; Phi = I; opts as for msp_batch_solve).
 * A: device FP32 n x n, lda >= n, symmetric PSD; 2 <= probes <= 4096.
 * estimate, std_err: host scalars (the mean and the standard error of the
 * per-probe values n - lambda g_j^T x_j), either may be NULL; q: NULL or a
 * device FP64 array of `probes` receiving those values. Returns the solve's
 * status (MSP_ENOCONV when a solve hit its caps; the estimate is still
 * written). */
MSP_API msp_status msp_effective_dimension(msp_ctx* ctx, const float* A, int64_t n, int64_t lda,
                                           double lambda, int64_t probes, uint64_t seed, int64_t s,
                                           int gamma, const msp_opts* opts, double* estimate,
                                           double* std_err, double* q);

/* Sketch size and shift chosen from d_lambda (Section 3: l = 2 d_lambda in
 * the kernel ridge regression corollary; Lemma 2.1):
 *   l = ceil(2 d), so lambda_l <= lambda (Lemma 2.1(1), gamma = 1);
 *   s = l rounded up to 16, capped at min(n, 1024) rounded down to 16
 *       (`capped` = 1 when s < l);
 *   lambda0 = 2 lambda d / s when s >= d: Lemma 2.1(2) bounds
 *       sum_{i > s} lambda_i by lambda d, so this is an upper bound of the
 *       paper's (2/s) sum_{i > s} lambda_i and lambda0 <= lambda;
 *       lambda0 = 0 when s < d (the lemma gives nothing there);
 *   direct = 1 when d >= n/4 (the paper then inverts A + lambda I directly).
 * d_std_err is the estimate's standard error (0 from msp_params_from_effdim). */
typedef struct {
    double d_lambda;
    double d_std_err;
    int64_t l;
    int64_t s;
    double lambda0;
    int capped;
    int direct;
} msp_param_choice;

/* The rule above for a given d (host only, no GPU work). MSP_EINVAL unless
 * d >= 0 finite, n >= 16, lambda > 0, out != NULL. */
MSP_API msp_status msp_params_from_effdim(double d, int64_t n, double lambda, msp_param_choice* out);

/* Estimate d_lambda (msp_effective_dimension with the largest sketch,
 * s = min(n, 1024) rounded down to 16, lambda0 = 0) and apply the rule to the
 * estimate clamped to [0, n]. Arguments as for msp_effective_dimension;
 * errors: those of msp_effective_dimension (a solve that hit its caps is an
 * error here: MSP_ENOCONV). */
MSP_API msp_status msp_auto_params(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, double lambda,
                                   int64_t probes, uint64_t seed, int gamma, const msp_opts* opts,
                                   msp_param_choice* out);

/* -------------------------- three-level MSP for (A^T A + lambda I) x = c */

/* Section 5 (the main technical result, Theorem 3.1): A is m x n, m >= n,
 * full column rank, FP32 row-major on the device (lda >= n; rows whose start
 * is not 16-byte aligned, or odd n, are copied once into a padded layout).
 * msp_general_create runs Algorithm 3 steps 2-6: lambda~ = lambda + lambda0,
 * S (s x n, gamma nonzeros per column, the streams of msp_sketch with `seed`),
 * A~ = A S^T (m x s), A^ = Phi A~ with Phi a phi x m sparse embedding
 * (gamma_phi nonzeros per column, the level-2 streams), M3a = A^^T A^ and
 * M3b = M3a + lambda~ I factored in FP64 (unshifted; on failure the FP64-data
 * shift rule of msp_nystrom)
 * and kept as dense FP64 inverses. A is read again by every solve and must
 * stay valid and unchanged for the life of the handle (unless it was copied).
 * Requires 16 <= n <= 8192, n <= m < 2^30, lambda >= 0, lambda0 >= 0 with
 * lambda + lambda0 > 0 (SolveM1 divides by lambda~), 16 <= s <= min(n, 1024),
 * s <= phi <= m. Errors: MSP_EINVAL, MSP_ENOMEM, MSP_ENOTPD (a level-3 Gram
 * not positive definite after the shift retries), MSP_ECUDA. */
typedef struct msp_general_s msp_general_t;
MSP_API msp_status msp_general_create(msp_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda,
                                      double lambda, double lambda0, int64_t s, int gamma, int64_t phi,
                                      int gamma_phi, uint64_t seed, msp_general_t** out);
MSP_API void msp_general_destroy(msp_general_t* g);
/* s_pad (the padded sketch width), lambda~, and the stabilising shifts added
 * to M3a and M3b (host scalars, each may be NULL). */
MSP_API msp_status msp_general_info(const msp_general_t* g, int64_t* s_pad, double* lambda_tilde,
                                    double* shift_a, double* shift_b);
/* Copies of the set-up for tests (device buffers, each may be NULL): A~ as
 * FP32 m x s row-major with leading dimension ld_at; M3a and M3b as FP64
 * s x s row-major (before the shift). */
MSP_API msp_status msp_general_get(msp_ctx* ctx, const msp_general_t* g, float* At, int64_t ld_at,
                                   double* M3a, double* M3b);
/* Solve (A^T A + lambda I) x = c by Algorithm 3 step 7: flexible PCG at
 * level 1 with SolveM1 (Algorithm 4: opts.level2_iters flexible PCG steps on
 * (A~^T A A^T A~ + lambda~ A~^T A~) y = A~^T A r, preconditioned by SolveM2,
 * then w = (r - A^T A~ y) / lambda~), SolveM2 (Algorithm 5: opts.level3_iters
 * PCG steps on A~^T A~ u = r and on (A~^T A~ + lambda~ I) v = r,
 * preconditioned by M3a^{-1} and M3b^{-1}, then z = (u - v) / lambda~; the
 * level-3 operator W = A~^T A~ is formed once in FP64, s x s).
 * Levels run in FP32 with FP64 dot products; MSP_PREC_MIXED wraps the solve
 * in FP64 refinement (r = c - (A^T A + lambda I) x accumulated in FP64, each
 * correction solved to opts.refine_tol). Stops at
 * |c - (A^T A + lambda I) x| <= opts.tol |c| (MSP_STOP_RESIDUAL only).
 * c, x: device FP64 vectors of length n. info (host, may be NULL): level-1
 * iterations, level-2 iterations, refinement steps, final relative residual
 * in FP64, lambda~. Errors: MSP_EINVAL (bad options), MSP_ENOCONV (x and info
 * hold the last iterate), MSP_ENOTPD / MSP_ENONFINITE (a breakdown), MSP_ECUDA. */
MSP_API msp_status msp_general_solve(msp_ctx* ctx, msp_general_t* g, const double* c, double* x,
                                     const msp_opts* opts, msp_info* info);
/* One application of SolveM1 (w ~ M^{-1} r, M = C W^{-1} C^T + lambda~ I,
 * C = A^T A~, W = A~^T A~) with t2 level-2 and t3 level-3 steps, and one of
 * SolveM2 (z ~ (W^2 + lambda~ W)^{-1} r) with t3 level-3 steps: device FP32
 * vectors (r, w of length n; r, z of length s); for tests. */
MSP_API msp_status msp_general_solve_m1(msp_ctx* ctx, msp_general_t* g, const float* r, float* w, int t2,
                                        int t3);
MSP_API msp_status msp_general_solve_m2(msp_ctx* ctx, msp_general_t* g, const float* r, float* z, int t3);
/* q = (A^T A + lambda I) p in FP32, the level-1 operator: one fused pass
 * over the rows of A (t = A p and A^T t together) and a column sum (device
 * FP32, length n). */
MSP_API msp_status msp_general_op(msp_ctx* ctx, msp_general_t* g, const float* p, float* q);
/* Change lambda and lambda0 of a general handle (lambda~ = lambda + lambda0
 * > 0): M3b is refactored and the exact-level inverses are rebuilt when next
 * used; A~, M3a and C = A^T A~ are kept. Errors: MSP_EINVAL, MSP_ENOTPD. */
MSP_API msp_status msp_general_set_lambda(msp_ctx* ctx, msp_general_t* g, double lambda, double lambda0);
/* y = (A^T A + lambda I) x with FP64 accumulation (device FP64, length n). */
MSP_API msp_status msp_general_matvec64(msp_ctx* ctx, msp_general_t* g, const double* x, double* y);

/* ------------------------------------------ Schatten-p for p in (0, 2) */

/* |A + zI|_p^p (z = 0: |A|_p^p) for a general A (m x n, m >= n, FP32
 * row-major on the device) from ridge solves (Section 3.2: eq.
 * schatten-ridge and the random shift A + zI, z a caller-drawn scalar,
 * square A only). With q = p/2, |A|_p^p = (sin(pi q)/pi) int_0^inf t^(q-1)
 * d_t dt (Balakrishnan's integral for fractional powers), d_t = n - t
 * tr((A^T A + t I)^{-1}); the trapezoidal rule in ln t on `nodes` points over
 * [t_min, t_max] with geometric tails from d_t ~ n (t -> 0) and
 * d_t ~ |A|_F^2 / t (t -> inf). Each d_t is a Hutchinson mean over `probes`
 * Rademacher probes (those of msp_schatten with `seed`), each term one
 * msp_general_solve (opts; s the sketch size, phi = min(4s, m)) with
 * lambda = t and lambda~ = max(t, lambda_floor_rel * |A|_2^2), |A|_2^2
 * estimated by 30 power iterations (1e-3 keeps the FP32 levels stable).
 * Cost: nodes x probes solves. estimate, std_err (host, may be NULL): the
 * mean and standard error over probes; X (host, may be NULL, `probes`
 * doubles): the per-probe estimates. */
MSP_API msp_status msp_schatten_p(msp_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, double p,
                                  double z, double t_min, double t_max, int nodes, int64_t probes, uint64_t seed,
                                  int64_t s, double lambda_floor_rel, const msp_opts* opts, double* estimate,
                                  double* std_err, double* X);

/* --------------------------------------------------------- least squares */

/* min_x |A x - b| for a tall A (n_rows x d, FP32 row-major on the device,
 * lda >= d) by sketch-and-precondition (Section 3, the least-squares
 * corollary): msp_lsq_create forms A~ = Phi A (s_ls x d, Phi an s_ls x
 * n_rows sparse embedding with gamma_ls nonzeros per column, streams 4 and 5
 * of `seed`) and a three-level handle on A~ (msp_general_create with
 * lambda = 0, lambda0 > 0, s, gamma, phi, gamma_phi, seed). A must stay
 * valid and unchanged for the life of the handle (unless it was copied).
 * Requires 16 <= d <= 8192, d <= s_ls <= n_rows < 2^30, lambda0 > 0, and the
 * msp_general_create conditions on (A~, s, phi). */
typedef struct msp_general_s msp_lsq_t;
MSP_API msp_status msp_lsq_create(msp_ctx* ctx, const float* A, int64_t n_rows, int64_t d, int64_t lda,
                                  int64_t s_ls, int gamma_ls, double lambda0, int64_t s, int gamma, int64_t phi,
                                  int gamma_phi, uint64_t seed, msp_lsq_t** out);
MSP_API void msp_lsq_destroy(msp_lsq_t* h);
/* Flexible PCG on A^T A x = A^T b (FP32, wrapped in FP64 refinement with
 * MSP_PREC_MIXED) preconditioned by (A~^T A~)^{-1}, each application an
 * inner solve on A~ (msp_general_solve's level-1 iteration) stopped at
 * relative residual opts.inner_tol or opts.max_inner iterations (constant
 * accuracy is enough, 1e-2 typical); opts.level2_iters / level3_iters select
 * the inner solve's levels as in msp_general_solve. Stops at
 * |A^T (b - A x)| <= opts.tol |A^T b|. b: device FP64 (n_rows), x: device
 * FP64 (d). info (host, may be NULL): level-1 iterations, inner iterations,
 * refinement steps, the final relative normal-equation residual (FP64);
 * resid_norm (host, may be NULL): |A x - b| in FP64. Errors as
 * msp_general_solve. */
MSP_API msp_status msp_lsq_solve(msp_ctx* ctx, msp_lsq_t* h, const double* b, double* x, const msp_opts* opts,
                                 msp_info* info, double* resid_norm);

/* ------------------------------------------------- a11: RBF and adjoint */

/* The Gaussian (RBF) kernel matrix of kernel ridge regression (Section 3,
 * the system (K + lambda I) x = y): K_ij = exp(-|p_i - p_j|^2 / (2 ell^2))
 * for n points in R^dim (1 <= dim <= 4), points: device FP64 row-major n x dim.
 * Computed in FP32 from the points rounded to FP32; K: device FP32 row-major,
 * ldk >= n (K_ii = 1 exactly). */
MSP_API msp_status msp_rbf_kernel(msp_ctx* ctx, const double* points, int64_t n, int dim,
                                  double ell, float* K, int64_t ldk);

/* Adjoint of the RBF length scale for x = (K + lambda I)^{-1} b: with the
 * adjoint solution a = (K + lambda I)^{-1} g of a loss L with dL/dx = g,
 * dL/d ell = -a^T (dK/d ell) x, dK_ij/d ell = K_ij d_ij^2 / ell^3. Each
 * pair's term is recomputed from the points (dK is never formed); FP32
 * pair terms with compensated sums, FP64 row totals. a, x: device FP64
 * vectors of n; out: device FP64 scalar (written when the work completes). */
MSP_API msp_status msp_rbf_grad_ell(msp_ctx* ctx, const double* points, int64_t n, int dim,
                                    double ell, const double* a, const double* x, double* out);

/* out = scale * x^T y for device FP64 vectors of n (FP64, fixed-order block
 * reduction), written to the device scalar out when the work completes. The
 * adjoint's dL/dlambda = -a^T x is msp_dot(a, x, scale = -1). */
MSP_API msp_status msp_dot(msp_ctx* ctx, const double* x, const double* y, int64_t n, double scale,
                           double* out);

/* No-allocation variant of msp_rbf_grad_ell (the paper has no counterpart:
 * this is an interface for callers, not a step of the method). Some callers
 * cannot allocate device memory at the point where they need the gradient:
 * a framework whose allocator owns the whole device, a time-critical loop
 * that forbids allocation after start-up, or code that must not disturb the
 * memory state of a pool it does not own. This entry point takes no context
 * and allocates nothing: the block partials and the reduction counter live in
 * a fixed array inside the library, and the result is identical to
 * msp_rbf_grad_ell's (same kernel, same fixed-order reduction).
 *   - points, a, x, out: device memory owned by the caller, as for
 *     msp_rbf_grad_ell; stream: the cudaStream_t to run on (NULL = legacy
 *     default stream); the current device is used.
 *   - n <= 524288 (one scratch slot per 8 points); larger n returns
 *     MSP_EINVAL with a message from msp_last_error(NULL).
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture
 *     on that device. The address is kept for the life of the process: after
 *     cudaDeviceReset on a device it is stale, so do not call this entry
 *     point on a device that has been reset.
 *   - A non-NULL stream must belong to the current device (MSP_EINVAL
 *     otherwise).
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents; each call clears the counter it needs on its stream.
 *     Calls whose work overlaps on the GPU (different streams, or several
 *     host threads) race on the array: serialise them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine. */
MSP_API msp_status msp_rbf_grad_ell_static(const double* points, int64_t n, int dim, double ell,
                                           const double* a, const double* x, double* out,
                                           void* stream);

/* ----------------------------------------------------- helpers (tests) */

/* L <= |A|_2 for symmetric PSD A from max(max_i |A e_i|_2, 1^T A 1 / n) (a
 * column norm and the Rayleigh quotient of the all-ones vector), one pass
 * over A (device, FP32 or FP64, lda >= n). Entries are summed in FP32 chunks
 * of 16 combined in FP64, and each term is lowered by the rounding bound of
 * those chunks, so the result is a certified lower bound, within about 1e-6
 * (relative to the sums of |a_ij|) of the exact expression. *out: host
 * scalar. */
MSP_API msp_status msp_norm_lower_bound(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                                        int64_t lda, double* out);

/* y = (A + lambda I) x, FP64 accumulation, FP64 x and y; A FP32 or FP64.
 * The residual operator of the refinement step (one pass over A). */
MSP_API msp_status msp_matvec_f64(msp_ctx* ctx, const void* A, msp_dtype dtype, int64_t n,
                          int64_t lda, double lambda, const double* x, double* y);

#ifdef __cplusplus
}
#endif
#endif /* MSP_H */
