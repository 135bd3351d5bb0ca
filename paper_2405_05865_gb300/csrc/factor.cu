// Level-2 preconditioner of Algorithm 1, step 4, on sm_103a:
//   M2 = C~^T C~ + lambda~ W   (s x s, assembled in FP64),
//   M2 + nu I = L L^T          (FP64 Cholesky; nu = 0, then the stabilising
//                               shift retries described in msp.h),
//   L^{-1}                     (FP64), stored in the working precision as
//                               B = L^{-1} and B^T so that the level-2
//                               iteration applies M2^{-1} v = B^T (B v).
// The factorisation recursion halves the matrix:
//   [A11 . ; A21 A22]:  (L11, X11) = f(A11);  L21 = A21 X11^T;
//   A22 -= L21 L21^T;   (L22, X22) = f(A22);  X21 = -X22 (L21 X11),
// with a one-block dense Cholesky + triangular inverse at the 64 x 64 leaves
// and an FP64 GEMM kernel for the rest.
#include "msp_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// ----------------------------------------------------------- Gram (SIMT)

// M2[a][b] = sum_k Ct[k][a] Ct[k][b] + lam_t * W[a][b], FP64 output; pad rows
// (a >= s or b >= s) get the identity. 64 x 64 output tile, 256 threads each
// 4 x 4, K chunks of 16. Accumulates in TA (FP32 for FP32 data).
template <typename TA>
__global__ void __launch_bounds__(256) k_gram(const TA* __restrict__ Ct, int64_t K,
                                             int64_t ld, const TA* __restrict__ W,
                                             double lam_t, int64_t s, int64_t s_pad,
                                             double* __restrict__ M2) {
    __shared__ TA As[16][64 + 4];
    __shared__ TA Bs[16][64 + 4];
    const int a0 = blockIdx.y * 64, b0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    TA acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TA(0);
    for (int64_t k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e >> 6, cc = e & 63;
            bool in = (k0 + kk) < K;
            As[kk][cc] = in ? Ct[(k0 + kk) * ld + a0 + cc] : TA(0);
            Bs[kk][cc] = in ? Ct[(k0 + kk) * ld + b0 + cc] : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            TA av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
            double v;
            if (a < s && b < s) v = (double)acc[i][j] + lam_t * (double)W[a * s_pad + b];
            else v = (a == b) ? 1.0 : 0.0;
            M2[a * s_pad + b] = v;
        }
}

// W <- (W + W^T)/2 in place (working precision) and W64 = (double)W.
template <typename T>
__global__ void k_symmetrize(T* __restrict__ W, double* __restrict__ W64, int64_t s_pad) {
    int64_t a = blockIdx.y * 32 + threadIdx.y, b = blockIdx.x * 32 + threadIdx.x;
    if (a >= s_pad || b >= s_pad || b > a) return;
    T v = (W[a * s_pad + b] + W[b * s_pad + a]) * T(0.5);
    W[a * s_pad + b] = v;
    W[b * s_pad + a] = v;
    W64[a * s_pad + b] = (double)v;
    W64[b * s_pad + a] = (double)v;
}

// ----------------------------------------------------------- FP64 GEMM

// Cm = alpha * op(A) op(B) + beta * Cm, row-major; op(A) is m x k, op(B) k x n.
// 32 x 32 tile, 256 threads each 2 x 2, K chunks of 16.
template <bool TA_, bool TB_>
__global__ void __launch_bounds__(256) k_dgemm(int64_t m, int64_t n, int64_t k, double alpha,
                                              const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb,
                                              double beta, double* __restrict__ Cm, int64_t ldc) {
    __shared__ double As[16][32 + 1];   // As[kk][i] = op(A)[i][k0+kk]
    __shared__ double Bs[16][32 + 1];   // Bs[kk][j] = op(B)[k0+kk][j]
    const int64_t i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t k0 = 0; k0 < k; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            int kk, ii;
            if (TA_) { ii = e & 31; kk = e >> 5; }   // A^T: read A[k][i], contiguous in i
            else { kk = e & 15; ii = e >> 4; }        // A: read A[i][k], contiguous in k
            int64_t gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < m && gk < k) v = TA_ ? A[gk * lda + gi] : A[gi * lda + gk];
            As[kk][ii] = v;
        }
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            int kk, jj;
            if (TB_) { kk = e & 15; jj = e >> 4; }    // B^T: read B[j][k], contiguous in k
            else { jj = e & 31; kk = e >> 5; }        // B: read B[k][j], contiguous in j
            int64_t gj = j0 + jj, gk = k0 + kk;
            double v = 0.0;
            if (gj < n && gk < k) v = TB_ ? B[gj * ldb + gk] : B[gk * ldb + gj];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
            double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int64_t gi = i0 + ty * 2 + i, gj = j0 + tx * 2 + j;
            if (gi < m && gj < n) {
                double c = beta == 0.0 ? 0.0 : beta * Cm[gi * ldc + gj];
                Cm[gi * ldc + gj] = c + alpha * acc[i][j];
            }
        }
}

// Leaf: dense Cholesky of the nb x nb block at M (ld) in place (lower), and
// its inverse into X (ld), one block of 256 threads, nb <= 64. On a
// non-positive or non-finite pivot sets *fail = 1.
constexpr int kLeafSmem = 2 * 64 * 65 * (int)sizeof(double);

__global__ void __launch_bounds__(256) k_chol_leaf(double* __restrict__ M, double* __restrict__ X,
                                                  int64_t ld, int nb, int* __restrict__ fail) {
    extern __shared__ __align__(16) double leaf_smem[];
    double (*a)[65] = reinterpret_cast<double (*)[65]>(leaf_smem);
    double (*x)[65] = reinterpret_cast<double (*)[65]>(leaf_smem + 64 * 65);
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        a[i][j] = (j <= i) ? M[i * ld + j] : 0.0;
    }
    __syncthreads();
    for (int kcol = 0; kcol < nb; ++kcol) {
        // pivot
        if (threadIdx.x == 0) {
            double d = a[kcol][kcol];
            if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
            a[kcol][kcol] = sqrt(d);
        }
        __syncthreads();
        double piv = a[kcol][kcol];
        for (int i = kcol + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][kcol] /= piv;
        __syncthreads();
        // trailing update of the lower triangle
        int rem = nb - kcol - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int i = kcol + 1 + e / rem, j = kcol + 1 + e % rem;
            if (j <= i) a[i][j] -= a[i][kcol] * a[j][kcol];
        }
        __syncthreads();
    }
    // X = L^{-1}: column j by forward substitution (thread per column)
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        for (int i = 0; i < nb; ++i) {
            double v = (i == j) ? 1.0 : 0.0;
            for (int kk = j; kk < i; ++kk) v -= a[i][kk] * x[kk][j];
            x[i][j] = (i < j) ? 0.0 : v / a[i][i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        if (j <= i) M[i * ld + j] = a[i][j];
        X[i * ld + j] = (j <= i) ? x[i][j] : 0.0;
    }
    if (threadIdx.x == 0 && bad) atomicExch(fail, 1);
}

__global__ void k_copy_add_diag(const double* __restrict__ src, double* __restrict__ dst,
                                int64_t s_pad, double nu) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    int64_t i = e / s_pad, j = e % s_pad;
    dst[e] = src[e] + ((i == j) ? nu : 0.0);
}

// Frobenius norm^2 partials (single block, deterministic order).
__global__ void k_fro2(const double* __restrict__ M, int64_t m, double* __restrict__ out) {
    __shared__ double part[32];
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < m; e += blockDim.x) acc += M[e] * M[e];
    acc = msp::warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        v = msp::warp_sum(v);
        if (threadIdx.x == 0) *out = v;
    }
}

template <typename T>
__global__ void k_cast_tri(const double* __restrict__ X, T* __restrict__ B, T* __restrict__ Bt,
                           int64_t s_pad) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s_pad * s_pad) return;
    int64_t i = e / s_pad, j = e % s_pad;
    double v = (j <= i) ? X[e] : 0.0;
    B[e] = (T)v;
    Bt[j * s_pad + i] = (T)v;
}

msp_status dgemm(msp_ctx* ctx, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* Cm, int64_t ldc) {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    if (!ta && !tb) k_dgemm<false, false><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
    else if (!ta && tb) k_dgemm<false, true><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
    else if (ta && !tb) k_dgemm<true, false><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
    else k_dgemm<true, true><<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
    MSP_CHECK_LAUNCH(ctx);
    return MSP_OK;
}

// Recursive Cholesky + inverse of the n x n block at offset `off` of M (ld),
// inverse into X (same offsets); T1/T2 are n x n temporaries (ld).
msp_status chol_inv(msp_ctx* ctx, double* M, double* X, double* T1, double* T2, int64_t ld,
                    int64_t off, int64_t n, int* fail) {
    if (n <= 64) {
        static bool attr_set = false;
        if (!attr_set) {
            MSP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_chol_leaf,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kLeafSmem));
            attr_set = true;
        }
        k_chol_leaf<<<1, 256, kLeafSmem, ctx->stream>>>(M + off * ld + off, X + off * ld + off, ld,
                                                         (int)n, fail);
        MSP_CHECK_LAUNCH(ctx);
        return MSP_OK;
    }
    int64_t n1 = std::max<int64_t>(64, (n / 2) / 64 * 64);
    int64_t n2 = n - n1;
    double* A21 = M + (off + n1) * ld + off;
    double* A22 = M + (off + n1) * ld + off + n1;
    double* X11 = X + off * ld + off;
    double* X21 = X + (off + n1) * ld + off;
    double* X22 = X + (off + n1) * ld + off + n1;
    MSP_TRY(chol_inv(ctx, M, X, T1, T2, ld, off, n1, fail));
    // T1 = L21 = A21 X11^T   (n2 x n1)
    MSP_TRY(dgemm(ctx, false, true, n2, n1, n1, 1.0, A21, ld, X11, ld, 0.0, T1, ld));
    // A22 -= L21 L21^T
    MSP_TRY(dgemm(ctx, false, true, n2, n2, n1, -1.0, T1, ld, T1, ld, 1.0, A22, ld));
    MSP_TRY(chol_inv(ctx, M, X, T1 + n1, T2 + n1, ld, off + n1, n2, fail));
    // T2 = L21 X11; X21 = -X22 T2
    MSP_TRY(dgemm(ctx, false, false, n2, n1, n1, 1.0, T1, ld, X11, ld, 0.0, T2, ld));
    MSP_TRY(dgemm(ctx, false, false, n2, n1, n2, -1.0, X22, ld, T2, ld, 0.0, X21, ld));
    // store L21 into M
    MSP_CUDA_TRY(ctx, cudaMemcpy2DAsync(A21, ld * 8, T1, ld * 8, n1 * 8, n2,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
    return MSP_OK;
}

}  // namespace

// Build W (symmetrised), M2, its shifted Cholesky inverse, and the working
// copies B, Bt. `Ct` is C~ (phi_rows x s_pad, dtype of the sketch).
msp_status msp_build_factor(msp_ctx* ctx, msp_factor_s* f, const void* Ct, int64_t phi_rows) {
    const int64_t sp = f->s_pad;
    const size_t ts = dtype_size(f->dtype);
    // W symmetrise + FP64 copy
    {
        dim3 blk(32, 32), grid((unsigned)((sp + 31) / 32), (unsigned)((sp + 31) / 32));
        if (f->dtype == MSP_F32)
            k_symmetrize<float><<<grid, blk, 0, ctx->stream>>>((float*)f->W, f->W64, sp);
        else
            k_symmetrize<double><<<grid, blk, 0, ctx->stream>>>((double*)f->W, f->W64, sp);
        MSP_CHECK_LAUNCH(ctx);
    }
    // M2 = Ct^T Ct + lam_t W
    {
        dim3 grid((unsigned)(sp / 64), (unsigned)(sp / 64));
        if (f->dtype == MSP_F32)
            k_gram<float><<<grid, 256, 0, ctx->stream>>>((const float*)Ct, phi_rows, sp,
                                                         (const float*)f->W, f->lam_tilde, f->s,
                                                         sp, f->M2);
        else
            k_gram<double><<<grid, 256, 0, ctx->stream>>>((const double*)Ct, phi_rows, sp,
                                                          (const double*)f->W, f->lam_tilde, f->s,
                                                          sp, f->M2);
        MSP_CHECK_LAUNCH(ctx);
    }
    // factor with shift retries
    void* scr = nullptr;
    size_t mat = (size_t)sp * sp * 8;
    MSP_TRY(msp_scratch(ctx, 3 * mat + 256, &scr));
    double* Mw = (double*)scr;
    double* T1 = Mw + sp * sp;
    double* T2 = T1 + sp * sp;
    int* fail = (int*)(T2 + sp * sp);
    double* fro = (double*)(fail + 16);
    double nu = 0.0;
    int* hflag = (int*)ctx->host_flags;
    for (int attempt = 0; attempt <= 4; ++attempt) {
        unsigned blocks = (unsigned)((sp * sp + 255) / 256);
        k_copy_add_diag<<<blocks, 256, 0, ctx->stream>>>(f->M2, Mw, sp, nu);
        MSP_CHECK_LAUNCH(ctx);
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(f->Linv64, 0, mat, ctx->stream));
        MSP_CUDA_TRY(ctx, cudaMemsetAsync(fail, 0, sizeof(int), ctx->stream));
        MSP_TRY(chol_inv(ctx, Mw, f->Linv64, T1, T2, sp, 0, sp, fail));
        MSP_CUDA_TRY(ctx, cudaMemcpyAsync(hflag, fail, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        if (hflag[0] == 0) {
            f->shift = nu;
            f->retries = attempt;
            unsigned b2 = (unsigned)((sp * sp + 255) / 256);
            if (f->dtype == MSP_F32)
                k_cast_tri<float><<<b2, 256, 0, ctx->stream>>>(f->Linv64, (float*)f->B,
                                                               (float*)f->Bt, sp);
            else
                k_cast_tri<double><<<b2, 256, 0, ctx->stream>>>(f->Linv64, (double*)f->B,
                                                                (double*)f->Bt, sp);
            MSP_CHECK_LAUNCH(ctx);
            (void)ts;
            return MSP_OK;
        }
        if (attempt == 0) {
            k_fro2<<<1, 1024, 0, ctx->stream>>>(f->M2, sp * sp, fro);
            MSP_CHECK_LAUNCH(ctx);
            double h = 0.0;
            MSP_CUDA_TRY(ctx, cudaMemcpyAsync(&h, fro, 8, cudaMemcpyDeviceToHost, ctx->stream));
            MSP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            // first shift at the rounding level of the data M2 was assembled from
            nu = (f->dtype == MSP_F64 ? (double)f->s * std::ldexp(1.0, -52)
                                      : std::ldexp(1.0, -24)) * std::sqrt(h);
        } else {
            nu *= 100.0;
        }
    }
    return msp_set_error(ctx, MSP_ENOTPD,
                         "M2 + shift is not positive definite after 4 retries (last shift %g)",
                         nu / 100.0);
}
