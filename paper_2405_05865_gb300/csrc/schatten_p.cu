// Schatten-p norms, p in (0, 2), of a general A (m x n, m >= n) from ridge
// solves (Section 3.2: the estimator needs only solves with A^T A + t I,
// eq. schatten-ridge, and a random diagonal shift A + zI for square A).
// The black box of that section is not printed; the integral
// representation used here (Balakrishnan's formula) is, with q = p/2,
//     |A|_p^p = (sin(pi q)/pi) int_0^inf t^(q-1) d_t dt,
//     d_t = tr(A^T A (A^T A + t I)^{-1}) = n - t tr((A^T A + t I)^{-1}),
// evaluated by the trapezoidal rule in u = ln t over [t_min, t_max] with
// geometric tails from the asymptotic forms d_t ~ n (t -> 0) and
// d_t ~ |A|_F^2 / t (t -> inf); each d_t is a Hutchinson mean over the same
// Rademacher probes g_k, each term a solve (A^T A + t I) x = g_k by the
// three-level handle (msp_general_solve), one handle for all nodes
// (msp_general_set_lambda).
#include "msp_internal.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

// g[i] = -1 iff the top bit of draw(seed, 7 + 2 floor(k / 256), i, k mod 256)
// is set, else +1: probe k of msp_schatten / msp_hutchinson, FP64, length n
__global__ void k_probe_vec(int64_t n, int64_t k, uint64_t seed, double* __restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t d = msp::draw(seed, 7u + 2u * (uint32_t)(k / 256), (uint64_t)i, (uint32_t)(k % 256));
    g[i] = (d >> 63) ? -1.0 : 1.0;
}

// colsq[j] = sum_i A[i][j]^2 (FP64; thread per column, rows in order)
__global__ void k_colsq(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, double* __restrict__ colsq) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const double v = A[i * lda + j];
        s = fma(v, v, s);
    }
    colsq[j] = s;
}

// B = A with z added to the diagonal (square, row-major, ld = lda)
__global__ void k_copy_shift(const float* __restrict__ A, int64_t n, int64_t lda, float z, float* __restrict__ B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    B[i * n + j] = A[i * lda + j] + (i == j ? z : 0.f);
}

// out = x . y (one block, FP64, fixed order)
__global__ void k_dot64(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], y[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

}  // namespace

extern "C" msp_status msp_schatten_p(msp_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, double p,
                                     double z, double t_min, double t_max, int nodes, int64_t probes,
                                     uint64_t seed, int64_t s, double lambda_floor_rel, const msp_opts* opts,
                                     double* estimate, double* std_err, double* X) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || !(p > 0.0) || !(p < 2.0) || !(t_min > 0.0) || !(t_max > t_min) || nodes < 2 || nodes > 4096 ||
        probes < 1 || probes > 4096 || !(lambda_floor_rel >= 0.0) || (z != 0.0 && m != n))
        return msp_set_error(ctx, MSP_EINVAL,
                             "schatten_p: need 0 < p < 2, 0 < t_min < t_max, 2 <= nodes <= 4096, "
                             "1 <= probes <= 4096, lambda_floor_rel >= 0, a square A for z != 0");
    msp::DeviceGuard guard(ctx->device);
    const double q = 0.5 * p;
    // device scratch: shifted copy (z != 0), column squares, probe, solution, dot
    float* Az = nullptr;
    double* work = nullptr;
    msp_general_t* g = nullptr;
    auto done = [&](msp_status r) {
        cudaStreamSynchronize(ctx->stream);
        if (g) msp_general_destroy(g);
        if (Az) cudaFreeAsync(Az, ctx->stream);
        if (work) cudaFreeAsync(work, ctx->stream);
        return r;
    };
    const float* Ause = A;
    int64_t ld = lda;
    if (z != 0.0) {
        MSP_TRY(msp_alloc(ctx, (void**)&Az, (size_t)n * n * 4));
        k_copy_shift<<<(unsigned)((n * n + 255) / 256), 256, 0, ctx->stream>>>(A, n, lda, (float)z, Az);
        if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: launch"));
        ++ctx->launches;
        Ause = Az;
        ld = n;
    }
    msp_status st = msp_alloc(ctx, (void**)&work, (size_t)(3 * n + 8) * 8);
    if (st != MSP_OK) return done(st);
    double* colsq = work;
    double* gk = work + n;
    double* xk = work + 2 * n;
    double* dot = work + 3 * n;
    k_colsq<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(Ause, m, n, ld, colsq);
    if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: launch"));
    ++ctx->launches;
    std::vector<double> cs(n);
    if (cudaMemcpyAsync(cs.data(), colsq, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: copy failed"));
    double fro2 = 0.0, cmax = 0.0;
    for (double v : cs) {
        fro2 += v;
        cmax = std::max(cmax, v);
    }
    const double step = (std::log(t_max) - std::log(t_min)) / (nodes - 1);
    auto tnode = [&](int j) { return std::exp(std::log(t_min) + step * j); };
    const double t0 = tnode(0);
    // the handle starts with lam~ = |A|_F^2 >= |A|_2^2 (safe for any A)
    if ((st = msp_general_create(ctx, Ause, m, n, ld, t0, std::max(0.0, fro2 - t0), s, 8,
                                 std::min<int64_t>(4 * s, m), 8, seed, &g)) != MSP_OK)
        return done(st);
    // |A|_2^2 by the power method on (A^T A + t0 I) (the estimate the shift
    // argument of Section 3.2 also uses); lam~ >= lambda_floor_rel |A|_2^2
    // keeps the FP32 levels' cancellation |A|^2 / lam~ bounded
    double smax2 = cmax;
    {
        float* pv = nullptr;
        if ((st = msp_alloc(ctx, (void**)&pv, (size_t)2 * n * 4)) != MSP_OK) return done(st);
        float* qv = pv + n;
        std::vector<float> hv(n), hq(n);
        for (int64_t i = 0; i < n; ++i) hv[i] = (i % 3 == 0 ? 1.f : -0.5f) + 1e-3f * (float)(i % 7);
        double lam_est = 0.0;
        for (int it = 0; it < 30 && st == MSP_OK; ++it) {
            double nn = 0.0;
            for (float v : hv) nn += (double)v * v;
            const float inv = (float)(1.0 / std::sqrt(nn));
            for (float& v : hv) v *= inv;
            if (cudaMemcpyAsync(pv, hv.data(), (size_t)n * 4, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
                st = msp_set_error(ctx, MSP_ECUDA, "schatten_p: copy failed");
            if (st == MSP_OK) st = msp_general_op(ctx, g, pv, qv);
            if (st == MSP_OK && (cudaMemcpyAsync(hq.data(), qv, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                                 ctx->stream) != cudaSuccess ||
                                 cudaStreamSynchronize(ctx->stream) != cudaSuccess))
                st = msp_set_error(ctx, MSP_ECUDA, "schatten_p: copy failed");
            double r = 0.0;
            for (int64_t i = 0; i < n; ++i) r += (double)hv[i] * hq[i];
            lam_est = r - t0;
            hv.swap(hq);
        }
        cudaFreeAsync(pv, ctx->stream);
        if (st != MSP_OK) return done(st);
        smax2 = std::max(smax2, lam_est);
    }
    const double floor = lambda_floor_rel * smax2;
    msp_opts o;
    if (opts) o = *opts;
    else msp_default_opts(&o);
    std::vector<double> V((size_t)nodes * probes);
    for (int j = 0; j < nodes; ++j) {
        const double t = tnode(j);
        if ((st = msp_general_set_lambda(ctx, g, t, std::max(0.0, floor - t))) != MSP_OK) return done(st);
        for (int64_t k = 0; k < probes; ++k) {
            k_probe_vec<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, k, seed, gk);
            if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: launch"));
            ++ctx->launches;
            msp_info inf;
            st = msp_general_solve(ctx, g, gk, xk, &o, &inf);
            if (st != MSP_OK) return done(st);
            k_dot64<<<1, 1024, 0, ctx->stream>>>(n, gk, xk, dot);
            if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: launch"));
            ++ctx->launches;
            double h = 0.0;
            if (cudaMemcpyAsync(&h, dot, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                return done(msp_set_error(ctx, MSP_ECUDA, "schatten_p: copy failed"));
            V[(size_t)j * probes + k] = (double)n - t * h;
        }
    }
    // per-probe estimates with the geometric tails
    const double c = std::sin(M_PI * q) / M_PI;
    const double a = std::exp(-q * step), b = std::exp(-(1.0 - q) * step);
    const double lower = step * (double)n * std::pow(t_min, q) * a / (1.0 - a);
    const double upper = step * fro2 * std::pow(t_max, q - 1.0) * b / (1.0 - b);
    std::vector<double> Xk(probes);
    double mean = 0.0;
    for (int64_t k = 0; k < probes; ++k) {
        double body = 0.0;
        for (int j = 0; j < nodes; ++j) body += step * std::pow(tnode(j), q) * V[(size_t)j * probes + k];
        Xk[k] = c * (body + lower + upper);
        mean += Xk[k];
    }
    mean /= (double)probes;
    double var = 0.0;
    for (double v : Xk) var += (v - mean) * (v - mean);
    if (estimate) *estimate = mean;
    if (std_err) *std_err = probes > 1 ? std::sqrt(var / (double)(probes - 1) / (double)probes) : NAN;
    if (X) std::memcpy(X, Xk.data(), (size_t)probes * 8);
    return done(MSP_OK);
}
