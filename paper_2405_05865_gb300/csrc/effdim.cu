// Effective dimension d_lambda = tr(A (A + lambda I)^{-1}) (Section 2, the
// quantity of Lemma 2.1 that sets the sketch size in the KRR analysis of
// Section 3), estimated by Hutchinson over regularised solves:
//   d_lambda = n - lambda tr((A + lambda I)^{-1}),
//   tr((A + lambda I)^{-1}) ~ (1/m) sum_j g_j^T (A + lambda I)^{-1} g_j.
// The m Rademacher probes are the right-hand sides of one batch whose
// instances all name A, so the sketch, the factor and the tiled copy of A are
// built once and the solves run in the batched kernel, 16 probes per instance.
#include "msp_internal.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

// B[j n + i] = -1 iff the top bit of draw(seed, 7 + 2 floor(j / 256), i,
// j mod 256) is set, else +1 (the probes of msp_schatten), column-major n x m.
__global__ void k_probe_cols(int64_t n, int64_t m, uint64_t seed, double* __restrict__ B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int64_t j = e / n, i = e % n;
    const uint64_t d = msp::draw(seed, 7u + 2u * (uint32_t)(j / 256), (uint64_t)i, (uint32_t)(j % 256));
    B[e] = (d >> 63) ? -1.0 : 1.0;
}

// q[j] = n - lambda g_j^T x_j, one block per probe, fixed-order sums.
__global__ void __launch_bounds__(256) k_probe_vals(const double* __restrict__ B, const double* __restrict__ X,
                                                   int64_t n, double lambda, double* __restrict__ q) {
    __shared__ double red[8];
    const double* b = B + (int64_t)blockIdx.x * n;
    const double* x = X + (int64_t)blockIdx.x * n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += b[i] * x[i];
    acc = msp::warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        q[blockIdx.x] = (double)n - lambda * t;
    }
}

}  // namespace

extern "C" msp_status msp_effective_dimension(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, double lambda,
                                              int64_t probes, uint64_t seed, int64_t s, int gamma,
                                              const msp_opts* opts, double* estimate, double* std_err,
                                              double* q_out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!A || n < 16 || lda < n || !(lambda > 0.0) || probes < 2 || probes > 4096)
        return msp_set_error(ctx, MSP_EINVAL,
                             "effective_dimension: need A, n >= 16, lda >= n, lambda > 0, 2 <= probes <= 4096");
    msp::DeviceGuard guard(ctx->device);
    const int64_t m = probes;
    void* mem = nullptr;
    const size_t vb = (size_t)round_up(n * m * 8, 256);
    MSP_TRY(msp_alloc(ctx, &mem, 2 * vb + (size_t)m * 8));
    double* B = (double*)mem;
    double* X = (double*)((char*)mem + vb);
    double* qd = (double*)((char*)mem + 2 * vb);
    msp_status st = MSP_OK;
    msp_batch_t* bt = nullptr;
    auto done = [&](msp_status r) {
        cudaStreamSynchronize(ctx->stream);
        if (bt) msp_batch_destroy(bt);
        cudaFreeAsync(mem, ctx->stream);
        return r;
    };
    k_probe_cols<<<(unsigned)((n * m + 255) / 256), 256, 0, ctx->stream>>>(n, m, seed, B);
    if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "effective_dimension: launch"));
    ++ctx->launches;
    // one instance per 16 probes, all on A: set-up shared by the batch
    const int nchunk = (int)((m + 15) / 16);
    std::vector<msp_instance> inst(nchunk);
    for (int c = 0; c < nchunk; ++c) {
        msp_instance& I = inst[c];
        std::memset(&I, 0, sizeof I);
        I.A = A;
        I.n = n;
        I.lda = lda;
        I.lambda = lambda;
        I.B = B + (int64_t)c * 16 * n;
        I.ldb = n;
        I.X = X + (int64_t)c * 16 * n;
        I.ldx = n;
        I.m = (int)std::min<int64_t>(16, m - 16 * (int64_t)c);
        I.gamma = gamma;
        I.s = s;
        I.phi = 0;
        I.gamma_phi = 8;
        I.seed = seed;
    }
    if ((st = msp_batch_create(ctx, nchunk, inst.data(), &bt)) != MSP_OK) return done(st);
    std::vector<msp_info> infos(nchunk);
    const msp_status sst = msp_batch_solve(ctx, bt, opts, infos.data());
    if (sst != MSP_OK && sst != MSP_ENOCONV) return done(sst);
    k_probe_vals<<<(unsigned)m, 256, 0, ctx->stream>>>(B, X, n, lambda, qd);
    if (cudaGetLastError() != cudaSuccess) return done(msp_set_error(ctx, MSP_ECUDA, "effective_dimension: launch"));
    ++ctx->launches;
    std::vector<double> q(m);
    if (cudaMemcpyAsync(q.data(), qd, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        (q_out && cudaMemcpyAsync(q_out, qd, (size_t)m * 8, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return done(msp_set_error(ctx, MSP_ECUDA, "effective_dimension: copy-out failed"));
    }
    double mean = 0.0;
    for (double v : q) mean += v;
    mean /= (double)m;
    double var = 0.0;
    for (double v : q) var += (v - mean) * (v - mean);
    var /= (double)(m - 1);
    if (estimate) *estimate = mean;
    if (std_err) *std_err = std::sqrt(var / (double)m);
    return done(sst);
}

// Parameters from d_lambda (Section 3, the proof of the KRR corollary, and
// Lemma 2.1): l = ceil(2 d), for which lambda_l <= lambda (Lemma 2.1(1) with
// gamma = 1); s = l rounded up to 16 and capped at the largest sketch the
// library builds; lambda0 = 2 lambda d / s, which bounds the paper's
// (2/s) sum_{i > s} lambda_i from above when s >= d (Lemma 2.1(2)); with the
// cap below that (s < d) the lemma says nothing and lambda0 = 0 (plain
// Nystrom preconditioner M = A_nys + lambda I). d >= n/4 marks the regime
// where the paper solves directly.
extern "C" msp_status msp_params_from_effdim(double d, int64_t n, double lambda, msp_param_choice* out) {
    if (!out || !(d >= 0.0) || !std::isfinite(d) || n < 16 || !(lambda > 0.0)) return MSP_EINVAL;
    const int64_t s_max = std::min<int64_t>(n, 1024) / 16 * 16;
    const int64_t l = std::max<int64_t>(1, (int64_t)std::ceil(2.0 * d));
    const int64_t s = std::max<int64_t>(16, std::min<int64_t>(s_max, (l + 15) / 16 * 16));
    out->d_lambda = d;
    out->l = l;
    out->s = s;
    out->capped = s < l ? 1 : 0;
    out->lambda0 = ((double)s >= d) ? 2.0 * lambda * d / (double)s : 0.0;
    out->direct = (4.0 * d >= (double)n) ? 1 : 0;
    return MSP_OK;
}

extern "C" msp_status msp_auto_params(msp_ctx* ctx, const float* A, int64_t n, int64_t lda, double lambda,
                                      int64_t probes, uint64_t seed, int gamma, const msp_opts* opts,
                                      msp_param_choice* out) {
    if (!ctx) return msp_set_error(nullptr, MSP_EINVAL, "ctx is NULL");
    if (!out) return msp_set_error(ctx, MSP_EINVAL, "auto_params: out is NULL");
    if (n < 16) return msp_set_error(ctx, MSP_EINVAL, "auto_params: need n >= 16");
    // pilot: the largest sketch, no shift
    const int64_t s_pilot = std::min<int64_t>(n, 1024) / 16 * 16;
    double d = 0.0, se = 0.0;
    const msp_status st = msp_effective_dimension(ctx, A, n, lda, lambda, probes, seed, s_pilot, gamma, opts, &d,
                                                  &se, nullptr);
    if (st != MSP_OK) return st;
    // the estimate can leave [0, n] by its spread: clamp to the range of tr
    const double dc = std::min<double>((double)n, std::max(0.0, d));
    if (msp_params_from_effdim(dc, n, lambda, out) != MSP_OK)
        return msp_set_error(ctx, MSP_EINVAL, "auto_params: bad estimate %g", d);
    out->d_lambda = d;
    out->d_std_err = se;
    return MSP_OK;
}
