// Reweighted energy distribution and the order-disorder interface tension (Sec. 5).
//
// ln P_beta(E_b) = ln n_b - ln W_b - beta E_b - ln sum_b' exp(...) over the sampled bins
// of the production sums (Eq. 2 applied to the energy histogram itself), one block per
// beta in FP64.  The interface tension follows Sec. 5: at the temperature where the two
// peaks of P_beta are equally high, sigma_od(L) = ln(P_max / P_min) / (2 L).  The peak
// search and the root finding are host code over the distributions the kernel returns.
#include <cmath>
#include <vector>

#include "muca_internal.cuh"

namespace muca {
namespace {

__global__ void __launch_bounds__(256) energy_dist_kernel(const uint64_t *samples, const double *lnw, int model,
                                                          int V, int n_bins, const double *betas, double *out)
{
    __shared__ double s_red[8];
    const double beta = betas[blockIdx.x];
    double *g = out + (size_t)blockIdx.x * n_bins;
    // pass 1: g_b and its maximum
    double mx = -INFINITY;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const uint64_t n = samples[b];
        double v = -INFINITY;
        if (n) {
            const double E = model == MUCA_ISING ? (double)(4 * b - 2 * V) : (double)(b - 2 * V);
            v = __dsub_rn(__dsub_rn(log((double)n), lnw[b]), __dmul_rn(beta, E));
        }
        g[b] = v;
        mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, s_red[w]);
    __syncthreads();
    // pass 2: sum of exp(g - max)
    double sum = 0.0;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double v = g[b];
        if (v != -INFINITY) sum += exp(v - mx);
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
    __syncthreads();
    sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[w];
    const double norm = mx + log(sum);
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) g[b] -= norm;  // -inf stays -inf
}

// ln P for n_beta betas (device) into out [n_beta][n_bins] (device)
int energy_dist(muca_ctx *ctx, const double *d_betas, int n_beta, double *d_out)
{
    energy_dist_kernel<<<n_beta, 256, 0, ctx->stream>>>(ctx->d_samples, ctx->d_lnw_prod, ctx->model, ctx->V,
                                                         ctx->n_bins, d_betas, d_out);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

struct Peaks {
    int b1, b2, dip;
    double h;  // ln P(b1) - ln P(b2), NaN if there are not two peaks
};

// Two peaks of ln P g: split at s, highest bin on each side (first on ties), s moved to
// the lowest bin between them (first on ties; unsampled bins never count), until s
// stays (at most 64 rounds); two peaks only if the dip is strictly inside and below.
Peaks two_peaks(const double *g, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < nb && !std::isfinite(g[lo])) ++lo;
    while (hi >= 0 && !std::isfinite(g[hi])) --hi;
    Peaks p{0, 0, 0, NAN};
    if (lo > hi) return p;
    int s = (lo + hi) / 2;
    int b1 = s, b2 = s, dip = s;
    for (int round = 0; round < 64; ++round) {
        int l = -1, r = -1;
        for (int b = lo; b <= s; ++b)
            if (std::isfinite(g[b]) && (l < 0 || g[b] > g[l])) l = b;
        for (int b = s + 1; b <= hi; ++b)
            if (std::isfinite(g[b]) && (r < 0 || g[b] > g[r])) r = b;
        if (l < 0 || r < 0) break;
        b1 = l;
        b2 = r;
        int d = -1;
        for (int b = b1; b <= b2; ++b)
            if (std::isfinite(g[b]) && (d < 0 || g[b] < g[d])) d = b;
        dip = d;
        if (dip == s) break;
        s = dip;
    }
    p.b1 = b1;
    p.b2 = b2;
    p.dip = dip;
    if (b1 < dip && dip < b2 && g[dip] < g[b1] && g[dip] < g[b2]) p.h = g[b1] - g[b2];
    return p;
}

}  // namespace
}  // namespace muca

using namespace muca;

extern "C" int muca_energy_distribution(muca_ctx *ctx, const double *betas, int n_beta, double *lnP_out)
{
    if (!ctx) return fail(MUCA_ERR_ARG, "null context");
    if (!betas || !lnP_out || n_beta < 1) return fail(MUCA_ERR_ARG, "need betas, lnP_out and n_beta >= 1");
    if (ctx->cfg.ensemble != MUCA_ENSEMBLE_ENERGY)
        return fail(MUCA_ERR_STATE, "no energy production sums in the multimagnetic ensemble");
    if (!ctx->samples_active) return fail(MUCA_ERR_STATE, "no production sums: run muca_produce first");
    cudaSetDevice(ctx->device);
    double *d_b = nullptr, *d_o = nullptr;
    const size_t nout = (size_t)n_beta * ctx->n_bins;
    if (cudaMalloc(reinterpret_cast<void **>(&d_b), sizeof(double) * n_beta) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&d_o), sizeof(double) * nout) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_b);
        return fail(MUCA_ERR_OOM, "energy distribution scratch");
    }
    int rc = MUCA_OK;
    if (cudaMemcpyAsync(d_b, betas, sizeof(double) * n_beta, cudaMemcpyDefault, ctx->stream) != cudaSuccess)
        rc = fail(MUCA_ERR_CUDA, "copy of betas");
    if (!rc) rc = energy_dist(ctx, d_b, n_beta, d_o);
    if (!rc && cudaMemcpyAsync(lnP_out, d_o, sizeof(double) * nout, cudaMemcpyDefault, ctx->stream) != cudaSuccess)
        rc = fail(MUCA_ERR_CUDA, "copy of the distributions");
    if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = fail(MUCA_ERR_CUDA, "synchronise");
    cudaFree(d_b);
    cudaFree(d_o);
    return rc;
}

extern "C" int muca_interface_tension(muca_ctx *ctx, double beta_lo, double beta_hi, int n_grid, int n_bisect,
                                      double *beta_eqh, double *ln_ratio, int *peaks)
{
    if (!ctx) return fail(MUCA_ERR_ARG, "null context");
    if (!(beta_hi > beta_lo) || n_grid < 2 || n_bisect < 0) return fail(MUCA_ERR_ARG, "bad bracket or counts");
    const int nb = ctx->n_bins;
    std::vector<double> grid(n_grid), dist((size_t)n_grid * nb);
    const double step = (beta_hi - beta_lo) / (n_grid - 1);
    for (int i = 0; i < n_grid; ++i) grid[i] = i == n_grid - 1 ? beta_hi : beta_lo + i * step;
    int rc = muca_energy_distribution(ctx, grid.data(), n_grid, dist.data());
    if (rc) return rc;
    if (beta_eqh) *beta_eqh = NAN;
    if (ln_ratio) *ln_ratio = NAN;
    if (peaks) peaks[0] = peaks[1] = peaks[2] = -1;
    // bracket: the first grid interval where h goes from negative to non-negative
    int k = -1;
    for (int i = 0; i + 1 < n_grid && k < 0; ++i) {
        const double h0 = two_peaks(&dist[(size_t)i * nb], nb).h, h1 = two_peaks(&dist[(size_t)(i + 1) * nb], nb).h;
        if (h0 < 0.0 && h1 >= 0.0) k = i;  // false for NaN
    }
    if (k < 0) return MUCA_OK;
    double a = grid[k], b = grid[k + 1];
    std::vector<double> g(nb);
    for (int it = 0; it < n_bisect; ++it) {
        double mid = 0.5 * (a + b);
        if ((rc = muca_energy_distribution(ctx, &mid, 1, g.data()))) return rc;
        const double h = two_peaks(g.data(), nb).h;
        if (std::isnan(h)) return MUCA_OK;
        if (h < 0.0)
            a = mid;
        else
            b = mid;
    }
    double beta = 0.5 * (a + b);
    if ((rc = muca_energy_distribution(ctx, &beta, 1, g.data()))) return rc;
    const Peaks p = two_peaks(g.data(), nb);
    if (std::isnan(p.h)) return MUCA_OK;
    if (beta_eqh) *beta_eqh = beta;
    if (ln_ratio) *ln_ratio = 0.5 * (g[p.b1] + g[p.b2]) - g[p.dip];
    if (peaks) {
        peaks[0] = p.b1;
        peaks[1] = p.b2;
        peaks[2] = p.dip;
    }
    return MUCA_OK;
}
