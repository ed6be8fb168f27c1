// Weight side of the parallel multicanonical method (arXiv:1212.3975, Secs. 2-3), on
// the device: the master-process step of the paper (histogram in, new weights out)
// runs as one FP64 kernel whose result every sweep block reads from global memory,
// so no host round trip and no broadcast is needed.
//
// FP64 operations use explicit round-to-nearest intrinsics (and this file is built
// with -fmad=false) so that every sum and product is rounded in the order the
// recursion is written; only exp/log come from the CUDA math library.
#include <algorithm>

#include "muca_internal.cuh"

namespace muca {
namespace {

__device__ __forceinline__ int bin_delta(int model, int col)
{
    if (model == MUCA_ISING) return col < 2 ? col - 2 : col - 1;  // -2 -1 1 2
    return col < 4 ? col - 4 : col - 3;                            // -4..-1 1..4
}

// Acceptance thresholds (Eq. 1 as an integer test): d = lnW[b'] - lnW[b];
// A = 2^32-1 if d >= 0, else min(floor(2^32 exp(d)), 2^32-1); 0 if b' is out of range
// or inaccessible (never entered).
__global__ void thresholds_kernel(const double *lnw, const uint8_t *acc, uint32_t *thr, int model, int n_bins,
                                  int n_de)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bins * n_de) return;
    const int b = t / n_de, col = t % n_de;
    const int bp = b + bin_delta(model, col);
    uint32_t A = 0u;
    if (acc[b] && bp >= 0 && bp < n_bins && acc[bp]) {
        const double d = __dsub_rn(lnw[bp], lnw[b]);
        if (d >= 0.0) {
            A = kAlways;
        } else {
            const double x = floor(ldexp(exp(d), 32));
            A = x >= 4294967295.0 ? kAlways : (uint32_t)x;
        }
    }
    thr[t] = A;
}

// Kernel layout of the thresholds for the warp-specialised sweep bodies: one row per
// bin, one column per local configuration so that the column offset follows from the
// neighbours without a branch.  Ising: column = number of unequal neighbours n
// (dE = 8 - 4n, so n = 2 is dE = 0 and always accepts); Potts: column = dE + 4.
__global__ void ktab_kernel(const uint32_t *thr, uint32_t *ktab, int model, int n_bins)
{
    const int width = model == MUCA_ISING ? 5 : 9;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bins * width) return;
    const int b = t / width, k = t % width;
    uint32_t v;
    if (model == MUCA_ISING) {
        // API columns by ascending dE: -8, -4, 4, 8 (n = 4, 3, 1, 0)
        v = k == 2 ? kAlways : thr[b * 4 + (k >= 3 ? 4 - k : 3 - k)];
    } else {
        const int dE = k - 4;
        v = dE == 0 ? kAlways : thr[b * 8 + (dE < 0 ? dE + 4 : dE + 3)];
    }
    ktab[t] = v;
}

struct BlockStats {
    unsigned long long total, mn, mx, n_sampled, K;
    int lo, hi;
};

// Single-block update (blockDim.x = 1024):
//   1. convergence statistics of H over accessible bins (Sec. 3);
//   2. recursion (Sec. 2) into per-pair differences d[u] (accumulated) or values;
//   3. sequential prefix over accessible bins in ascending order (thread 0);
//   4. boundary correction beyond [lo, hi] with the slope of the innermost
//      `width` bins (Sec. 3);
//   5. ln W -= max over accessible bins; inaccessible bins = 0.
__device__ __forceinline__ void update_body(double *lnw, double *P, double *scratch, const uint64_t *H,
                                            const uint8_t *acc, int n_bins, int accumulated, int width_cfg,
                                            muca_iter_stats *stats)
{
    __shared__ unsigned long long s_total[32], s_min[32], s_max[32], s_ns[32], s_K[32];
    __shared__ int s_lo[32], s_hi[32];
    __shared__ double s_top[32];
    __shared__ int sh_lo, sh_hi;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

    // 1. statistics
    unsigned long long tot = 0, mn = ~0ull, mx = 0, ns = 0, K = 0;
    int lo = n_bins, hi = -1;
    for (int b = tid; b < n_bins; b += blockDim.x) {
        if (!acc[b]) continue;
        const unsigned long long h = H[b];
        tot += h;
        mn = min(mn, h);
        mx = max(mx, h);
        K += 1;
        if (h) {
            ns += 1;
            lo = min(lo, b);
            hi = max(hi, b);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
        K += __shfl_xor_sync(0xffffffffu, K, o);
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        s_total[warp] = tot; s_min[warp] = mn; s_max[warp] = mx; s_ns[warp] = ns; s_K[warp] = K;
        s_lo[warp] = lo; s_hi[warp] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; ++w) {
            tot += s_total[w]; mn = min(mn, s_min[w]); mx = max(mx, s_max[w]); ns += s_ns[w]; K += s_K[w];
            lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]);
        }
        const double mean = (double)tot / (double)K;
        muca_iter_stats st;
        st.covered = (ns == K);
        st.flat = st.covered && ((double)mn >= 0.5 * mean) && ((double)mx <= 2.0 * mean);
        st.lo = hi >= 0 ? lo : -1;
        st.hi = hi >= 0 ? hi : -1;
        st.n_sampled = (int64_t)ns;
        st.min_over_mean = mean > 0 ? (double)mn / mean : 0.0;
        st.max_over_mean = mean > 0 ? (double)mx / mean : 0.0;
        st.total = tot;
        *stats = st;
        sh_lo = st.lo;
        sh_hi = st.hi;
    }
    __syncthreads();

    // 2. recursion.  scratch[u] = difference to the next accessible bin (accumulated)
    if (accumulated) {
        for (int u = tid; u < n_bins; u += blockDim.x) {
            if (!acc[u]) continue;
            int v = u + 1;
            while (v < n_bins && !acc[v]) ++v;
            if (v >= n_bins) continue;
            double d = __dsub_rn(lnw[v], lnw[u]);
            const uint64_t hu_i = H[u], hv_i = H[v];
            if (hu_i > 0 && hv_i > 0) {
                const double hu = (double)hu_i, hv = (double)hv_i;
                const double g0 = __ddiv_rn(__dmul_rn(hu, hv), __dadd_rn(hu, hv));
                const double pu = __dadd_rn(P[u], g0);
                P[u] = pu;
                const double g = __ddiv_rn(g0, pu);
                d = __dsub_rn(d, __dmul_rn(g, __dsub_rn(log(hv), log(hu))));
            }
            scratch[u] = d;
        }
    } else {
        for (int b = tid; b < n_bins; b += blockDim.x) {
            if (!acc[b]) continue;
            double v = lnw[b];
            if (H[b] > 0) v = __dsub_rn(v, log((double)H[b]));
            scratch[b] = v;
        }
    }
    __syncthreads();

    // 3. prefix in ascending order (one thread: keeps the oracle's rounding order)
    if (tid == 0) {
        if (accumulated) {
            int u = 0;
            while (!acc[u]) ++u;
            double cur = 0.0;
            lnw[u] = cur;
            for (int v = u + 1; v < n_bins; ++v) {
                if (!acc[v]) continue;
                cur = __dadd_rn(cur, scratch[u]);
                lnw[v] = cur;
                u = v;
            }
        }
    }
    if (!accumulated) {
        for (int b = tid; b < n_bins; b += blockDim.x)
            if (acc[b]) lnw[b] = scratch[b];
    }
    __syncthreads();

    // 4. boundary correction
    const int slo = sh_lo, shi = sh_hi;
    if (slo >= 0 && shi > slo) {
        const int width = min(width_cfg, shi - slo);
        __shared__ double sl_lo, sl_hi;
        if (tid == 0) {
            int b2 = slo + width;
            while (!acc[b2]) ++b2;
            int b1 = shi - width;
            while (!acc[b1]) --b1;
            sl_lo = __ddiv_rn(__dsub_rn(lnw[b2], lnw[slo]), (double)(b2 - slo));
            sl_hi = __ddiv_rn(__dsub_rn(lnw[shi], lnw[b1]), (double)(shi - b1));
        }
        __syncthreads();
        const double vlo = lnw[slo], vhi = lnw[shi];
        __syncthreads();
        for (int b = tid; b < n_bins; b += blockDim.x) {
            if (!acc[b]) continue;
            if (b < slo) lnw[b] = __dadd_rn(vlo, __dmul_rn(sl_lo, (double)(b - slo)));
            else if (b > shi) lnw[b] = __dadd_rn(vhi, __dmul_rn(sl_hi, (double)(b - shi)));
        }
    }
    __syncthreads();

    // 5. normalisation: max over accessible bins is 0
    double top = -INFINITY;
    for (int b = tid; b < n_bins; b += blockDim.x)
        if (acc[b]) top = fmax(top, lnw[b]);
    for (int o = 16; o > 0; o >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, o));
    if (lane == 0) s_top[warp] = top;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; ++w) top = fmax(top, s_top[w]);
        s_top[0] = top;
    }
    __syncthreads();
    top = s_top[0];
    for (int b = tid; b < n_bins; b += blockDim.x) lnw[b] = acc[b] ? __dsub_rn(lnw[b], top) : 0.0;
}

__global__ void __launch_bounds__(1024) update_kernel(double *lnw, double *P, double *scratch, const uint64_t *H,
                                                      const uint8_t *acc, int n_bins, int accumulated,
                                                      int width_cfg, muca_iter_stats *stats)
{
    update_body(lnw, P, scratch, H, acc, n_bins, accumulated, width_cfg, stats);
}

// one block per lattice of a batch
__global__ void __launch_bounds__(1024) update_batch_kernel(const BatchJob *jobs)
{
    const BatchJob &j = jobs[blockIdx.x];
    if (!*j.active) return;  // converged lattice: frozen
    update_body(j.lnw, j.P, j.wscratch, j.H, j.acc, j.n_bins, j.accumulated, j.width, j.stats);
}

// thresholds of every lattice of a batch: blockIdx.y = lattice
__global__ void thresholds_batch_kernel(const BatchJob *jobs)
{
    const BatchJob &j = jobs[blockIdx.y];
    if (!*j.active) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < j.n_bins * j.n_de; t += gridDim.x * blockDim.x) {
        const int b = t / j.n_de, col = t % j.n_de;
        const int bp = b + bin_delta(j.model, col);
        uint32_t A = 0u;
        if (j.acc[b] && bp >= 0 && bp < j.n_bins && j.acc[bp]) {
            const double d = __dsub_rn(j.lnw[bp], j.lnw[b]);
            if (d >= 0.0) {
                A = kAlways;
            } else {
                const double x = floor(ldexp(exp(d), 32));
                A = x >= 4294967295.0 ? kAlways : (uint32_t)x;
            }
        }
        j.thr[t] = A;
    }
}

}  // namespace

cudaError_t launch_batch_update(const BatchJob *d_jobs, int n_jobs, int max_thr, cudaStream_t st)
{
    update_batch_kernel<<<n_jobs, 1024, 0, st>>>(d_jobs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((max_thr + 255) / 256, n_jobs);
    thresholds_batch_kernel<<<grid, 256, 0, st>>>(d_jobs);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(2);
    return e;
}

int launch_thresholds(muca_ctx *ctx)
{
    if (ctx->cfg.ensemble == MUCA_ENSEMBLE_MAGNETIZATION) return launch_muma_thresholds(ctx);
    const int n = ctx->n_bins * ctx->n_de;
    thresholds_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_lnw, ctx->d_acc, ctx->d_thr, ctx->model,
                                                               ctx->n_bins, ctx->n_de);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    ctx->ktab_dirty = 1;
    return MUCA_OK;
}

int launch_update(muca_ctx *ctx)
{
    const int width = ctx->cfg.correction_width > 0 ? ctx->cfg.correction_width : ctx->L;
    update_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->d_lnw, ctx->d_P, ctx->d_wscratch, ctx->d_H, ctx->d_acc, ctx->n_bins,
                                               ctx->cfg.recursion == MUCA_RECURSION_ACCUMULATED, width,
                                               ctx->d_stats);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return launch_thresholds(ctx);
}

int launch_ktab(muca_ctx *ctx)
{
    const int width = ctx->model == MUCA_ISING ? 5 : 9;
    const int n = ctx->n_bins * width;
    ktab_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_thr, ctx->d_ktab, ctx->model, ctx->n_bins);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    ctx->ktab_dirty = 0;
    return MUCA_OK;
}

}  // namespace muca
