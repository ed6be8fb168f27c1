// Multimagnetic Ising ensemble (Sec. 4, Fig. 6): the weights live on the
// magnetisation M at a fixed inverse temperature beta, so a chain samples
// W(M) exp(-beta E) and the histograms are over the V+1 bins (M + V)/2.
//
// Threshold table: per M bin 10 columns, column 5 (s == +1) + n for the flipped spin s
// and its n unequal neighbours; then E' - E = 8 - 4n and the bin moves by -s.  The
// sweep kernel is one thread per chain over the bit-packed lattice, in typewriter
// order, with the Ising random streams (group i >> 2, word i & 3) and the integer
// acceptance test (A = 2^32-1 or u < A); the histogram is incremented after every
// attempt.
#include <cmath>

#include "muca_internal.cuh"

namespace muca {
namespace {

__global__ void muma_thresholds_kernel(const double *lnw, uint32_t *thr, int n_bins, double beta)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bins * 10) return;
    const int b = t / 10, col = t % 10;
    const int s = col >= 5 ? 1 : -1, n = col % 5;
    const int bp = b - s;
    uint32_t A = 0u;
    if (bp >= 0 && bp < n_bins) {
        const double d = __dsub_rn(__dsub_rn(lnw[bp], lnw[b]), __dmul_rn(beta, (double)(8 - 4 * n)));
        if (d >= 0.0) {
            A = kAlways;
        } else {
            const double x = floor(ldexp(exp(d), 32));
            A = x >= 4294967295.0 ? kAlways : (uint32_t)x;
        }
    }
    thr[t] = A;
}

struct MumaArgs {
    uint32_t *lat;
    int32_t *E, *M;
    const uint32_t *thr;
    uint64_t *H;
    int32_t *E_rec, *M_rec;
    int L, p, p_pad, row_words, n_bins, n_sweeps, rec_stride;
    uint32_t sweep0, iteration, ctr3, key0;
};

template <bool HIST, bool SMEM_HIST>
__global__ void __launch_bounds__(128) muma_sweep_kernel(MumaArgs a)
{
    extern __shared__ uint32_t s_hist[];
    if (HIST && SMEM_HIST) {
        for (int i = threadIdx.x; i < a.n_bins; i += blockDim.x) s_hist[i] = 0u;
        __syncthreads();
    }
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.p) {
        const int L = a.L, V = L * L, RW = a.row_words;
        uint32_t *lat = a.lat + c;
        const size_t ps = (size_t)a.p_pad;
        auto bit = [&](int x, int y) -> uint32_t { return (lat[(size_t)(y * RW + (x >> 5)) * ps] >> (x & 31)) & 1u; };
        int E = a.E[c], M = a.M[c];
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t sweep = a.sweep0 + (uint32_t)sw;
            uint4 blk = make_uint4(0u, 0u, 0u, 0u);
            for (int i = 0; i < V; ++i) {
                if ((i & 3) == 0 || i == 0)
                    blk = philox4x32_10(make_uint4((uint32_t)i >> 2, sweep, a.iteration, a.ctr3), a.key0, (uint32_t)c);
                const uint32_t u = (i & 3) == 0 ? blk.x : (i & 3) == 1 ? blk.y : (i & 3) == 2 ? blk.z : blk.w;
                const int x = i % L, y = i / L;
                const uint32_t me = bit(x, y);
                const int unequal = (int)((bit(x == L - 1 ? 0 : x + 1, y) ^ me) + (bit(x == 0 ? L - 1 : x - 1, y) ^ me) +
                                          (bit(x, y == L - 1 ? 0 : y + 1) ^ me) + (bit(x, y == 0 ? L - 1 : y - 1) ^ me));
                const int b = (M + V) >> 1;
                const uint32_t A = a.thr[b * 10 + (me ? 5 : 0) + unequal];
                if (A == kAlways || u < A) {
                    lat[(size_t)(y * RW + (x >> 5)) * ps] ^= 1u << (x & 31);
                    E += 8 - 4 * unequal;
                    M -= me ? 2 : -2;
                }
                if (HIST) {
                    const int bn = (M + V) >> 1;
                    if (SMEM_HIST)
                        atomicAdd(&s_hist[bn], 1u);
                    else
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[bn]), 1ull);
                }
            }
            if (a.E_rec) a.E_rec[(size_t)sw * a.rec_stride + c] = E;
            if (a.M_rec) a.M_rec[(size_t)sw * a.rec_stride + c] = M;
        }
        a.E[c] = E;
        a.M[c] = M;
    }
    if (HIST && SMEM_HIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < a.n_bins; i += blockDim.x) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}

}  // namespace

int launch_muma_thresholds(muca_ctx *ctx)
{
    const int n = ctx->n_bins * 10;
    muma_thresholds_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_lnw, ctx->d_thr, ctx->n_bins,
                                                                    ctx->cfg.beta);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

int launch_muma_sweeps(muca_ctx *ctx, uint32_t phase, int n_sweeps, uint32_t sweep0, uint32_t iteration, bool hist,
                       int32_t *E_rec, int32_t *M_rec)
{
    MumaArgs a;
    a.lat = ctx->d_lat;
    a.E = ctx->d_E;
    a.M = ctx->d_M;
    a.thr = ctx->d_thr;
    a.H = ctx->d_H;
    a.E_rec = E_rec;
    a.M_rec = M_rec;
    a.L = ctx->L;
    a.p = ctx->p;
    a.p_pad = ctx->p_pad;
    a.row_words = ctx->row_words;
    a.n_bins = ctx->n_bins;
    a.n_sweeps = n_sweeps;
    a.rec_stride = ctx->p;
    a.sweep0 = sweep0;
    a.iteration = iteration;
    a.ctr3 = ((uint32_t)(ctx->seed >> 32) << 2) | phase;
    a.key0 = (uint32_t)ctx->seed;
    const int blocks = (ctx->p + 127) / 128;
    const size_t smem = (size_t)ctx->n_bins * sizeof(uint32_t);
    // block histograms are uint32: 128 chains x n_sweeps x V entries per launch
    const bool smem_hist = smem <= 48 * 1024 && 128.0 * n_sweeps * ctx->V < 4.0e9;
    if (!hist)
        muma_sweep_kernel<false, false><<<blocks, 128, 0, ctx->stream>>>(a);
    else if (smem_hist)
        muma_sweep_kernel<true, true><<<blocks, 128, smem, ctx->stream>>>(a);
    else
        muma_sweep_kernel<true, false><<<blocks, 128, 0, ctx->stream>>>(a);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

}  // namespace muca
