// Time-series reweighting (arXiv:1212.3975, Eq. 2; C_V of Sec. 5) on the device.
//
// The production records are already reduced to exact integer sums per energy bin
// (count n, sum |M|, sum M^2), so Eq. 2 becomes, per inverse temperature beta,
//     <X>_beta = sum_b w_b(beta) X_b / sum_b w_b(beta),
//     w_b(beta) = exp(lnOmega_b - beta E_b - shift_beta),  lnOmega_b = ln n_b - ln W_b,
// with X_b the per-bin means {1, E, E^2, |M|, M^2}.  The contraction uses centred
// columns {1, dE, dE^2, d|m|, d|m|^2, var_b(|m|)} around a reference bin, so that C
// and chi do not suffer from cancellation.
//
// MUCA_FP64 and MUCA_FP32 (muca_reweight and muca_reweight_noalloc): GB300 runs FP64 at
// a small fraction of its FP32 rate, so FP64 work is kept to what the precision needs.
//   1. prep: per bin, FP64 lnOmega_b and the means; a float copy of lnOmega_b and the
//      sampled range of bins (atomic min / max).
//   2. setup, one block per tile of 8 betas: reference bin k_T = argmax of
//      lnOmega_b - beta_T E_b (beta_T the tile's middle beta) found in FP32, the
//      window of bins whose weight can reach e^-100 of the largest for some beta of
//      the tile, and a per-beta shift c_t (the negated maximum of the exponent).
//      Any shift common to all bins of a beta cancels in <X> = sum w X / sum w, so an
//      approximate (FP32) maximum is enough: it only keeps the exponents in range.
//   3. scan: the tiles' bin windows are cut into chunks (at most 32 per tile) and
//      numbered, so that
//   4. sums: a persistent grid fills every SM with (tile, chunk) items, each writing
//      FP64 partial sums of the six centred columns for the tile's betas;
//   5. combine: per beta, the partial sums in chunk order (deterministic), then the
//      observables.
// The exponent of bin b at beta_t is a = G_b + c_t - (beta_t - beta_T)(E_b - E_kT) with
// G_b = lnOmega_b - lnOmega_kT - beta_T (E_b - E_kT) formed in FP64 once per (tile,
// bin).  MUCA_FP64 evaluates a and exp(a) in FP64 and skips a < -100.  MUCA_FP32
// evaluates a as an unevaluated sum of two floats (G_b and beta_t - beta_T split into
// high and low floats, the product by the exact integer E_b - E_kT with its FMA-exact
// error, error-free additions) and w = exp2(a_hi) (1 + a_lo ln 2): at a beta far from
// the sampled range the observables come from bins of relative weight ~1e-12, i.e.
// |a| ~ 40 (log2 units), where a single float exponent would carry a relative error of
// ~|a| 2^-24 into those weights.  Weights and column sums are FP32 within a thread and
// a warp, FP64 across warps and chunks.
//
// MUCA_BF16 (muca_reweight only): one block of 8 warps per tile of 16 betas (the M
// dimension of mma.m16n8k16), an FP64 prologue per tile (reference bin, window,
// shifts), table entries and columns split into three BF16 terms and multiplied on the
// tensor cores with FP32 accumulation flushed to FP64 per chunk of 16 bins.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "muca_internal.cuh"

namespace muca {
namespace {

constexpr double kCut = -100.0;  // ln of the smallest relative term kept
constexpr double kLog2e = 1.4426950408889634;

struct BinData {
    double *lnO;  // ln n_b - lnW_b, -inf where n_b = 0
    double *E;    // bin energy
    double *x1;   // mean |M| in the bin
    double *x2;   // mean M^2 in the bin
    double *v;    // x2 - x1^2 (within-bin variance of |M|)
};

__global__ void prep_kernel(const uint64_t *samples, const double *lnw, BinData d, int model, int V,
                            int n_bins)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    const uint64_t n = samples[b];
    d.E[b] = model == MUCA_ISING ? (double)(4 * b - 2 * V) : (double)(b - 2 * V);
    if (n == 0) {
        d.lnO[b] = -INFINITY;
        d.x1[b] = d.x2[b] = d.v[b] = 0.0;
        return;
    }
    const double nd = (double)n;
    d.lnO[b] = __dsub_rn(log(nd), lnw[b]);
    const double x1 = __ddiv_rn((double)samples[n_bins + b], nd);
    const double x2 = __ddiv_rn((double)samples[2 * n_bins + b], nd);
    d.x1[b] = x1;
    d.x2[b] = x2;
    d.v[b] = x2 - x1 * x1;
}

// block-wide max with the smallest index among ties
__device__ void block_argmax(double &val, int &idx, double *s_val, int *s_idx)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, val, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    __syncthreads();
    if (lane == 0) { s_val[warp] = val; s_idx[warp] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (s_val[w] > val || (s_val[w] == val && s_idx[w] < idx)) { val = s_val[w]; idx = s_idx[w]; }
        s_val[0] = val;
        s_idx[0] = idx;
    }
    __syncthreads();
    val = s_val[0];
    idx = s_idx[0];
    __syncthreads();
}

struct Observables {
    double *e, *C, *absm, *chi;  // [n_beta] each (device)
};

__device__ void write_obs(Observables o, int j, double beta, double Eref, double x1ref, double S0, double S1,
                          double S2, double S3, double S4, double S5, int V, double mnorm)
{
    const double m1 = S1 / S0;
    const double var = S2 / S0 - m1 * m1;
    const double dm = S3 / S0;
    const double mvar = S5 / S0 + S4 / S0 - dm * dm;
    o.e[j] = (Eref + m1) / V;
    o.C[j] = beta * beta * var / V;
    o.absm[j] = (x1ref + dm) / mnorm;
    o.chi[j] = beta * V * mvar / (mnorm * mnorm);
}

// ------------------------------ BF16 prologue ----------------------------------
// FP64 shift of every beta of a tile, one warp per beta at a time: c_t = (lnO_T - beta_t
// E_T) - max_b (lnO_b - beta_t E_b) over the window, in log2 units, and beta_t - beta_T.
// The maximum is exact, so the order of the reduction does not change it.
template <int TILE>
__device__ void tile_shifts(const BinData &d, const double *betas, int j0, int nt, int lo, int hi, double lnOT,
                            double ET, double betaT, float *s_c, float *s_db)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = warp; t < TILE; t += nw) {
        if (t >= nt) {
            if (lane == 0) {
                s_c[t] = -1e30f;
                s_db[t] = 0.f;
            }
            continue;
        }
        const double beta = betas[j0 + t];
        double m = -INFINITY;
#pragma unroll 4
        for (int b = lo + lane; b <= hi; b += 32) {
            const double l = d.lnO[b];
            if (l != -INFINITY) m = fmax(m, __dsub_rn(l, __dmul_rn(beta, d.E[b])));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            s_c[t] = (float)(((lnOT - beta * ET) - m) * kLog2e);
            s_db[t] = (float)((beta - betaT) * kLog2e);
        }
    }
    __syncthreads();
}

// ------------------------------ BF16 tensor cores ------------------------------
// Tile of 16 betas = the M dimension of mma.m16n8k16; 16 bins per K step; the 6
// centred observable columns (padded to 8) are N.  Table entries and columns are
// split into three BF16 terms, x = x_h + x_m + x_l (residual below 2^-26 |x|), and
// multiplied as the six products of order <= 2 (hh, hm, mh, hl, lh, mm; the dropped
// ones are below 2^-24 relative); each chunk's six products are accumulated by the
// tensor cores in FP32 from zero (their FP32 accumulation need not round to nearest)
// and added to FP64 registers.  The FP64 prologue (reference bin, window, per-beta shifts) is the one of
// the FP32 form.
template <int TILE>
__device__ void tile_prologue(const BinData &d, const double *betas, int n_beta, int n_bins, int j0, int nt,
                              double *s_val, int *s_idx, float *s_c, float *s_db, double &lnOT, double &ET,
                              double &x1T, double &betaT, int &lo, int &hi)
{
    betaT = betas[j0 + nt / 2];
    double best = -INFINITY;
    int kT = n_bins;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double a = __dsub_rn(l, __dmul_rn(betaT, d.E[b]));
        if (a > best || (a == best && b < kT)) { best = a; kT = b; }
    }
    block_argmax(best, kT, s_val, s_idx);
    lnOT = d.lnO[kT];
    ET = d.E[kT];
    x1T = d.x1[kT];
    double dbmax = 0.0;
    for (int t = 0; t < nt; ++t) dbmax = fmax(dbmax, fabs(betas[j0 + t] - betaT));
    lo = n_bins;
    hi = -1;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double dE = d.E[b] - ET;
        const double G = (l - lnOT) - betaT * dE;
        if (G + dbmax * fabs(dE) >= kCut) { lo = min(lo, b); hi = max(hi, b); }
    }
    double v1 = -(double)lo;
    int i1 = 0;
    block_argmax(v1, i1, s_val, s_idx);
    lo = (int)(-v1);
    double v2 = (double)hi;
    int i2 = 0;
    block_argmax(v2, i2, s_val, s_idx);
    hi = (int)v2;
    tile_shifts<TILE>(d, betas, j0, nt, lo, hi, lnOT, ET, betaT, s_c, s_db);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float first, float second)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(first, second);  // .x (low half) = first
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kBf16Warps = 8;  // warps per tile of 16 betas (each takes every 8th chunk of 16 bins)

__global__ void __launch_bounds__(32 * kBf16Warps) reweight_bf16_kernel(BinData d, const double *betas, int n_beta,
                                                                        int n_bins, int V, double mnorm, Observables o)
{
    constexpr int TILE = 16, NW = kBf16Warps;
    __shared__ double s_val[32 * 6];
    __shared__ int s_idx[32];
    __shared__ float s_c[TILE], s_db[TILE];
    __shared__ double s_red[NW][TILE][8];
    const int j0 = blockIdx.x * TILE;
    const int nt = min(TILE, n_beta - j0);
    double lnOT, ET, x1T, betaT;
    int lo, hi;
    tile_prologue<TILE>(d, betas, n_beta, n_bins, j0, nt, s_val, s_idx, s_c, s_db, lnOT, ET, x1T, betaT, lo, hi);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;          // fragment coordinates
    const float c0 = s_c[g], db0 = s_db[g], c1 = s_c[g + 8], db1 = s_db[g + 8];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    double accd[4] = {0.0, 0.0, 0.0, 0.0};
    for (int base = lo + 16 * warp; base <= hi; base += 16 * NW) {
        // each lane prepares one bin of the chunk (lanes 16..31 repeat lanes 0..15)
        const int b = base + (lane & 15);
        float G = -1e30f, dE = 0.f, dx = 0.f, vb = 0.f;
        if (b <= hi) {
            const double l = d.lnO[b];
            if (l != -INFINITY) {
                const double dEd = d.E[b] - ET;
                G = (float)(((l - lnOT) - betaT * dEd) * kLog2e);
                dE = (float)dEd;
                dx = (float)(d.x1[b] - x1T);
                vb = (float)d.v[b];
            }
        }
        float x[2][4], col[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 2 * t4 + (q & 1) + 8 * (q >> 1);  // bin of the chunk held by this thread
            const float Gq = __shfl_sync(0xffffffffu, G, k);
            const float dEq = __shfl_sync(0xffffffffu, dE, k);
            const float dxq = __shfl_sync(0xffffffffu, dx, k);
            const float vq = __shfl_sync(0xffffffffu, vb, k);
            x[0][q] = exp2f(fmaf(-db0, dEq, Gq + c0));
            x[1][q] = exp2f(fmaf(-db1, dEq, Gq + c1));
            const float cv = g == 0 ? 1.f : g == 1 ? dEq : g == 2 ? dEq * dEq : g == 3 ? dxq : g == 4 ? dxq * dxq
                                                                                 : g == 5 ? vq : 0.f;
            col[q] = Gq > -1e29f ? cv : 0.f;
        }
        uint32_t ah[4], am[4], al[4], bh[2], bm[2], bl[2];
        // three-term split of a pair of FP32 values into packed BF16 registers
        auto split3 = [](float v0, float v1, uint32_t &h, uint32_t &m, uint32_t &l) {
            const float h0 = bf16_round(v0), h1 = bf16_round(v1);
            const float m0 = bf16_round(v0 - h0), m1 = bf16_round(v1 - h1);
            h = pack_bf16x2(h0, h1);
            m = pack_bf16x2(m0, m1);
            l = pack_bf16x2((v0 - h0) - m0, (v1 - h1) - m1);
        };
        // A registers: {row g, bins q0,q1}, {row g+8, q0,q1}, {row g, q2,q3}, {row g+8, q2,q3}
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = r & 1, qp = (r >> 1) * 2;
            split3(x[row][qp], x[row][qp + 1], ah[r], am[r], al[r]);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) split3(col[2 * r], col[2 * r + 1], bh[r], bm[r], bl[r]);
        // smallest products first
        mma_bf16_16816(acc, am, bm);
        mma_bf16_16816(acc, ah, bl);
        mma_bf16_16816(acc, al, bh);
        mma_bf16_16816(acc, ah, bm);
        mma_bf16_16816(acc, am, bh);
        mma_bf16_16816(acc, ah, bh);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            accd[i] += (double)acc[i];
            acc[i] = 0.f;
        }
    }
    // accumulators: (row g, cols 2t4, 2t4+1), (row g+8, cols 2t4, 2t4+1)
    s_red[warp][g][2 * t4] = accd[0];
    s_red[warp][g][2 * t4 + 1] = accd[1];
    s_red[warp][g + 8][2 * t4] = accd[2];
    s_red[warp][g + 8][2 * t4 + 1] = accd[3];
    __syncthreads();
    if ((int)threadIdx.x < nt) {
        const int t = threadIdx.x;
        double S[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < NW; ++w)
            for (int k = 0; k < 6; ++k) S[k] += s_red[w][t][k];
        write_obs(o, j0 + t, betas[j0 + t], ET, x1T, S[0], S[1], S[2], S[3], S[4], S[5], V, mnorm);
    }
}

// ============================ tiled context path =================================
constexpr int kRwMinChunk = 256;   // bins per chunk at least
constexpr double kLn2 = 0.6931471805599453;

struct TileParams {
    int kT, lo, ch, nch;           // reference bin, first bin of the window, chunk size, chunks
    double lnOT, ET, x1T, betaT;
};
static_assert(sizeof(TileParams) == kRwTileParamsBytes, "tile parameter layout");

struct RwScratch {
    BinData d;
    float *lnOf;                   // float copy of lnOmega (-inf where unsampled)
    int *range;                    // [2]: lowest and highest sampled bin
    TileParams *tiles;             // [n_tiles]
    double *c;                     // [n_beta] per-beta shift (ln units)
    int *off;                      // [n_tiles + 1] item offsets of the tiles
    double *part;                  // [n_tiles * kRwMaxChunks][kRwTile][6] partial sums
};

__device__ __forceinline__ double bin_energy(int model, int V, int b)
{
    return model == MUCA_ISING ? (double)(4 * b - 2 * V) : (double)(b - 2 * V);
}

__global__ void rw_prep_kernel(const uint64_t *samples, const double *lnw, RwScratch r, int model, int V,
                               int n_bins)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    const uint64_t n = samples[b];
    r.d.E[b] = bin_energy(model, V, b);
    if (n == 0) {
        r.d.lnO[b] = -INFINITY;
        r.lnOf[b] = -INFINITY;
        r.d.x1[b] = r.d.x2[b] = r.d.v[b] = 0.0;
        return;
    }
    const double nd = (double)n;
    const double l = __dsub_rn(log(nd), lnw[b]);
    r.d.lnO[b] = l;
    r.lnOf[b] = (float)l;
    const double x1 = __ddiv_rn((double)samples[n_bins + b], nd);
    const double x2 = __ddiv_rn((double)samples[2 * n_bins + b], nd);
    r.d.x1[b] = x1;
    r.d.x2[b] = x2;
    r.d.v[b] = x2 - x1 * x1;
    atomicMin(&r.range[0], b);
    atomicMax(&r.range[1], b);
}

__device__ __forceinline__ void warp_argmax(float &v, int &i)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

// One block (256 threads) per tile: reference bin, window, chunks and per-beta shifts.
__global__ void __launch_bounds__(256) rw_setup_kernel(RwScratch r, const double *betas, int n_beta, int model, int V)
{
    __shared__ float s_v[8];
    __shared__ int s_i[8], s_lo[8], s_hi[8];
    const int T = blockIdx.x, j0 = T * kRwTile, nt = min(kRwTile, n_beta - j0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lo_s = r.range[0], hi_s = r.range[1];
    const double betaT = betas[j0 + nt / 2];
    const float bTf = (float)betaT;
    // approximate reference bin (FP32 scan of the sampled range)
    float best = -INFINITY;
    int kT = max(0, hi_s);  // replaced by a sampled bin whenever there is one
    for (int b = lo_s + (int)threadIdx.x; b <= hi_s; b += blockDim.x) {
        const float l = r.lnOf[b];
        if (l == -INFINITY) continue;
        const float a = l - bTf * (float)bin_energy(model, V, b);
        if (a > best) { best = a; kT = b; }
    }
    warp_argmax(best, kT);
    if (lane == 0) { s_v[warp] = best; s_i[warp] = kT; }
    __syncthreads();
    if (threadIdx.x < 32) {
        best = lane < 8 ? s_v[lane] : -INFINITY;
        kT = lane < 8 ? s_i[lane] : max(0, hi_s);
        warp_argmax(best, kT);
        if (lane == 0) { s_v[0] = best; s_i[0] = kT; }
    }
    __syncthreads();
    kT = s_i[0];
    const float lTf = r.lnOf[kT];
    const double ETd = bin_energy(model, V, kT);
    const float ETf = (float)ETd;
    float dbmax = 0.f;
    for (int t = 0; t < nt; ++t) dbmax = fmaxf(dbmax, fabsf((float)(betas[j0 + t] - betaT)));
    // window: bins that can reach e^-100 of the largest weight for some beta of the tile
    // (approximate exponents, 2 units of margin)
    int lo = hi_s + 1, hi = lo_s - 1;
    for (int b = lo_s + (int)threadIdx.x; b <= hi_s; b += blockDim.x) {
        const float l = r.lnOf[b];
        if (l == -INFINITY) continue;
        const float dE = (float)bin_energy(model, V, b) - ETf;
        if ((l - lTf) - bTf * dE + dbmax * fabsf(dE) >= (float)kCut - 2.f) { lo = min(lo, b); hi = max(hi, b); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    lo = s_lo[0];
    hi = s_hi[0];
    for (int w = 1; w < 8; ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
    if (lo > hi) {  // no sampled bin at all: an empty window
        lo = 0;
        hi = -1;
    }
    // per-beta shift: minus the approximate maximum of the exponent over the window
    for (int t = warp; t < nt; t += 8) {
        const float db = (float)(betas[j0 + t] - betaT);
        float m = -INFINITY;
        for (int b = lo + lane; b <= hi; b += 32) {
            const float l = r.lnOf[b];
            if (l == -INFINITY) continue;
            const float dE = (float)bin_energy(model, V, b) - ETf;
            m = fmaxf(m, (l - lTf) - bTf * dE - db * dE);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) r.c[j0 + t] = -(double)m;
    }
    if (threadIdx.x == 0) {
        const int width = max(0, hi - lo + 1);
        int ch = max(kRwMinChunk, (width + kRwMaxChunks - 1) / kRwMaxChunks);
        ch = (ch + 31) & ~31;
        TileParams tp;
        tp.kT = kT;
        tp.lo = lo;
        tp.ch = ch;
        tp.nch = (width + ch - 1) / ch;
        tp.lnOT = r.d.lnO[kT];
        tp.ET = ETd;
        tp.x1T = r.d.x1[kT];
        tp.betaT = betaT;
        r.tiles[T] = tp;
    }
}

// Exclusive prefix of the tiles' chunk counts (one block).
__global__ void __launch_bounds__(1024) rw_scan_kernel(RwScratch r, int n_tiles)
{
    __shared__ int s_part[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n_tiles; base += blockDim.x) {
        const int T = base + (int)threadIdx.x;
        const int v = T < n_tiles ? r.tiles[T].nch : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_part[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_part[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_part[warp - 1] : 0) + s_carry;
        if (T < n_tiles) r.off[T] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) r.off[n_tiles] = s_carry;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Persistent grid over the (tile, chunk) items.  FP64: exponents and weights in FP64;
// FP32: compensated exponents, weights and sums in FP32 per thread, FP64 across warps.
template <bool FP64>
__global__ void __launch_bounds__(256) rw_sums_kernel(RwScratch r, const double *betas, int n_beta, int n_tiles)
{
    using acc_t = typename std::conditional<FP64, double, float>::type;
    __shared__ double s_red[8][kRwTile][6];
    __shared__ int s_T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = r.off[n_tiles];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        __syncthreads();  // s_red and s_T of the previous item are consumed
        if (threadIdx.x == 0) {
            int a = 0, b = n_tiles - 1;  // last tile with off <= item
            while (a < b) {
                const int m = (a + b + 1) >> 1;
                if (r.off[m] <= item) a = m; else b = m - 1;
            }
            s_T = a;
        }
        __syncthreads();
        const int T = s_T;
        const TileParams tp = r.tiles[T];
        const int chunk = item - r.off[T];
        const int j0 = T * kRwTile, nt = min(kRwTile, n_beta - j0);
        const int b0 = tp.lo + chunk * tp.ch;
        const int b1 = min(b0 + tp.ch, tp.lo + tp.nch * tp.ch);
        // per-beta constants of the tile
        double cd[kRwTile], dbd[kRwTile];
        float ch_[kRwTile], dbh[kRwTile], dbl[kRwTile];
#pragma unroll
        for (int t = 0; t < kRwTile; ++t) {
            const bool ok = t < nt;
            cd[t] = ok ? r.c[j0 + t] : -1e300;
            dbd[t] = ok ? betas[j0 + t] - tp.betaT : 0.0;
            const double dbl2 = dbd[t] * kLog2e;
            dbh[t] = (float)dbl2;
            dbl[t] = (float)(dbl2 - (double)dbh[t]);
            ch_[t] = ok ? (float)(cd[t] * kLog2e) : -1e30f;
        }
        acc_t acc[kRwTile][6];
#pragma unroll
        for (int t = 0; t < kRwTile; ++t)
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[t][k] = 0;
        for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
            const double l = r.d.lnO[b];
            if (l == -INFINITY) continue;
            const double dEd = r.d.E[b] - tp.ET;
            const double G = __dsub_rn(__dsub_rn(l, tp.lnOT), __dmul_rn(tp.betaT, dEd));
            const double dx = r.d.x1[b] - tp.x1T, vb = r.d.v[b];
            if (FP64) {
#pragma unroll
                for (int t = 0; t < kRwTile; ++t) {
                    const double a = __fma_rn(-dbd[t], dEd, G + cd[t]);
                    if (a < kCut) continue;
                    const double w = exp(a);
                    acc[t][0] += (acc_t)w;
                    acc[t][1] += (acc_t)(w * dEd);
                    acc[t][2] += (acc_t)(w * dEd * dEd);
                    acc[t][3] += (acc_t)(w * dx);
                    acc[t][4] += (acc_t)(w * dx * dx);
                    acc[t][5] += (acc_t)(w * vb);
                }
            } else {
                const double G2 = G * kLog2e;
                const float Gh = (float)G2, Gl = (float)(G2 - (double)Gh);
                const float dE = (float)dEd, dxf = (float)dx, vf = (float)vb;
                const float dE2 = dE * dE, dx2 = dxf * dxf;
#pragma unroll
                for (int t = 0; t < kRwTile; ++t) {
                    // a = (Gh + Gl) + c - (dbh + dbl) dE as a float pair
                    const float p = __fmul_rn(dbh[t], dE);
                    const float pe = __fmaf_rn(dbh[t], dE, -p);
                    const float q = __fmul_rn(dbl[t], dE);
                    float s1, e1, s2, e2;
                    two_sum(Gh, ch_[t], s1, e1);
                    two_sum(s1, -p, s2, e2);
                    const float lo = __fsub_rn(__fadd_rn(__fadd_rn(e1, e2), Gl), __fadd_rn(pe, q));
                    const float ah = __fadd_rn(s2, lo);
                    const float al = __fsub_rn(lo, __fsub_rn(ah, s2));
                    const float w0 = exp2f(ah);
                    const float w = __fmaf_rn(w0, al * (float)kLn2, w0);
                    acc[t][0] += (acc_t)w;
                    acc[t][1] = __fmaf_rn(w, dE, acc[t][1]);
                    acc[t][2] = __fmaf_rn(w, dE2, acc[t][2]);
                    acc[t][3] = __fmaf_rn(w, dxf, acc[t][3]);
                    acc[t][4] = __fmaf_rn(w, dx2, acc[t][4]);
                    acc[t][5] = __fmaf_rn(w, vf, acc[t][5]);
                }
            }
        }
        // reduce: within the warp in the accumulation type, across warps in FP64
#pragma unroll
        for (int t = 0; t < kRwTile; ++t)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                acc_t x = acc[t][k];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) s_red[warp][t][k] = (double)x;
            }
        __syncthreads();
        if ((int)threadIdx.x < kRwTile * 6) {
            const int t = threadIdx.x / 6, k = threadIdx.x % 6;
            double x = 0.0;
            for (int w = 0; w < 8; ++w) x += s_red[w][t][k];
            r.part[((size_t)item * kRwTile + t) * 6 + k] = x;
        }
    }
}

// Per beta: partial sums of its tile in chunk order, then the observables.
__global__ void rw_combine_kernel(RwScratch r, const double *betas, int n_beta, int V, double mnorm, Observables o)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_beta) return;
    const int T = j / kRwTile, t = j % kRwTile;
    const TileParams tp = r.tiles[T];
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int i = r.off[T]; i < r.off[T + 1]; ++i)
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] += r.part[((size_t)i * kRwTile + t) * 6 + k];
    write_obs(o, j, betas[j], tp.ET, tp.x1T, S[0], S[1], S[2], S[3], S[4], S[5], V, mnorm);
}

}  // namespace

namespace {

// setup, scan, sums and combine of one batch of betas (the per-bin arrays of `r` are
// prepared); `n_sm` sizes the persistent grid of the sums
cudaError_t launch_tiles(const RwScratch &r, const double *d_betas, int n_beta, int precision, int model, int V,
                         double mnorm, const Observables &o, int n_sm, cudaStream_t st)
{
    const int n_tiles = (n_beta + kRwTile - 1) / kRwTile;
    rw_setup_kernel<<<n_tiles, 256, 0, st>>>(r, d_betas, n_beta, model, V);
    rw_scan_kernel<<<1, 1024, 0, st>>>(r, n_tiles);
    const int grid = std::max(1, std::min(n_tiles * kRwMaxChunks, 4 * n_sm));
    if (precision == MUCA_FP64)
        rw_sums_kernel<true><<<grid, 256, 0, st>>>(r, d_betas, n_beta, n_tiles);
    else
        rw_sums_kernel<false><<<grid, 256, 0, st>>>(r, d_betas, n_beta, n_tiles);
    rw_combine_kernel<<<(n_beta + 127) / 128, 128, 0, st>>>(r, d_betas, n_beta, V, mnorm, o);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(4);
    return e;
}

size_t align256(size_t bytes) { return rw_align256(bytes); }
size_t tile_part_bytes(int n_beta) { return rw_tile_part_bytes((size_t)n_beta); }

RwScratch carve(void *bins, size_t nb, void *tiles, int n_beta)
{
    RwScratch r;
    char *pb = reinterpret_cast<char *>(bins);
    double *base = reinterpret_cast<double *>(pb);
    r.d = BinData{base, base + nb, base + 2 * nb, base + 3 * nb, base + 4 * nb};
    r.lnOf = reinterpret_cast<float *>(pb + align256(5 * nb * sizeof(double)));
    r.range = reinterpret_cast<int *>(r.lnOf + nb);
    const size_t n_tiles = (size_t)(n_beta + kRwTile - 1) / kRwTile;
    char *pt = reinterpret_cast<char *>(tiles);
    r.tiles = reinterpret_cast<TileParams *>(pt);
    pt += align256(sizeof(TileParams) * n_tiles);
    r.c = reinterpret_cast<double *>(pt);
    pt += align256(sizeof(double) * n_beta);
    r.off = reinterpret_cast<int *>(pt);
    pt += align256(sizeof(int) * (n_tiles + 1));
    r.part = reinterpret_cast<double *>(pt);
    return r;
}

// per-bin preparation, including the sampled range (reset first)
cudaError_t launch_prep(const RwScratch &r, const uint64_t *samples, const double *lnw, int model, int V, int nb,
                        cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(r.range, 0x7F, sizeof(int), st);  // lowest bin starts at 0x7F7F7F7F
    if (e == cudaSuccess) e = cudaMemsetAsync(r.range + 1, 0xFF, sizeof(int), st);  // highest at -1
    if (e != cudaSuccess) return e;
    rw_prep_kernel<<<(nb + 255) / 256, 256, 0, st>>>(samples, lnw, r, model, V, nb);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(1);
    return e;
}

}  // namespace

// The tiled kernels with every buffer supplied by the caller: `scratch` of
// kNoallocScratchBytes (n_bins <= kNoallocMaxBins), production sums [3][n_bins],
// weights [n_bins], betas [n_beta] and the output [4][n_beta] (all device memory).
// Betas are taken in passes of at most kNoallocBetasPerPass, so the scratch does not
// depend on n_beta.  Launches on `st`; allocates nothing.
cudaError_t launch_reweight_buffers(double *scratch, const uint64_t *samples, const double *lnw, int model, int L,
                                    int q, const double *d_betas, int n_beta, int precision, double *d_out,
                                    int n_sm, cudaStream_t st)
{
    const int V = L * L;
    const int nb = n_bins_of(model, L);
    char *base = reinterpret_cast<char *>(scratch);
    RwScratch r = carve(base, nb, base + rw_bin_part_bytes(kNoallocMaxBins), kNoallocBetasPerPass);
    cudaError_t e = launch_prep(r, samples, lnw, model, V, nb, st);
    if (e != cudaSuccess) return e;
    const double mnorm = model == MUCA_ISING ? (double)V : (double)(q - 1) * V;
    for (int j0 = 0; j0 < n_beta; j0 += kNoallocBetasPerPass) {
        const int nj = std::min(kNoallocBetasPerPass, n_beta - j0);
        Observables o{d_out + j0, d_out + n_beta + j0, d_out + 2 * (size_t)n_beta + j0,
                      d_out + 3 * (size_t)n_beta + j0};
        e = launch_tiles(r, d_betas + j0, nj, precision, model, V, mnorm, o, n_sm, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int launch_reweight(muca_ctx *ctx, const double *d_betas, int n_beta, int precision, double *d_out)
{
    const size_t nb = ctx->n_bins;
    double *base = reinterpret_cast<double *>(ctx->d_rw);
    BinData d{base, base + nb, base + 2 * nb, base + 3 * nb, base + 4 * nb};
    Observables o{d_out, d_out + n_beta, d_out + 2 * n_beta, d_out + 3 * n_beta};
    const double mnorm = ctx->model == MUCA_ISING ? (double)ctx->V : (double)(ctx->q - 1) * ctx->V;
    if (precision == MUCA_BF16) {
        prep_kernel<<<(ctx->n_bins + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_samples, ctx->d_lnw_prod, d,
                                                                       ctx->model, ctx->V, ctx->n_bins);
        MUCA_CUDA_TRY(cudaGetLastError());
        const int tiles = (n_beta + 15) / 16;
        reweight_bf16_kernel<<<tiles, 32 * kBf16Warps, 0, ctx->stream>>>(d, d_betas, n_beta, ctx->n_bins, ctx->V,
                                                                         mnorm, o);
        MUCA_CUDA_TRY(cudaGetLastError());
        note_launches(2);
        return MUCA_OK;
    }
    if (precision != MUCA_FP64 && precision != MUCA_FP32)
        return fail(MUCA_ERR_ARG, "precision must be MUCA_FP64, MUCA_FP32 or MUCA_BF16");
    // per-call scratch: tile parameters, shifts, item offsets, partial sums
    const size_t need = tile_part_bytes(n_beta);
    if (ctx->rwtile_bytes < need) {
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (ctx->d_rwtile) cudaFree(ctx->d_rwtile);
        ctx->d_rwtile = nullptr;
        ctx->rwtile_bytes = 0;
        if (cudaMalloc(&ctx->d_rwtile, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(MUCA_ERR_OOM, "reweighting scratch");
        }
        ctx->rwtile_bytes = need;
    }
    const RwScratch r = carve(ctx->d_rw, nb, ctx->d_rwtile, n_beta);
    MUCA_CUDA_TRY(launch_prep(r, ctx->d_samples, ctx->d_lnw_prod, ctx->model, ctx->V, ctx->n_bins, ctx->stream));
    MUCA_CUDA_TRY(launch_tiles(r, d_betas, n_beta, precision, ctx->model, ctx->V, mnorm, o, ctx->n_sm, ctx->stream));
    return MUCA_OK;
}

}  // namespace muca
