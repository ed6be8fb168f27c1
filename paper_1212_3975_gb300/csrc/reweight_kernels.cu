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
// ~|a| 2^-24 into those weights.  Column sums are float pairs (an error-free addition
// per term) within a thread and a warp, FP64 across warps and chunks.
//
// MUCA_BF16 (muca_reweight only): one block of 8 warps per tile of 16 betas (the M
// dimension of mma.m16n8k16), an FP64 prologue per tile (reference bin, window,
// shifts), table entries and columns split into three BF16 terms and multiplied on the
// tensor cores with FP32 accumulation flushed to FP64 per chunk of 16 bins.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

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
    float lTh, lTl, x1Th, x1Tl;    // lnOmega and mean |M| of the reference bin as float pairs
    float bTh, bTl;                // beta_T as a float pair
};
static_assert(sizeof(TileParams) == kRwTileParamsBytes, "tile parameter layout");

struct RwScratch {
    BinData d;
    float *lnOf;                   // float copy of lnOmega (-inf where unsampled): high part
    float *lnOl;                   //   and low part of lnOmega as a float pair
    float *x1h, *x1l;              // mean |M| as a float pair
    float *vf;                     // within-bin variance of |M| (float)
    int2 *blkrange;                // [ceil(n_bins / 256)] lowest / highest sampled bin of each prep block
    int nblk;
    TileParams *tiles;             // [n_tiles]
    double *c;                     // [n_beta] per-beta shift (ln units)
    float4 *bc;                    // [n_beta] float constants: (beta - beta_T) log2 e as a pair, c log2 e,
                                   //   and the beta's reference energy E_ref - E_T (an exact integer)
    double *xref;                  // [n_beta] mean |M| of the beta's reference bin
    float2 *xrf;                   //   and as a float pair
    int *off;                      // [n_tiles + 1] item offsets of the tiles
    unsigned *cnt0;                // completion counter of the setup kernel (zero between calls)
    unsigned *cnt;                 // [n_tiles] completion counters of the tiles (zeroed by the setup)
    int *item_tile;                // [n_tiles * kRwMaxChunks] tile of every item
    double *part;                  // [n_tiles * kRwMaxChunks][kRwTile][6] partial sums
};

__device__ __forceinline__ double bin_energy(int model, int V, int b)
{
    return model == MUCA_ISING ? (double)(4 * b - 2 * V) : (double)(b - 2 * V);
}

// Per bin: FP64 lnOmega and means, the float copy, and the block's sampled range.
__global__ void __launch_bounds__(256) rw_prep_kernel(const uint64_t *samples, const double *lnw, RwScratch r,
                                                      int model, int V, int n_bins)
{
    __shared__ int s_lo[8], s_hi[8];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    int lo = 0x7FFFFFFF, hi = -1;
    if (b < n_bins) {
        const uint64_t n = samples[b];
        r.d.E[b] = bin_energy(model, V, b);
        if (n == 0) {
            r.d.lnO[b] = -INFINITY;
            r.lnOf[b] = -INFINITY;
            r.lnOl[b] = r.x1h[b] = r.x1l[b] = r.vf[b] = 0.f;
            r.d.x1[b] = r.d.x2[b] = r.d.v[b] = 0.0;
        } else {
            const double nd = (double)n;
            const double l = __dsub_rn(log(nd), lnw[b]);
            r.d.lnO[b] = l;
            const float lh = (float)l;
            r.lnOf[b] = lh;
            r.lnOl[b] = (float)(l - (double)lh);
            const double x1 = __ddiv_rn((double)samples[n_bins + b], nd);
            const double x2 = __ddiv_rn((double)samples[2 * n_bins + b], nd);
            r.d.x1[b] = x1;
            r.d.x2[b] = x2;
            r.d.v[b] = x2 - x1 * x1;
            const float xh = (float)x1;
            r.x1h[b] = xh;
            r.x1l[b] = (float)(x1 - (double)xh);
            r.vf[b] = (float)(x2 - x1 * x1);
            lo = hi = b;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
        r.blkrange[blockIdx.x] = make_int2(lo, hi);
    }
}

__device__ __forceinline__ void warp_argmax(float &v, int &i)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

// Exclusive prefix of the tiles' chunk counts, by one block of 256 threads (the last
// setup block); tiles without a sampled bin get NaN observables here.
__device__ void scan_tiles(RwScratch &r, int n_tiles, int n_beta, Observables o)
{
    __shared__ int s_part[8];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n_tiles; base += blockDim.x) {
        const int T = base + (int)threadIdx.x;
        const int v = T < n_tiles ? __ldcg(&r.tiles[T].nch) : 0;
        if (T < n_tiles && v == 0)
            for (int j = T * kRwTile; j < min(n_beta, (T + 1) * kRwTile); ++j)
                o.e[j] = o.C[j] = o.absm[j] = o.chi[j] = NAN;
        int x = v;
        for (int k = 1; k < 32; k <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, k);
            if (lane >= k) x += y;
        }
        if (lane == 31) s_part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < 8 ? s_part[lane] : 0;
            for (int k = 1; k < 8; k <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, k);
                if (lane >= k) w += y;
            }
            if (lane < 8) s_part[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_part[warp - 1] : 0) + s_carry;
        if (T < n_tiles) {
            r.off[T] = incl - v;
            for (int i = incl - v; i < incl; ++i) r.item_tile[i] = T;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) r.off[n_tiles] = s_carry;
}

// One block (256 threads) per tile: reference bin, window, chunks and per-beta shifts,
// in two passes over the sampled bins; the block that finishes last numbers the chunks
// of all tiles.
__global__ void __launch_bounds__(256) rw_setup_kernel(RwScratch r, const double *betas, int n_beta, int model, int V,
                                                       Observables o)
{
    __shared__ float s_v[8], s_m[8][kRwTile];
    __shared__ int s_i[8], s_lo[8], s_hi[8], s_mi[8][kRwTile];
    __shared__ int s_last;
    const int T = blockIdx.x, j0 = T * kRwTile, nt = min(kRwTile, n_beta - j0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) r.cnt[T] = 0u;  // the sums kernel counts this tile's chunks from zero
    // sampled range of the bins, from the preparation blocks' ranges
    int lo_s = 0x7FFFFFFF, hi_s = -1;
    for (int i = threadIdx.x; i < r.nblk; i += blockDim.x) {
        const int2 br = r.blkrange[i];
        lo_s = min(lo_s, br.x);
        hi_s = max(hi_s, br.y);
    }
    for (int k = 16; k > 0; k >>= 1) {
        lo_s = min(lo_s, __shfl_xor_sync(0xffffffffu, lo_s, k));
        hi_s = max(hi_s, __shfl_xor_sync(0xffffffffu, hi_s, k));
    }
    if (lane == 0) { s_lo[warp] = lo_s; s_hi[warp] = hi_s; }
    __syncthreads();
    lo_s = s_lo[0];
    hi_s = s_hi[0];
    for (int w = 1; w < 8; ++w) { lo_s = min(lo_s, s_lo[w]); hi_s = max(hi_s, s_hi[w]); }
    __syncthreads();
    const double betaT = betas[j0 + nt / 2];
    const float bTf = (float)betaT;
    // pass 1: approximate reference bin (FP32)
    float best = -INFINITY;
    int kT = max(0, hi_s);  // replaced by a sampled bin whenever there is one
#pragma unroll 4
    for (int b = lo_s + (int)threadIdx.x; b <= hi_s; b += 256) {
        const float l = r.lnOf[b];
        const float a = l - bTf * (float)bin_energy(model, V, b);
        if (l != -INFINITY && a > best) { best = a; kT = b; }
    }
    warp_argmax(best, kT);
    if (lane == 0) { s_v[warp] = best; s_i[warp] = kT; }
    __syncthreads();
    if (threadIdx.x < 32) {
        best = lane < 8 ? s_v[lane] : -INFINITY;
        kT = lane < 8 ? s_i[lane] : max(0, hi_s);
        warp_argmax(best, kT);
        if (lane == 0) s_i[0] = kT;
    }
    __syncthreads();
    kT = s_i[0];
    const float lTf = r.lnOf[kT];
    const double ETd = bin_energy(model, V, kT);
    const float ETf = (float)ETd;
    float db[kRwTile], dbmax = 0.f;
#pragma unroll
    for (int t = 0; t < kRwTile; ++t) {
        db[t] = t < nt ? (float)(betas[j0 + t] - betaT) : 0.f;
        dbmax = fmaxf(dbmax, fabsf(db[t]));
    }
    // pass 2: the window (bins that can reach e^-100 of the largest weight for some beta
    // of the tile, approximate exponents with 2 units of margin), and every beta's
    // maximum exponent and the bin that attains it: the beta's own reference, around
    // which its columns are centred (a tile may hold betas whose weights peak far apart;
    // centred on one tile-wide bin, C and chi would cancel there)
    int lo = hi_s + 1, hi = lo_s - 1;
    float mx[kRwTile];
    int mi[kRwTile];
#pragma unroll
    for (int t = 0; t < kRwTile; ++t) {
        mx[t] = -INFINITY;
        mi[t] = kT;
    }
#pragma unroll 2
    for (int b = lo_s + (int)threadIdx.x; b <= hi_s; b += 256) {
        const float l = r.lnOf[b];
        if (l == -INFINITY) continue;
        const float dE = (float)bin_energy(model, V, b) - ETf;
        const float G = (l - lTf) - bTf * dE;
        if (G + dbmax * fabsf(dE) >= (float)kCut - 2.f) { lo = min(lo, b); hi = max(hi, b); }
#pragma unroll
        for (int t = 0; t < kRwTile; ++t) {
            const float v = G - db[t] * dE;
            if (v > mx[t]) {
                mx[t] = v;
                mi[t] = b;
            }
        }
    }
    for (int k = 16; k > 0; k >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, k));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, k));
#pragma unroll
        for (int t = 0; t < kRwTile; ++t) {
            const float ov = __shfl_xor_sync(0xffffffffu, mx[t], k);
            const int oi = __shfl_xor_sync(0xffffffffu, mi[t], k);
            if (ov > mx[t] || (ov == mx[t] && oi < mi[t])) {
                mx[t] = ov;
                mi[t] = oi;
            }
        }
    }
    __syncthreads();
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
#pragma unroll
        for (int t = 0; t < kRwTile; ++t) {
            s_m[warp][t] = mx[t];
            s_mi[warp][t] = mi[t];
        }
    }
    __syncthreads();
    lo = s_lo[0];
    hi = s_hi[0];
    for (int w = 1; w < 8; ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
    if (lo > hi) {  // no sampled bin at all: an empty window
        lo = 0;
        hi = -1;
    }
    if ((int)threadIdx.x < nt) {
        const int t = threadIdx.x, j = j0 + t;
        float m = s_m[0][t];
        int k = s_mi[0][t];
        for (int w = 1; w < 8; ++w)
            if (s_m[w][t] > m || (s_m[w][t] == m && s_mi[w][t] < k)) {
                m = s_m[w][t];
                k = s_mi[w][t];
            }
        const double c = -(double)m;  // per-beta shift (ln units)
        r.c[j] = c;
        const double db2 = (betas[j] - betaT) * kLog2e;
        const float dbh = (float)db2;
        // the beta's reference: E_ref - E_T (an exact integer, also as a float) and the
        // bin's mean |M|
        const float dref = (float)(bin_energy(model, V, k) - ETd);
        r.bc[j] = make_float4(dbh, (float)(db2 - (double)dbh), (float)(c * kLog2e), dref);
        r.xref[j] = r.d.x1[k];
        r.xrf[j] = make_float2(r.x1h[k], r.x1l[k]);
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
        tp.lTh = r.lnOf[kT];
        tp.lTl = r.lnOl[kT];
        tp.x1Th = r.x1h[kT];
        tp.x1Tl = r.x1l[kT];
        tp.bTh = (float)betaT;
        tp.bTl = (float)(betaT - (double)tp.bTh);
        r.tiles[T] = tp;
    }
    // the last block to finish numbers the chunks (the classic last-block pattern: no
    // block waits for another)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(r.cnt0, 1u) == (unsigned)gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        scan_tiles(r, gridDim.x, n_beta, o);
        if (threadIdx.x == 0) *r.cnt0 = 0u;
    }
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Persistent grid over the (tile, chunk) items.  FP64: exponents, weights and sums in
// FP64.  FP32: compensated exponents and weights in FP32; every column sum is kept as a
// float pair (high part and the accumulated rounding errors of its additions), through
// the thread's bins and the warp's tree, and combined in FP64 across warps.  (Plain
// FP32 sums of 32 terms lost up to ~1e-6 relative on C and chi.)
template <bool FP64>
__global__ void __launch_bounds__(256) rw_sums_kernel(RwScratch r, const double *betas, int n_beta, int n_tiles,
                                                      int model, int V, double mnorm, Observables o)
{
    __shared__ double s_red[8][kRwTile][6];
    __shared__ float2 s_rf[8][kRwTile][6];
    __shared__ int s_done;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = r.off[n_tiles];
    const int dstep = model == MUCA_ISING ? 4 : 1;  // energy step between neighbouring bins
    const int n_bins = model == MUCA_ISING ? V + 1 : 2 * V + 1;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int T = r.item_tile[item];
        const TileParams tp = r.tiles[T];
        const int chunk = item - r.off[T];
        const int j0 = T * kRwTile, nt = min(kRwTile, n_beta - j0);
        const int b0 = tp.lo + chunk * tp.ch;
        // chunks are whole multiples of 32 bins: the last one may reach past the last
        // bin, where the per-bin arrays end (the next array follows directly)
        const int b1 = min(min(b0 + tp.ch, tp.lo + tp.nch * tp.ch), n_bins);
        if (FP64) {
            double cd[kRwTile], dbd[kRwTile], drd[kRwTile], xrd[kRwTile];
#pragma unroll
            for (int t = 0; t < kRwTile; ++t) {
                const bool ok = t < nt;
                cd[t] = ok ? r.c[j0 + t] : -1e300;
                dbd[t] = ok ? betas[j0 + t] - tp.betaT : 0.0;
                drd[t] = ok ? (double)r.bc[j0 + t].w : 0.0;
                xrd[t] = ok ? r.xref[j0 + t] : 0.0;
            }
            double acc[kRwTile][6];
#pragma unroll
            for (int t = 0; t < kRwTile; ++t)
#pragma unroll
                for (int k = 0; k < 6; ++k) acc[t][k] = 0.0;
            for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
                const double l = r.d.lnO[b];
                if (l == -INFINITY) continue;
                const double dEd = (double)(dstep * (b - tp.kT));
                const double G = __dsub_rn(__dsub_rn(l, tp.lnOT), __dmul_rn(tp.betaT, dEd));
                const double x1 = r.d.x1[b], vb = r.d.v[b];
#pragma unroll
                for (int t = 0; t < kRwTile; ++t) {
                    const double a = __fma_rn(-dbd[t], dEd, G + cd[t]);
                    if (a < kCut) continue;
                    const double w = exp(a);
                    // columns centred on the beta's reference bin
                    const double d = dEd - drd[t], dx = x1 - xrd[t];
                    const double cols[6] = {1.0, d, d * d, dx, dx * dx, vb};
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[t][k] = __fma_rn(w, cols[k], acc[t][k]);
                }
            }
#pragma unroll
            for (int t = 0; t < kRwTile; ++t)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    double x = acc[t][k];
                    for (int q = 16; q > 0; q >>= 1) x += __shfl_xor_sync(0xffffffffu, x, q);
                    if (lane == 0) s_red[warp][t][k] = x;
                }
            __syncthreads();
            if ((int)threadIdx.x < kRwTile * 6) {
                const int t = threadIdx.x / 6, k = threadIdx.x % 6;
                double x = 0.0;
                for (int w = 0; w < 8; ++w) x += s_red[w][t][k];
                r.part[((size_t)item * kRwTile + t) * 6 + k] = x;
            }
        } else {
            // FP32 only: the tile's reference and every beta's constants come as floats
            float dbh[kRwTile], dbl[kRwTile], chv[kRwTile], drf[kRwTile], xrh[kRwTile], xrl[kRwTile];
#pragma unroll
            for (int t = 0; t < kRwTile; ++t) {
                const float4 kc = t < nt ? r.bc[j0 + t] : make_float4(0.f, 0.f, -1e30f, 0.f);
                const float2 xr = t < nt ? r.xrf[j0 + t] : make_float2(0.f, 0.f);
                dbh[t] = kc.x;
                dbl[t] = kc.y;
                chv[t] = kc.z;
                drf[t] = kc.w;
                xrh[t] = xr.x;
                xrl[t] = xr.y;
            }
            const float L2h = (float)kLog2e, L2l = (float)(kLog2e - (double)(float)kLog2e);
            float hi[kRwTile][6], lo[kRwTile][6];
#pragma unroll
            for (int t = 0; t < kRwTile; ++t)
#pragma unroll
                for (int k = 0; k < 6; ++k) hi[t][k] = lo[t][k] = 0.f;
            for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
                const float lh = r.lnOf[b];
                if (lh == -INFINITY) continue;
                const float dE = (float)(dstep * (b - tp.kT));  // exact
                // G = (lnOmega_b - lnOmega_kT) - beta_T dE as a float pair, in log2 units
                float d1, e1, g1, e2;
                two_sum(lh, -tp.lTh, d1, e1);
                const float dlo = __fadd_rn(e1, __fsub_rn(r.lnOl[b], tp.lTl));
                const float p = __fmul_rn(tp.bTh, dE);
                const float pe = __fmaf_rn(tp.bTh, dE, -p);
                const float q = __fmul_rn(tp.bTl, dE);
                two_sum(d1, -p, g1, e2);
                const float glo = __fsub_rn(__fsub_rn(__fadd_rn(e2, dlo), pe), q);
                const float Gh = __fmul_rn(g1, L2h);
                const float Gl = __fadd_rn(__fmaf_rn(g1, L2h, -Gh), __fadd_rn(__fmul_rn(g1, L2l), __fmul_rn(glo, L2h)));
                const float x1h = r.x1h[b], x1l = r.x1l[b], vb = r.vf[b];
#pragma unroll
                for (int t = 0; t < kRwTile; ++t) {
                    // a = (Gh + Gl) + c - (dbh + dbl) dE as a float pair
                    const float pt = __fmul_rn(dbh[t], dE);
                    const float pte = __fmaf_rn(dbh[t], dE, -pt);
                    const float qt = __fmul_rn(dbl[t], dE);
                    float s1, f1, s2, f2;
                    two_sum(Gh, chv[t], s1, f1);
                    two_sum(s1, -pt, s2, f2);
                    const float rl = __fsub_rn(__fadd_rn(__fadd_rn(f1, f2), Gl), __fadd_rn(pte, qt));
                    const float ah = __fadd_rn(s2, rl);
                    const float al = __fsub_rn(rl, __fsub_rn(ah, s2));
                    const float w0 = exp2f(ah);
                    const float w = __fmaf_rn(w0, al * (float)kLn2, w0);
                    // columns centred on the beta's reference bin: the energy offset is an
                    // exact integer, the mean |M| a float pair
                    const float d = __fsub_rn(dE, drf[t]);
                    float xa, xe;
                    two_sum(x1h, -xrh[t], xa, xe);
                    const float dxf = __fadd_rn(xa, __fadd_rn(xe, __fsub_rn(x1l, xrl[t])));
                    const float cols[6] = {1.f, d, __fmul_rn(d, d), dxf, __fmul_rn(dxf, dxf), vb};
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        float sum, err;
                        two_sum(hi[t][k], __fmul_rn(w, cols[k]), sum, err);
                        hi[t][k] = sum;
                        lo[t][k] = __fadd_rn(lo[t][k], err);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < kRwTile; ++t)
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    float h = hi[t][k], e = lo[t][k];
                    for (int q = 16; q > 0; q >>= 1) {
                        const float oh = __shfl_xor_sync(0xffffffffu, h, q);
                        const float oe = __shfl_xor_sync(0xffffffffu, e, q);
                        float sum, err;
                        two_sum(h, oh, sum, err);
                        h = sum;
                        e = __fadd_rn(__fadd_rn(e, oe), err);
                    }
                    if (lane == 0) s_rf[warp][t][k] = make_float2(h, e);
                }
            __syncthreads();
            if ((int)threadIdx.x < kRwTile * 6) {
                const int t = threadIdx.x / 6, k = threadIdx.x % 6;
                float h = s_rf[0][t][k].x, e = s_rf[0][t][k].y;
                for (int w = 1; w < 8; ++w) {
                    float sum, err;
                    two_sum(h, s_rf[w][t][k].x, sum, err);
                    h = sum;
                    e = __fadd_rn(__fadd_rn(e, s_rf[w][t][k].y), err);
                }
                r.part[((size_t)item * kRwTile + t) * 6 + k] = (double)h + (double)e;
            }
        }
        // the block that completes a tile's last chunk combines the tile's partial sums
        // in chunk order (deterministic) and writes its observables
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_done = atomicAdd(&r.cnt[T], 1u) + 1u == (unsigned)tp.nch;
        __syncthreads();
        if (s_done) {
            __threadfence();
            if ((int)threadIdx.x < nt) {
                const int t = threadIdx.x;
                double S[6] = {0, 0, 0, 0, 0, 0};
                for (int i = r.off[T]; i < r.off[T] + tp.nch; ++i)
#pragma unroll
                    for (int k = 0; k < 6; ++k) S[k] += __ldcg(&r.part[((size_t)i * kRwTile + t) * 6 + k]);
                write_obs(o, j0 + t, betas[j0 + t], tp.ET + (double)r.bc[j0 + t].w, r.xref[j0 + t], S[0], S[1], S[2],
                          S[3], S[4], S[5], V, mnorm);
            }
        }
    }
}

}  // namespace

namespace {

// setup (with the chunk numbering) and sums (with the per-tile combine) of one batch of
// betas, the per-bin arrays of `r` prepared; `n_sm` sizes the persistent grid of the sums
cudaError_t launch_tiles(const RwScratch &r, const double *d_betas, int n_beta, int precision, int model, int V,
                         double mnorm, const Observables &o, int n_sm, cudaStream_t st)
{
    const int n_tiles = (n_beta + kRwTile - 1) / kRwTile;
    rw_setup_kernel<<<n_tiles, 256, 0, st>>>(r, d_betas, n_beta, model, V, o);
    const int grid = std::max(1, std::min(n_tiles * kRwMaxChunks, 4 * n_sm));
    if (precision == MUCA_FP64)
        rw_sums_kernel<true><<<grid, 256, 0, st>>>(r, d_betas, n_beta, n_tiles, model, V, mnorm, o);
    else
        rw_sums_kernel<false><<<grid, 256, 0, st>>>(r, d_betas, n_beta, n_tiles, model, V, mnorm, o);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(2);
    return e;
}

size_t align256(size_t bytes) { return rw_align256(bytes); }

// Pointers into the scratch.  The per-bin part is laid out for `cap` bins (>= nb), so
// that the setup counter at its end stays at one place for every lattice served.
RwScratch carve(void *bins, size_t cap, size_t nb, void *tiles, int n_beta)
{
    RwScratch r;
    char *pb = reinterpret_cast<char *>(bins);
    double *base = reinterpret_cast<double *>(pb);
    r.d = BinData{base, base + cap, base + 2 * cap, base + 3 * cap, base + 4 * cap};
    pb += align256(5 * cap * sizeof(double));
    r.lnOf = reinterpret_cast<float *>(pb);
    pb += align256(cap * sizeof(float));
    r.lnOl = reinterpret_cast<float *>(pb);
    pb += align256(cap * sizeof(float));
    r.x1h = reinterpret_cast<float *>(pb);
    pb += align256(cap * sizeof(float));
    r.x1l = reinterpret_cast<float *>(pb);
    pb += align256(cap * sizeof(float));
    r.vf = reinterpret_cast<float *>(pb);
    pb += align256(cap * sizeof(float));
    r.blkrange = reinterpret_cast<int2 *>(pb);
    r.nblk = (int)((nb + 255) / 256);
    pb += align256(sizeof(int2) * ((cap + 255) / 256));
    r.cnt0 = reinterpret_cast<unsigned *>(pb);
    const size_t n_tiles = (size_t)(n_beta + kRwTile - 1) / kRwTile;
    char *pt = reinterpret_cast<char *>(tiles);
    r.tiles = reinterpret_cast<TileParams *>(pt);
    pt += align256(sizeof(TileParams) * n_tiles);
    r.c = reinterpret_cast<double *>(pt);
    pt += align256(sizeof(double) * n_beta);
    r.bc = reinterpret_cast<float4 *>(pt);
    pt += align256(sizeof(float4) * n_beta);
    r.xref = reinterpret_cast<double *>(pt);
    pt += align256(sizeof(double) * n_beta);
    r.xrf = reinterpret_cast<float2 *>(pt);
    pt += align256(sizeof(float2) * n_beta);
    r.off = reinterpret_cast<int *>(pt);
    pt += align256(sizeof(int) * (n_tiles + 1));
    r.cnt = reinterpret_cast<unsigned *>(pt);
    pt += align256(sizeof(unsigned) * (n_tiles + 1));  // (one spare entry)
    r.item_tile = reinterpret_cast<int *>(pt);
    pt += align256(sizeof(int) * n_tiles * kRwMaxChunks);
    r.part = reinterpret_cast<double *>(pt);
    return r;
}

cudaError_t launch_prep(const RwScratch &r, const uint64_t *samples, const double *lnw, int model, int V, int nb,
                        cudaStream_t st)
{
    rw_prep_kernel<<<r.nblk, 256, 0, st>>>(samples, lnw, r, model, V, nb);
    cudaError_t e = cudaGetLastError();
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
    RwScratch r = carve(base, kNoallocMaxBins, nb, base + rw_bin_part_bytes(kNoallocMaxBins), kNoallocBetasPerPass);
    // the setup counter is cleared by every call here: calls that overlapped on the GPU
    // (a race the caller must avoid) then spoil their own results only
    cudaError_t e = cudaMemsetAsync(r.cnt0, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    e = launch_prep(r, samples, lnw, model, V, nb, st);
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

int launch_reweight(muca_ctx *ctx, const double *d_betas, int n_beta, int precision, double *const out[4])
{
    const size_t nb = ctx->n_bins;
    double *base = reinterpret_cast<double *>(ctx->d_rw);
    BinData d{base, base + nb, base + 2 * nb, base + 3 * nb, base + 4 * nb};
    Observables o{out[0], out[1], out[2], out[3]};
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
    // per-call scratch: tile parameters, shifts, item offsets, counters, partial sums
    const size_t need = rw_tile_part_bytes((size_t)n_beta);
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
    const RwScratch r = carve(ctx->d_rw, nb, nb, ctx->d_rwtile, n_beta);
    MUCA_CUDA_TRY(launch_prep(r, ctx->d_samples, ctx->d_lnw_prod, ctx->model, ctx->V, ctx->n_bins, ctx->stream));
    MUCA_CUDA_TRY(launch_tiles(r, d_betas, n_beta, precision, ctx->model, ctx->V, mnorm, o, ctx->n_sm, ctx->stream));
    return MUCA_OK;
}

}  // namespace muca
