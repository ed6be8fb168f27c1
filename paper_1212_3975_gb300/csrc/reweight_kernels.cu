// Time-series reweighting (arXiv:1212.3975, Eq. 2; C_V of Sec. 5) on the device.
//
// The production records are already reduced to exact integer sums per energy bin
// (count n, sum |M|, sum M^2), so Eq. 2 becomes, per inverse temperature beta,
//     <X>_beta = sum_b w_b(beta) X_b / sum_b w_b(beta),
//     w_b(beta) = exp(lnOmega_b - beta E_b - shift_beta),  lnOmega_b = ln n_b - ln W_b,
// with X_b the per-bin means {1, E, E^2, |M|, M^2} and shift_beta the log-sum-exp
// shift max_b(lnOmega_b - beta E_b), always in FP64.
//
// MUCA_FP64: one block per beta, FP64 table and sums; terms with exponent below
//            -100 are skipped (each is < e^-100 of the largest, invisible in FP64).
// MUCA_FP32: one block per tile of betas.  The block finds in FP64 the reference
//            bin k_T (maximum at the tile's middle beta), the window of bins that
//            can matter for any beta of the tile, and every beta's FP64 shift; the
//            table is then evaluated in FP32 in locally referenced form
//                a = G_T(b) + c_beta - (beta - beta_T)(E_b - E_kT)   (log2 units)
//            with G_T(b) = lnOmega_b - lnOmega_kT - beta_T (E_b - E_kT) <= 0, so no
//            large numbers cancel in FP32, and the contraction uses centred columns
//            {1, dE, dE^2, d|m|, d|m|^2, var_b(|m|)} so that C and chi do not suffer
//            from cancellation.  Sums are combined across threads in FP64.
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

template <int N>
__device__ void block_sum(double (&x)[N], double *s_buf)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_xor_sync(0xffffffffu, x[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) s_buf[warp * N + k] = x[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] += s_buf[w * N + k];
#pragma unroll
        for (int k = 0; k < N; ++k) s_buf[k] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = s_buf[k];
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

// ------------------------------ FP64 -------------------------------------------
__global__ void __launch_bounds__(256) reweight_fp64_kernel(BinData d, const double *betas, int n_bins, int V,
                                                            double mnorm, Observables o)
{
    __shared__ double s_val[32 * 6];
    __shared__ int s_idx[32];
    const int j = blockIdx.x;
    const double beta = betas[j];
    double best = -INFINITY;
    int bi = n_bins;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double a = __dsub_rn(l, __dmul_rn(beta, d.E[b]));
        if (a > best || (a == best && b < bi)) { best = a; bi = b; }
    }
    block_argmax(best, bi, s_val, s_idx);
    const double shift = best;
    const double Eref = d.E[bi], x1ref = d.x1[bi];
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double a = __dsub_rn(__dsub_rn(l, __dmul_rn(beta, d.E[b])), shift);
        if (a < kCut) continue;
        const double w = exp(a);
        const double dE = d.E[b] - Eref, dx = d.x1[b] - x1ref;
        S[0] += w;
        S[1] += w * dE;
        S[2] += w * dE * dE;
        S[3] += w * dx;
        S[4] += w * dx * dx;
        S[5] += w * d.v[b];
    }
    block_sum<6>(S, s_val);
    if (threadIdx.x == 0) write_obs(o, j, beta, Eref, x1ref, S[0], S[1], S[2], S[3], S[4], S[5], V, mnorm);
}

// ------------------------------ FP32 -------------------------------------------
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

template <int TILE>
__global__ void __launch_bounds__(256) reweight_fp32_kernel(BinData d, const double *betas, int n_beta,
                                                            int n_bins, int V, double mnorm, Observables o)
{
    __shared__ double s_val[32 * 6];
    __shared__ int s_idx[32];
    __shared__ float s_c[TILE], s_db[TILE];
    __shared__ double s_red[8 * 6 * TILE];
    const int j0 = blockIdx.x * TILE;
    const int nt = min(TILE, n_beta - j0);
    const double betaT = betas[j0 + nt / 2];

    // reference bin of the tile (FP64)
    double best = -INFINITY;
    int kT = n_bins;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double a = __dsub_rn(l, __dmul_rn(betaT, d.E[b]));
        if (a > best || (a == best && b < kT)) { best = a; kT = b; }
    }
    block_argmax(best, kT, s_val, s_idx);
    const double lnOT = d.lnO[kT], ET = d.E[kT], x1T = d.x1[kT];
    double dbmax = 0.0;
    for (int t = 0; t < nt; ++t) dbmax = fmax(dbmax, fabs(betas[j0 + t] - betaT));

    // window of bins that can contribute above e^kCut for some beta of the tile
    int lo = n_bins, hi = -1;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double dE = d.E[b] - ET;
        const double G = (l - lnOT) - betaT * dE;
        if (G + dbmax * fabs(dE) >= kCut) { lo = min(lo, b); hi = max(hi, b); }
    }
    {
        double v1 = -(double)lo;
        int i1 = 0;
        block_argmax(v1, i1, s_val, s_idx);
        lo = (int)(-v1);
        double v2 = (double)hi;
        int i2 = 0;
        block_argmax(v2, i2, s_val, s_idx);
        hi = (int)v2;
    }

    // FP64 shift of every beta of the tile (maximum lies inside the window)
    tile_shifts<TILE>(d, betas, j0, nt, lo, hi, lnOT, ET, betaT, s_c, s_db);
    float cj[TILE], dbj[TILE];
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
        cj[t] = t < nt ? s_c[t] : -1e30f;
        dbj[t] = t < nt ? s_db[t] : 0.f;
    }

    // FP32 table and contraction
    float acc[TILE][6];
#pragma unroll
    for (int t = 0; t < TILE; ++t)
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[t][k] = 0.f;
    for (int b = lo + (int)threadIdx.x; b <= hi; b += blockDim.x) {
        const double l = d.lnO[b];
        if (l == -INFINITY) continue;
        const double dEd = d.E[b] - ET;
        const float G = (float)(((l - lnOT) - betaT * dEd) * kLog2e);
        const float dE = (float)dEd;
        const float dx = (float)(d.x1[b] - x1T);
        const float vb = (float)d.v[b];
        const float dE2 = dE * dE, dx2 = dx * dx;
#pragma unroll
        for (int t = 0; t < TILE; ++t) {
            const float a = fmaf(-dbj[t], dE, G + cj[t]);
            const float w = exp2f(a);
            acc[t][0] += w;
            acc[t][1] = fmaf(w, dE, acc[t][1]);
            acc[t][2] = fmaf(w, dE2, acc[t][2]);
            acc[t][3] = fmaf(w, dx, acc[t][3]);
            acc[t][4] = fmaf(w, dx2, acc[t][4]);
            acc[t][5] = fmaf(w, vb, acc[t][5]);
        }
    }
    // reduce: FP32 within a warp, FP64 across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < TILE; ++t)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float x = acc[t][k];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) s_red[(warp * TILE + t) * 6 + k] = (double)x;
        }
    __syncthreads();
    if ((int)threadIdx.x < nt) {
        const int t = threadIdx.x;
        double S[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 6; ++k) S[k] += s_red[(w * TILE + t) * 6 + k];
        write_obs(o, j0 + t, betas[j0 + t], ET, x1T, S[0], S[1], S[2], S[3], S[4], S[5], V, mnorm);
    }
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

}  // namespace

// Same kernels with every buffer supplied by the caller: per-bin scratch of
// 5 * n_bins doubles, production sums [3][n_bins], weights [n_bins], betas and the
// output [4][n_beta] (all device memory).  Launches on `st`; allocates nothing.
cudaError_t launch_reweight_buffers(double *scratch, const uint64_t *samples, const double *lnw, int model, int L,
                                    int q, const double *d_betas, int n_beta, int precision, double *d_out,
                                    cudaStream_t st)
{
    const int V = L * L;
    const int nb = n_bins_of(model, L);
    BinData d{scratch, scratch + nb, scratch + 2 * (size_t)nb, scratch + 3 * (size_t)nb, scratch + 4 * (size_t)nb};
    prep_kernel<<<(nb + 255) / 256, 256, 0, st>>>(samples, lnw, d, model, V, nb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(1);
    Observables o{d_out, d_out + n_beta, d_out + 2 * n_beta, d_out + 3 * n_beta};
    const double mnorm = model == MUCA_ISING ? (double)V : (double)(q - 1) * V;
    if (precision == MUCA_FP64)
        reweight_fp64_kernel<<<n_beta, 256, 0, st>>>(d, d_betas, nb, V, mnorm, o);
    else
        reweight_fp32_kernel<8><<<(n_beta + 7) / 8, 256, 0, st>>>(d, d_betas, n_beta, nb, V, mnorm, o);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(1);
    return e;
}

int launch_reweight(muca_ctx *ctx, const double *d_betas, int n_beta, int precision, double *d_out)
{
    const size_t nb = ctx->n_bins;
    double *base = reinterpret_cast<double *>(ctx->d_rw);
    BinData d{base, base + nb, base + 2 * nb, base + 3 * nb, base + 4 * nb};
    prep_kernel<<<(ctx->n_bins + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_samples, ctx->d_lnw_prod, d, ctx->model,
                                                                   ctx->V, ctx->n_bins);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    Observables o{d_out, d_out + n_beta, d_out + 2 * n_beta, d_out + 3 * n_beta};
    const double mnorm = ctx->model == MUCA_ISING ? (double)ctx->V : (double)(ctx->q - 1) * ctx->V;
    if (precision == MUCA_FP64) {
        reweight_fp64_kernel<<<n_beta, 256, 0, ctx->stream>>>(d, d_betas, ctx->n_bins, ctx->V, mnorm, o);
    } else if (precision == MUCA_FP32) {
        const int tiles = (n_beta + 7) / 8;
        reweight_fp32_kernel<8><<<tiles, 256, 0, ctx->stream>>>(d, d_betas, n_beta, ctx->n_bins, ctx->V, mnorm, o);
    } else if (precision == MUCA_BF16) {
        const int tiles = (n_beta + 15) / 16;
        reweight_bf16_kernel<<<tiles, 32 * kBf16Warps, 0, ctx->stream>>>(d, d_betas, n_beta, ctx->n_bins, ctx->V,
                                                                         mnorm, o);
    } else {
        return fail(MUCA_ERR_ARG, "precision must be MUCA_FP64, MUCA_FP32 or MUCA_BF16");
    }
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

}  // namespace muca
