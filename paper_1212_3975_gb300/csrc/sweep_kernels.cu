// Sweep kernels of the parallel multicanonical method (arXiv:1212.3975, Secs. 2-3):
// one CUDA thread runs one Markov chain; the 32 chains of a warp sweep their own
// lattices in lockstep typewriter order, so every lattice access of a warp is one
// coalesced 128-byte row of the chain-interleaved layout.
//
// Per attempt (Sec. 3: a sweep is V single-spin updates, site order i = y*L + x):
//   Philox4x32-10 draw -> energy change dE from the four neighbours -> acceptance
//   min(1, W(E')/W(E)) of Eq. 1 as an integer test u < A[bin(E)][dE] (A = 2^32-1
//   always accepts; dE = 0 always accepts) -> flip/update E, M -> histogram of the
//   energy after the attempt (run-length merged, flushed when the bin changes).
// Histograms go to a block-shared uint32 histogram (or straight to the global uint64
// one when it does not fit) and are merged into H = sum_i H_i at the end of the
// launch (Sec. 2, Parallel Version).
#include <algorithm>
#include <cstdio>

#include "muca_internal.cuh"

namespace muca {
namespace {

constexpr int kMaxSmem = 227 * 1024;

template <bool HSMEM>
__device__ __forceinline__ void flush_run(uint32_t *s_hist, uint64_t *g_hist, int bin,
                                          uint32_t run)
{
    if (HSMEM)
        atomicAdd(&s_hist[bin], run);
    else
        atomicAdd(reinterpret_cast<unsigned long long *>(&g_hist[bin]),
                  static_cast<unsigned long long>(run));
}

__device__ __forceinline__ void record_sample(const SweepArgs &a, int sw, int c, int E,
                                              int M, int bin)
{
    if (a.E_rec) a.E_rec[(size_t)sw * a.rec_stride + c] = E;
    if (a.M_rec) a.M_rec[(size_t)sw * a.rec_stride + c] = M;
    if (a.samples) {
        const unsigned long long am = (unsigned long long)(M < 0 ? -M : M);
        unsigned long long *s = reinterpret_cast<unsigned long long *>(a.samples);
        atomicAdd(&s[bin], 1ull);
        atomicAdd(&s[a.n_bins + bin], am);
        atomicAdd(&s[2 * a.n_bins + bin], am * am);
    }
}

// Potts state counts packed as 16-bit fields: lo = states 0..3, hi = states 4..7.
__device__ __forceinline__ void count_add(uint64_t &lo, uint64_t &hi, uint32_t s, int64_t d)
{
    const uint64_t one = 1ull << (16 * (s & 3u));
    if (s < 4) lo += d > 0 ? one : (0ull - one);
    else hi += d > 0 ? one : (0ull - one);
}

__device__ __forceinline__ int count_max(uint64_t lo, uint64_t hi)
{
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        m = max(m, (int)((lo >> (16 * k)) & 0xFFFFu));
        m = max(m, (int)((hi >> (16 * k)) & 0xFFFFu));
    }
    return m;
}

// ---------------------------------------------------------------------------
// Ising, bit-packed.
// ---------------------------------------------------------------------------
template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
__global__ void __launch_bounds__(256) ising_sweep_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_thr = a.n_bins * 4;
    uint32_t *s_thr = smem;
    uint32_t *s_hist = smem + (TSMEM ? n_thr : 0);
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? a.n_bins : 0);
    const int cpb = blockDim.x, tid = threadIdx.x;
    const int c = blockIdx.x * cpb + tid;

    if (TSMEM) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.thr);
        uint4 *dst = reinterpret_cast<uint4 *>(s_thr);
        for (int i = tid; i < a.n_bins; i += cpb) dst[i] = src[i];
    }
    if (HIST && HSMEM)
        for (int i = tid; i < a.n_bins; i += cpb) s_hist[i] = 0u;
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * cpb + tid] = a.lat[(size_t)k * a.p_pad + c];
    __syncthreads();

    uint32_t *lp = LSMEM ? s_lat + tid : a.lat + c;
    const size_t ls = LSMEM ? (size_t)cpb : (size_t)a.p_pad;
#define LAT(k) lp[(size_t)(k) * ls]
#define THR(i) (TSMEM ? s_thr[(i)] : __ldg(a.thr + (i)))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L;
        const int last_bits = L - 32 * (RW - 1);
        int bin = (a.E[c] + 2 * V) >> 2;
        int M = a.M[c];
        int run_bin = bin;
        uint32_t run = 0;
        uint4 blk = make_uint4(0, 0, 0, 0);
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;  // row above: updated (old for y = 0)
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;  // row below: old (new for y = L-1)
                uint32_t R = LAT(kr);
                // left neighbour of site 0 is site L-1 of this row, not yet updated
                uint32_t left = (LAT(kr + RW - 1) >> (last_bits - 1)) & 1u;
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w) {
                    const bool lastw = (w == RW - 1);
                    const int nb = lastw ? last_bits : 32;
                    const uint32_t U = LAT(ku + w), D = LAT(kd + w);
                    const uint32_t Rn = lastw ? 0u : LAT(kr + w + 1);
                    // right neighbour of the word's last site: next word (old) or,
                    // at the row end, site 0 of this row (already updated)
                    const uint32_t edge = lastw ? first_new : (Rn & 1u);
                    const uint32_t ua = R ^ U, ub = R ^ D;  // unequal up/down neighbours
                    for (int j = 0; j < nb; ++j, ++site) {
                        if (j == 0 || (site & 3) == 0)
                            blk = philox4x32_10(make_uint4((uint32_t)site >> 2, ctr1, a.iteration, a.ctr3),
                                                a.key0, (uint32_t)c);
                        const int sel = site & 3;
                        const uint32_t u = sel == 0 ? blk.x : sel == 1 ? blk.y : sel == 2 ? blk.z : blk.w;
                        const uint32_t s = (R >> j) & 1u;
                        uint32_t r;
                        if (j + 1 < nb) r = (R >> (j + 1)) & 1u;
                        else r = (RW == 1) ? (R & 1u) : edge;
                        const int nneq = (int)(((ua >> j) & 1u) + ((ub >> j) & 1u) + (s ^ left) + (s ^ r));
                        bool acc = true;
                        if (nneq != 2) {
                            // bin change 2 - nneq; columns ordered by ascending dE
                            const int col = nneq >= 3 ? 4 - nneq : 3 - nneq;
                            const uint32_t A = THR(bin * 4 + col);
                            acc = (u < A) || (A == kAlways);
                        }
                        if (acc) {
                            R ^= 1u << j;
                            bin += 2 - nneq;
                            M += s ? -2 : 2;
                        }
                        left = s ^ (acc ? 1u : 0u);
                        if (HIST) {
                            if (bin != run_bin) {
                                flush_run<HSMEM>(s_hist, a.H, run_bin, run);
                                run_bin = bin;
                                run = 0;
                            }
                            ++run;
                        }
                    }
                    if (w == 0) first_new = R & 1u;
                    LAT(kr + w) = R;
                    R = Rn;
                }
            }
            if (RECORD) record_sample(a, sw, c, 4 * bin - 2 * V, M, bin);
        }
        a.E[c] = 4 * bin - 2 * V;
        a.M[c] = M;
        if (HIST && run) flush_run<HSMEM>(s_hist, a.H, run_bin, run);
    }
#undef LAT
#undef THR
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) a.lat[(size_t)k * a.p_pad + c] = s_lat[k * cpb + tid];
    if (HIST && HSMEM) {
        __syncthreads();
        for (int i = tid; i < a.n_bins; i += cpb) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}

// ---------------------------------------------------------------------------
// 8-state Potts, one byte per site.
// ---------------------------------------------------------------------------
template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
__global__ void __launch_bounds__(256) potts_sweep_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_thr = a.n_bins * 8;
    uint32_t *s_thr = smem;
    uint32_t *s_hist = smem + (TSMEM ? n_thr : 0);
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? a.n_bins : 0);
    const int cpb = blockDim.x, tid = threadIdx.x;
    const int c = blockIdx.x * cpb + tid;

    if (TSMEM) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.thr);
        uint4 *dst = reinterpret_cast<uint4 *>(s_thr);
        for (int i = tid; i < 2 * a.n_bins; i += cpb) dst[i] = src[i];
    }
    if (HIST && HSMEM)
        for (int i = tid; i < a.n_bins; i += cpb) s_hist[i] = 0u;
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * cpb + tid] = a.lat[(size_t)k * a.p_pad + c];
    __syncthreads();

    uint32_t *lp = LSMEM ? s_lat + tid : a.lat + c;
    const size_t ls = LSMEM ? (size_t)cpb : (size_t)a.p_pad;
#define LAT(k) lp[(size_t)(k) * ls]
#define THR(i) (TSMEM ? s_thr[(i)] : __ldg(a.thr + (i)))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L, q = a.q;
        const int last_sites = L - 4 * (RW - 1);
        int bin = a.E[c] + 2 * V;
        uint64_t cnt_lo = a.cnt[c], cnt_hi = a.cnt[a.p_pad + c];
        int run_bin = bin;
        uint32_t run = 0;
        uint4 blk = make_uint4(0, 0, 0, 0);
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;
                uint32_t R = LAT(kr);
                uint32_t left = (LAT(kr + RW - 1) >> (8 * (last_sites - 1))) & 0xFFu;
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w) {
                    const bool lastw = (w == RW - 1);
                    const int ns = lastw ? last_sites : 4;
                    const uint32_t U = LAT(ku + w), D = LAT(kd + w);
                    const uint32_t Rn = lastw ? 0u : LAT(kr + w + 1);
                    const uint32_t edge = lastw ? first_new : (Rn & 0xFFu);
                    for (int j = 0; j < ns; ++j, ++site) {
                        if (j == 0 || (site & 1) == 0)
                            blk = philox4x32_10(make_uint4((uint32_t)site >> 1, ctr1, a.iteration, a.ctr3),
                                                a.key0, (uint32_t)c);
                        const bool odd = (site & 1) != 0;
                        const uint32_t u = odd ? blk.z : blk.x;
                        const uint32_t pw = odd ? blk.w : blk.y;
                        const uint32_t s = (R >> (8 * j)) & 0xFFu;
                        uint32_t r;
                        if (j + 1 < ns) r = (R >> (8 * (j + 1))) & 0xFFu;
                        else r = (RW == 1) ? (R & 0xFFu) : edge;
                        uint32_t sn = s + 1u + __umulhi(pw, (uint32_t)(q - 1));
                        if (sn >= (uint32_t)q) sn -= (uint32_t)q;
                        const uint32_t nb4 = ((U >> (8 * j)) & 0xFFu) | (((D >> (8 * j)) & 0xFFu) << 8) |
                                             (left << 16) | (r << 24);
                        const int same_old = __popc(__vcmpeq4(nb4, s * 0x01010101u)) >> 3;
                        const int same_new = __popc(__vcmpeq4(nb4, sn * 0x01010101u)) >> 3;
                        const int dE = same_old - same_new;
                        bool acc = true;
                        if (dE != 0) {
                            const int col = dE < 0 ? dE + 4 : dE + 3;
                            const uint32_t A = THR(bin * 8 + col);
                            acc = (u < A) || (A == kAlways);
                        }
                        if (acc) {
                            R = (R & ~(0xFFu << (8 * j))) | (sn << (8 * j));
                            bin += dE;
                            count_add(cnt_lo, cnt_hi, s, -1);
                            count_add(cnt_lo, cnt_hi, sn, +1);
                        }
                        left = acc ? sn : s;
                        if (HIST) {
                            if (bin != run_bin) {
                                flush_run<HSMEM>(s_hist, a.H, run_bin, run);
                                run_bin = bin;
                                run = 0;
                            }
                            ++run;
                        }
                    }
                    if (w == 0) first_new = R & 0xFFu;
                    LAT(kr + w) = R;
                    R = Rn;
                }
            }
            if (RECORD) record_sample(a, sw, c, bin - 2 * V, q * count_max(cnt_lo, cnt_hi) - V, bin);
        }
        a.E[c] = bin - 2 * V;
        a.M[c] = q * count_max(cnt_lo, cnt_hi) - V;
        a.cnt[c] = cnt_lo;
        a.cnt[a.p_pad + c] = cnt_hi;
        if (HIST && run) flush_run<HSMEM>(s_hist, a.H, run_bin, run);
    }
#undef LAT
#undef THR
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) a.lat[(size_t)k * a.p_pad + c] = s_lat[k * cpb + tid];
    if (HIST && HSMEM) {
        __syncthreads();
        for (int i = tid; i < a.n_bins; i += cpb) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}

// ---------------------------------------------------------------------------
// Infinite-temperature start (Sec. 3): spins from Philox phase 0, one thread per
// (word, chain).  Ising: site i takes word i & 3 of block i >> 2, s = +1 iff its
// top bit is set.  Potts: the same words, s = (word * q) >> 32.
// ---------------------------------------------------------------------------
__global__ void init_lattice_kernel(uint32_t *lat, int model, int L, int q, int p, int p_pad,
                                    int row_words, int lat_words, uint32_t key0, uint32_t ctr3)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (c >= p_pad || k >= lat_words) return;
    uint32_t word = 0u;
    if (c < p) {
        const int y = k / row_words, w = k % row_words;
        const int per = model == MUCA_ISING ? 32 : 4;
        for (int j = 0; j < per; ++j) {
            const int x = per * w + j;
            if (x >= L) break;
            const int i = y * L + x;
            const uint4 b = philox4x32_10(make_uint4((uint32_t)i >> 2, 0u, 0u, ctr3), key0, (uint32_t)c);
            const uint32_t r = (i & 3) == 0 ? b.x : (i & 3) == 1 ? b.y : (i & 3) == 2 ? b.z : b.w;
            if (model == MUCA_ISING)
                word |= (r >> 31) << j;
            else
                word |= __umulhi(r, (uint32_t)q) << (8 * j);
        }
    }
    lat[(size_t)k * p_pad + c] = word;
}

__device__ __forceinline__ uint32_t site_value(const uint32_t *lat, int model, int L, int row_words,
                                               int p_pad, int c, int x, int y)
{
    if (model == MUCA_ISING) {
        const uint32_t wv = lat[(size_t)(y * row_words + (x >> 5)) * p_pad + c];
        return (wv >> (x & 31)) & 1u;
    }
    const uint32_t wv = lat[(size_t)(y * row_words + (x >> 2)) * p_pad + c];
    return (wv >> (8 * (x & 3))) & 0xFFu;
}

// Full recount of E, M and (Potts) the state counts of every chain.
__global__ void recount_kernel(const uint32_t *lat, int32_t *E, int32_t *M, uint64_t *cnt, int model,
                               int L, int q, int p, int p_pad, int row_words)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p) return;
    int e = 0, m = 0;
    uint32_t count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            const uint32_t s = site_value(lat, model, L, row_words, p_pad, c, x, y);
            const uint32_t r = site_value(lat, model, L, row_words, p_pad, c, (x + 1) % L, y);
            const uint32_t d = site_value(lat, model, L, row_words, p_pad, c, x, (y + 1) % L);
            if (model == MUCA_ISING) {
                e -= (s == r) ? 1 : -1;
                e -= (s == d) ? 1 : -1;
                m += s ? 1 : -1;
            } else {
                e -= (s == r);
                e -= (s == d);
                count[s & 7u] += 1;
            }
        }
    }
    if (model == MUCA_POTTS) {
        uint64_t lo = 0, hi = 0;
        uint32_t mx = 0;
        for (int k = 0; k < 4; ++k) {
            lo |= (uint64_t)count[k] << (16 * k);
            hi |= (uint64_t)count[k + 4] << (16 * k);
        }
        for (int k = 0; k < 8; ++k) mx = max(mx, count[k]);
        cnt[c] = lo;
        cnt[p_pad + c] = hi;
        m = q * (int)mx - L * L;
    }
    E[c] = e;
    M[c] = m;
}

__global__ void unpack_kernel(const uint32_t *lat, int8_t *out, int model, int L, int p, int p_pad,
                              int row_words)
{
    const size_t V = (size_t)L * L;
    const size_t total = V * (size_t)p;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / V);
        const int i = (int)(t % V);
        const uint32_t s = site_value(lat, model, L, row_words, p_pad, c, i % L, i / L);
        out[t] = model == MUCA_ISING ? (int8_t)(s ? 1 : -1) : (int8_t)s;
    }
}

template <int MODEL, bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
cudaError_t launch_one(const SweepArgs &a, int blocks, int cpb, size_t smem, cudaStream_t st)
{
    auto kern = MODEL == MUCA_ISING ? ising_sweep_kernel<HIST, RECORD, TSMEM, HSMEM, LSMEM>
                                    : potts_sweep_kernel<HIST, RECORD, TSMEM, HSMEM, LSMEM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, cpb, smem, st>>>(a);
    return cudaGetLastError();
}

template <int MODEL, bool HIST, bool RECORD>
cudaError_t dispatch_staging(const SweepArgs &a, const SweepPlan &pl, int blocks, cudaStream_t st)
{
    const int cpb = pl.chains_per_block;
    const size_t sm = pl.smem_bytes;
    const int key = (pl.table_smem ? 4 : 0) | ((HIST && pl.hist_smem) ? 2 : 0) | (pl.lattice_smem ? 1 : 0);
    switch (key) {
    case 0: return launch_one<MODEL, HIST, RECORD, false, false, false>(a, blocks, cpb, sm, st);
    case 1: return launch_one<MODEL, HIST, RECORD, false, false, true>(a, blocks, cpb, sm, st);
    case 2: return launch_one<MODEL, HIST, RECORD, false, true, false>(a, blocks, cpb, sm, st);
    case 3: return launch_one<MODEL, HIST, RECORD, false, true, true>(a, blocks, cpb, sm, st);
    case 4: return launch_one<MODEL, HIST, RECORD, true, false, false>(a, blocks, cpb, sm, st);
    case 5: return launch_one<MODEL, HIST, RECORD, true, false, true>(a, blocks, cpb, sm, st);
    case 6: return launch_one<MODEL, HIST, RECORD, true, true, false>(a, blocks, cpb, sm, st);
    default: return launch_one<MODEL, HIST, RECORD, true, true, true>(a, blocks, cpb, sm, st);
    }
}

template <int MODEL>
cudaError_t dispatch_mode(const SweepArgs &a, const SweepPlan &pl, int blocks, bool hist, bool record,
                          cudaStream_t st)
{
    if (hist && record) return dispatch_staging<MODEL, true, true>(a, pl, blocks, st);
    if (hist) return dispatch_staging<MODEL, true, false>(a, pl, blocks, st);
    if (record) return dispatch_staging<MODEL, false, true>(a, pl, blocks, st);
    return dispatch_staging<MODEL, false, false>(a, pl, blocks, st);
}

}  // namespace

SweepPlan plan_sweeps(const muca_ctx *ctx, bool allow_pairs, bool allow_compact)
{
    SweepPlan pl;
    pl.compact = false;
    pl.t16 = false;
    pl.hist16 = false;
    int cpb = ctx->cfg.chains_per_block;
    if (cpb <= 0) {
        // Spread the chains over the SMs: one warp per block while that leaves SMs
        // idle, larger blocks once there are more warps than SMs.
        const int warps = ctx->p_pad / 32;
        cpb = warps <= ctx->n_sm ? 32 : warps <= 4 * ctx->n_sm ? 64 : 128;
    }
    cpb = std::max(32, std::min(256, (cpb / 32) * 32));
    const bool fast = (ctx->L % 4) == 0;
    // the warp-specialised kernels serve 32 chains per block
    const bool ws = fast;
    if (ws) cpb = 32;
    pl.chains_per_block = cpb;
    pl.warp_specialized = ws;
    const size_t cap = (size_t)kMaxSmem - (ws ? ws_extra_smem(ctx->model) : 0);
    const int width = fast ? (ctx->model == MUCA_ISING ? 5 : 9) : ctx->n_de;
    const size_t table = ((size_t)ctx->n_bins * width * 4 + 15) & ~(size_t)15;
    // (+ one slot per lane for the inactive lanes of the warp-specialised kernels)
    const size_t hist = (((size_t)ctx->n_bins * 4 + 15) & ~(size_t)15) + 128;
    const size_t lat = (size_t)ctx->lat_words * 4 * cpb;
    size_t used = 0;
    pl.table_smem = table <= 96 * 1024;
    if (pl.table_smem) used += table;
    pl.hist_smem = used + hist <= 160 * 1024;
    // Ising histograms too large for 32-bit counts in shared memory (256 x 256: 262 KB):
    // 16-bit counts, two bins per word, flushed into the merged histogram by rows
    // (otherwise every bin change of a chain is a global atomic) -- where the lattices
    // cannot be staged in shared memory anyway, so that the histogram takes no room from
    // them (at 224 x 224 they fit, and staging them is worth more to thermalisation and
    // production than the 16-bit counts to the iterations)
    const int staging = ctx->cfg.staging;
    const size_t hist16 = ((((size_t)ctx->n_bins + 1) / 2 * 4 + 15) & ~(size_t)15) + 128;
    if (!pl.hist_smem && ws && ctx->model == MUCA_ISING && staging != MUCA_STAGING_SHARED && used + lat > cap &&
        used + hist16 <= 160 * 1024)
        pl.hist_smem = pl.hist16 = true;  // (the table is in global memory here too)
    if (pl.hist_smem) used += pl.hist16 ? hist16 : hist;
    pl.lattice_smem = staging == MUCA_STAGING_SHARED || (staging == MUCA_STAGING_AUTO && used + lat <= cap);
    if (pl.lattice_smem) used += lat;
    // warp-specialised launches: the histogram of attempt pairs (one count per bin
    // change of a single attempt: 5 for Ising, 9 for Potts) when it fits beside the
    // table and the lattices
    const size_t pairs = (((size_t)ctx->n_bins * width * 4 + 15) & ~(size_t)15) + 128;
    pl.hist_pairs = allow_pairs && ws && !pl.hist16 && pl.table_smem && pl.hist_smem && pl.lattice_smem &&
                    used - hist + pairs <= cap;
    if (pl.hist_pairs) used += pairs - hist;
    pl.smem_bytes = used;
    pl.table_bytes = pl.table_smem ? table : 0;
    pl.hist_bytes = pl.hist_smem ? (pl.hist_pairs ? pairs : pl.hist16 ? hist16 : hist) : 0;
    pl.lat_bytes = pl.lattice_smem ? lat : 0;
    // More groups of 32 chains than SMs (the throughput regime): a plan whose block
    // takes more than half of an SM's shared memory runs one block per SM and leaves
    // the other groups waiting for a second wave.  The compact Ising staging keeps the
    // table and a histogram of single attempts in shared memory, the lattices in
    // global memory (L1/L2) and three draw-ring slots, which fits two blocks per SM.
    const size_t per_sm = (size_t)ctx->smem_per_sm, reserved = (size_t)ctx->smem_reserved;
    if (allow_compact && ws && ctx->model == MUCA_ISING && staging != MUCA_STAGING_SHARED &&
        ctx->p_pad / 32 > ctx->n_sm && pl.table_smem) {
        const size_t full = used + ws_extra_smem(ctx->model);
        const size_t comp = table + hist + ws_extra_smem(ctx->model, true);
        if (2 * (full + reserved) > per_sm && 2 * (comp + reserved) <= per_sm) {
            pl.compact = true;
            pl.hist_smem = true;
            pl.lattice_smem = false;
            pl.hist_pairs = false;
            pl.smem_bytes = table + hist;
            pl.hist_bytes = hist;
            pl.lat_bytes = 0;
        }
        // More groups than two per SM, and rows of whole words (at least two: the
        // stream decider): the table of the upper 16-bit halves of the thresholds (ties
        // replayed from the 32-bit table) fits a third block per SM.  A block of three
        // per SM takes about 1.26 times as long as one of two per SM (measured at
        // 64 x 64), so three per SM pays when it needs enough fewer waves: at 3 or 6
        // groups per SM, not at 4.
        const size_t table16 = ((size_t)ctx->n_bins * 5 * 2 + 15) & ~(size_t)15;
        const size_t comp16 = table16 + hist + ws_extra_smem(ctx->model, true);
        const long groups = ctx->p_pad / 32, n_sm = ctx->n_sm;
        const long waves2 = (groups + 2 * n_sm - 1) / (2 * n_sm), waves3 = (groups + 3 * n_sm - 1) / (3 * n_sm);
        if (ctx->L % 32 == 0 && ctx->L >= 64 && groups > 2 * n_sm && 126 * waves3 <= 100 * waves2 &&
            3 * (comp16 + reserved) <= per_sm) {
            pl.compact = true;
            pl.t16 = true;
            pl.hist_smem = true;
            pl.lattice_smem = false;
            pl.hist_pairs = false;
            pl.smem_bytes = table16 + hist;
            pl.table_bytes = table16;
            pl.hist_bytes = hist;
            pl.lat_bytes = 0;
        }
    }
    return pl;
}

int plan_flags(const SweepPlan &pl)
{
    return (pl.lattice_smem ? MUCA_PLAN_LATTICE_SMEM : 0) | (pl.hist_smem ? MUCA_PLAN_HIST_SMEM : 0) |
           (pl.table_smem ? MUCA_PLAN_TABLE_SMEM : 0) | (pl.hist_pairs ? MUCA_PLAN_PAIR_HIST : 0) |
           (pl.compact ? MUCA_PLAN_COMPACT : 0) | (pl.warp_specialized ? MUCA_PLAN_WARP_SPECIALIZED : 0) |
           (pl.t16 ? MUCA_PLAN_TABLE16 : 0) | (pl.hist16 ? MUCA_PLAN_HIST16 : 0);
}

int launch_sweeps(muca_ctx *ctx, uint32_t phase, int n_sweeps, uint32_t sweep0, uint32_t iteration, bool hist,
                  int32_t *E_rec, int32_t *M_rec, bool samples)
{
    if (ctx->cfg.ensemble == MUCA_ENSEMBLE_MAGNETIZATION)
        return launch_muma_sweeps(ctx, phase, n_sweeps, sweep0, iteration, hist, E_rec, M_rec);
    SweepPlan pl = plan_sweeps(ctx);
    const bool fast = (ctx->L % 4) == 0;
    if (fast && ctx->ktab_dirty) {
        int rc = launch_ktab(ctx);
        if (rc) return rc;
    }
    if (pl.smem_bytes + (pl.warp_specialized ? ws_extra_smem(ctx->model, pl.compact) : 0) > (size_t)kMaxSmem)
        return fail(MUCA_ERR_ARG, "shared-memory staging does not fit: " + std::to_string(pl.smem_bytes) + " bytes");
    SweepArgs a;
    a.lat = ctx->d_lat;
    a.E = ctx->d_E;
    a.M = ctx->d_M;
    a.cnt = ctx->d_cnt;
    a.thr = ctx->d_thr;
    a.ktab = ctx->d_ktab;
    a.H = ctx->d_H;
    a.samples = samples ? ctx->d_samples : nullptr;
    a.L = ctx->L;
    a.q = ctx->q;
    a.p = ctx->p;
    a.p_pad = ctx->p_pad;
    a.cpg = ctx->cpg;
    a.row_words = ctx->row_words;
    a.lat_words = ctx->lat_words;
    a.n_bins = ctx->n_bins;
    a.iteration = iteration;
    a.ctr3 = ((uint32_t)(ctx->seed >> 32) << 2) | phase;
    a.key0 = (uint32_t)ctx->seed;
    a.rec_stride = ctx->p;
    const int cpb = pl.chains_per_block;
    // warp-specialised kernels: one block per group of cpg chains
    const int blocks = pl.warp_specialized ? (ctx->p + ctx->cpg - 1) / ctx->cpg : (ctx->p + cpb - 1) / cpb;
    // keep every uint32 run length and block-histogram entry below 2^31
    const uint64_t per_sweep = (uint64_t)cpb * ctx->V;
    const int chunk = (int)std::max<uint64_t>(1, std::min<uint64_t>((1ull << 31) / per_sweep, 1u << 30));
    for (int done = 0; done < n_sweeps; done += chunk) {
        const int n = std::min(chunk, n_sweeps - done);
        a.n_sweeps = n;
        a.sweep0 = sweep0 + (uint32_t)done;
        a.E_rec = E_rec ? E_rec + (size_t)done * ctx->p : nullptr;
        a.M_rec = M_rec ? M_rec + (size_t)done * ctx->p : nullptr;
        const bool record = E_rec || M_rec || samples;
        cudaError_t e = pl.warp_specialized ? launch_ws_sweep(a, pl, ctx->model, blocks, hist, record, ctx->stream)
                        : ctx->model == MUCA_ISING ? dispatch_mode<MUCA_ISING>(a, pl, blocks, hist, record, ctx->stream)
                                                   : dispatch_mode<MUCA_POTTS>(a, pl, blocks, hist, record, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel launch");
        note_launches(1);
    }
    return MUCA_OK;
}

int launch_init_lattice(muca_ctx *ctx)
{
    dim3 grid((ctx->p_pad + 127) / 128, ctx->lat_words);
    init_lattice_kernel<<<grid, 128, 0, ctx->stream>>>(ctx->d_lat, ctx->model, ctx->L, ctx->q, ctx->p, ctx->p_pad,
                                                      ctx->row_words, ctx->lat_words, (uint32_t)ctx->seed,
                                                      ((uint32_t)(ctx->seed >> 32) << 2) | kPhaseInit);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return launch_recount(ctx);
}

int launch_recount(muca_ctx *ctx)
{
    recount_kernel<<<(ctx->p + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_lat, ctx->d_E, ctx->d_M, ctx->d_cnt,
                                                                 ctx->model, ctx->L, ctx->q, ctx->p, ctx->p_pad,
                                                                 ctx->row_words);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

int launch_unpack_spins(muca_ctx *ctx, int8_t *d_out)
{
    const size_t total = (size_t)ctx->V * ctx->p;
    const int grid = (int)std::min<size_t>((size_t)ctx->n_sm * 16, (total + 255) / 256);
    unpack_kernel<<<grid, 256, 0, ctx->stream>>>(ctx->d_lat, d_out, ctx->model, ctx->L, ctx->p, ctx->p_pad,
                                                ctx->row_words);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

}  // namespace muca
