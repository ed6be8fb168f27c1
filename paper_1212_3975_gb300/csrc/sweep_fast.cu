// Branch-free sweep kernels for lattices with L % 4 == 0 (every workload of the
// benchmark); other sizes use the general kernels of sweep_kernels.cu.  Same Markov
// chain, same random numbers, same histograms -- bit for bit.
//
// Layout of one attempt (Sec. 3 typewriter order, acceptance of Eq. 1):
//   * sites are handled in groups of 4 with static positions; the Philox block of a
//     group is computed up front, independent of the chain state, so it overlaps
//     with the dependent part of the previous sites;
//   * Ising: the row word is rotated right one bit per site, so the current site is
//     always bit 0 and its right neighbour bit 1 (no variable shifts);
//   * the threshold is read unconditionally from a kernel table indexed directly by
//     the local configuration (Ising: number of unequal neighbours 0..4, Potts:
//     dE + 4), whose dE = 0 column holds the always-accept value 2^32-1;
//   * the run-length histogram flush is a predicated reduction (red.shared /
//     red.global), so no lane ever branches around it.
// The dependent chain per attempt is: left neighbour -> local sum -> table load ->
// compare -> accept; everything else can issue in its shadow.
#include <algorithm>

#include "muca_internal.cuh"

namespace muca {
namespace {

__device__ __forceinline__ void red_add_shared_if(bool p, uint32_t *addr, uint32_t v)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared.add.u32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
        "r"(a), "r"(v)
        : "memory");
}

__device__ __forceinline__ void red_add_global_if(bool p, uint64_t *addr, uint64_t v)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.global.add.u64 [%1], %2;\n\t}" ::"r"((uint32_t)p),
        "l"(addr), "l"(v)
        : "memory");
}

template <bool HSMEM>
__device__ __forceinline__ void flush_if(bool p, uint32_t *s_hist, uint64_t *g_hist, int bin, uint32_t run)
{
    if (HSMEM)
        red_add_shared_if(p, s_hist + bin, run);
    else
        red_add_global_if(p, g_hist + bin, (uint64_t)run);
}

// number of zero bytes of x (exact: no carries between bytes)
__device__ __forceinline__ int zero_bytes(uint32_t x)
{
    const uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    return __popc(~t & 0x80808080u);
}

__device__ __forceinline__ void record_sample(const SweepArgs &a, int sw, int c, int E, int M, int bin)
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

// ---------------------------------------------------------------------------
// Ising
// ---------------------------------------------------------------------------
template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
__global__ void __launch_bounds__(256) ising_fast_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_tab = a.n_bins * 5;
    uint32_t *s_tab = smem;
    uint32_t *s_hist = smem + (TSMEM ? ((n_tab + 3) & ~3) : 0);
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? ((a.n_bins + 3) & ~3) : 0);
    const int cpb = blockDim.x, tid = threadIdx.x;
    const int c = blockIdx.x * cpb + tid;

    if (TSMEM)
        for (int i = tid; i < n_tab; i += cpb) s_tab[i] = a.ktab[i];
    if (HIST && HSMEM)
        for (int i = tid; i < a.n_bins; i += cpb) s_hist[i] = 0u;
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * cpb + tid] = a.lat[(size_t)k * a.p_pad + c];
    __syncthreads();

    uint32_t *lp = LSMEM ? s_lat + tid : a.lat + c;
    const size_t ls = LSMEM ? (size_t)cpb : (size_t)a.p_pad;
#define LAT(k) lp[(size_t)(k) * ls]
#define TAB(i) (TSMEM ? s_tab[(i)] : __ldg(a.ktab + (i)))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L;
        const int last_bits = L - 32 * (RW - 1);
        int bin = (a.E[c] + 2 * V) >> 2;
        int M = 0;
        if (RECORD) {
            int up = 0;
            for (int k = 0; k < a.lat_words; ++k) up += __popc(LAT(k));
            M = 2 * up - V;
        }
        int run_bin = bin;
        uint32_t run = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;  // row above: updated (old for y = 0)
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;  // row below: old (new for y = L-1)
                uint32_t R = LAT(kr), U = LAT(ku), D = LAT(kd);
                uint32_t left = (LAT(kr + RW - 1) >> (last_bits - 1)) & 1u;  // site L-1, old
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w) {
                    const bool lastw = (w == RW - 1);
                    const int nb = lastw ? last_bits : 32;
                    uint32_t Rn = 0u, Un = 0u, Dn = 0u;
                    if (!lastw) {
                        Rn = LAT(kr + w + 1);
                        Un = LAT(ku + w + 1);
                        Dn = LAT(kd + w + 1);
                    }
                    uint32_t ua = R ^ U, ub = R ^ D;  // unequal up / down neighbours
                    for (int g = 0; g < nb; g += 4, site += 4) {
                        const uint4 blk = philox4x32_10(make_uint4((uint32_t)site >> 2, ctr1, a.iteration, a.ctr3),
                                                        a.key0, (uint32_t)c);
                        const bool lastg = (g + 4 == nb);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t u = k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w;
                            const uint32_t s = R & 1u;
                            uint32_t r = (R >> 1) & 1u;
                            // right neighbour of the word's last site: next word (old), or at
                            // the row end site 0 of this row (already updated, maybe in this group)
                            if (k == 3) r = lastg ? (lastw ? first_new : (Rn & 1u)) : r;
                            const uint32_t nneq = (ua & 1u) + (ub & 1u) + (s ^ r) + (s ^ left);
                            const uint32_t A = TAB(bin * 5 + (int)nneq);
                            const bool acc = (u < A) | (A == kAlways);
                            const uint32_t au = acc ? 1u : 0u;
                            R ^= au;
                            bin += acc ? 2 - (int)nneq : 0;
                            if (RECORD) M += acc ? 2 - 4 * (int)s : 0;
                            left = s ^ au;
                            if (k == 0 && w == 0 && g == 0) first_new = left;
                            if (HIST) {
                                const bool fl = bin != run_bin;
                                flush_if<HSMEM>(fl, s_hist, a.H, run_bin, run);
                                run = fl ? 1u : run + 1u;
                                run_bin = bin;
                            }
                            R = __funnelshift_r(R, R, 1);
                            ua >>= 1;
                            ub >>= 1;
                        }
                    }
                    if (nb < 32) R = __funnelshift_r(R, R, 32 - nb);  // back to site order
                    LAT(kr + w) = R;
                    R = Rn;
                    U = Un;
                    D = Dn;
                }
            }
            if (RECORD) record_sample(a, sw, c, 4 * bin - 2 * V, M, bin);
        }
        a.E[c] = 4 * bin - 2 * V;
        if (!RECORD) {
            int up = 0;
            for (int k = 0; k < a.lat_words; ++k) up += __popc(LAT(k));
            M = 2 * up - V;
        }
        a.M[c] = M;
        if (HIST) flush_if<HSMEM>(run != 0u, s_hist, a.H, run_bin, run);
    }
#undef LAT
#undef TAB
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
// 8-state Potts
// ---------------------------------------------------------------------------
__device__ __forceinline__ void potts_counts(uint32_t word, uint32_t (&cnt)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt[k] += zero_bytes(word ^ (0x01010101u * (uint32_t)k));
}

__device__ __forceinline__ void count_move(uint64_t &lo, uint64_t &hi, uint32_t from, uint32_t to)
{
    const uint64_t df = 1ull << (16 * (from & 3u)), dt = 1ull << (16 * (to & 3u));
    if (from < 4) lo -= df; else hi -= df;
    if (to < 4) lo += dt; else hi += dt;
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

template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
__global__ void __launch_bounds__(256) potts_fast_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_tab = a.n_bins * 9;
    uint32_t *s_tab = smem;
    uint32_t *s_hist = smem + (TSMEM ? ((n_tab + 3) & ~3) : 0);
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? ((a.n_bins + 3) & ~3) : 0);
    const int cpb = blockDim.x, tid = threadIdx.x;
    const int c = blockIdx.x * cpb + tid;

    if (TSMEM)
        for (int i = tid; i < n_tab; i += cpb) s_tab[i] = a.ktab[i];
    if (HIST && HSMEM)
        for (int i = tid; i < a.n_bins; i += cpb) s_hist[i] = 0u;
    if (LSMEM && c < a.p_pad)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * cpb + tid] = a.lat[(size_t)k * a.p_pad + c];
    __syncthreads();

    uint32_t *lp = LSMEM ? s_lat + tid : a.lat + c;
    const size_t ls = LSMEM ? (size_t)cpb : (size_t)a.p_pad;
#define LAT(k) lp[(size_t)(k) * ls]
#define TAB(i) (TSMEM ? s_tab[(i)] : __ldg(a.ktab + (i)))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L;
        int bin = a.E[c] + 2 * V;
        uint64_t cnt_lo = 0, cnt_hi = 0;
        if (RECORD) {
            uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < a.lat_words; ++k) potts_counts(LAT(k), cnt);
            for (int k = 0; k < 4; ++k) {
                cnt_lo |= (uint64_t)cnt[k] << (16 * k);
                cnt_hi |= (uint64_t)cnt[k + 4] << (16 * k);
            }
        }
        int run_bin = bin;
        uint32_t run = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;
                uint32_t R = LAT(kr), U = LAT(ku), D = LAT(kd);
                uint32_t left = LAT(kr + RW - 1) >> 24;  // site L-1, old
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w, site += 4) {
                    const bool lastw = (w == RW - 1);
                    uint32_t Rn = 0u, Un = 0u, Dn = 0u;
                    if (!lastw) {
                        Rn = LAT(kr + w + 1);
                        Un = LAT(ku + w + 1);
                        Dn = LAT(kd + w + 1);
                    }
                    const uint4 b0 = philox4x32_10(make_uint4((uint32_t)site >> 1, ctr1, a.iteration, a.ctr3),
                                                   a.key0, (uint32_t)c);
                    const uint4 b1 = philox4x32_10(make_uint4(((uint32_t)site >> 1) + 1u, ctr1, a.iteration, a.ctr3),
                                                   a.key0, (uint32_t)c);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t u = k == 0 ? b0.x : k == 1 ? b0.z : k == 2 ? b1.x : b1.z;
                        const uint32_t pw = k == 0 ? b0.y : k == 1 ? b0.w : k == 2 ? b1.y : b1.w;
                        const uint32_t s = (R >> (8 * k)) & 0xFFu;
                        // right neighbour: next byte; after the word's last site the next word
                        // (old) or, at the row end, site 0 of this row (already updated)
                        const uint32_t r = k < 3 ? (R >> (8 * (k + 1))) & 0xFFu : (lastw ? first_new : (Rn & 0xFFu));
                        const uint32_t sn = (s + 1u + __umulhi(pw, 7u)) & 7u;
                        // neighbours: up, down, left, right as the four bytes of one word
                        const uint32_t ud = __byte_perm(U, D, (uint32_t)(k | ((k + 4) << 4)));
                        const uint32_t nbw = __byte_perm(ud, left | (r << 8), 0x5410u);
                        const int dE = zero_bytes(nbw ^ (0x01010101u * s)) - zero_bytes(nbw ^ (0x01010101u * sn));
                        const uint32_t A = TAB(bin * 9 + dE + 4);
                        const bool acc = (u < A) | (A == kAlways);
                        const uint32_t mask = 0xFFu << (8 * k);
                        R = acc ? ((R & ~mask) | (sn << (8 * k))) : R;
                        bin += acc ? dE : 0;
                        if (RECORD && acc) count_move(cnt_lo, cnt_hi, s, sn);
                        left = acc ? sn : s;
                        if (k == 0 && w == 0) first_new = left;
                        if (HIST) {
                            const bool fl = bin != run_bin;
                            flush_if<HSMEM>(fl, s_hist, a.H, run_bin, run);
                            run = fl ? 1u : run + 1u;
                            run_bin = bin;
                        }
                    }
                    LAT(kr + w) = R;
                    R = Rn;
                    U = Un;
                    D = Dn;
                }
            }
            if (RECORD) record_sample(a, sw, c, bin - 2 * V, 8 * count_max(cnt_lo, cnt_hi) - V, bin);
        }
        a.E[c] = bin - 2 * V;
        if (!RECORD) {
            uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < a.lat_words; ++k) potts_counts(LAT(k), cnt);
            cnt_lo = cnt_hi = 0;
            for (int k = 0; k < 4; ++k) {
                cnt_lo |= (uint64_t)cnt[k] << (16 * k);
                cnt_hi |= (uint64_t)cnt[k + 4] << (16 * k);
            }
        }
        a.M[c] = 8 * count_max(cnt_lo, cnt_hi) - V;
        a.cnt[c] = cnt_lo;
        a.cnt[a.p_pad + c] = cnt_hi;
        if (HIST) flush_if<HSMEM>(run != 0u, s_hist, a.H, run_bin, run);
    }
#undef LAT
#undef TAB
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

// Kernel table from the API table: Ising [bin][nneq 0..4], Potts [bin][dE+4 0..8];
// the dE = 0 column always accepts.
__global__ void ktab_kernel(const uint32_t *thr, uint32_t *ktab, int model, int n_bins)
{
    const int width = model == MUCA_ISING ? 5 : 9;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bins * width) return;
    const int b = t / width, k = t % width;
    uint32_t v;
    if (model == MUCA_ISING) {
        // nneq unequal neighbours -> dE = 8 - 4 nneq; API columns by ascending dE
        v = k == 2 ? kAlways : thr[b * 4 + (k >= 3 ? 4 - k : 3 - k)];
    } else {
        const int dE = k - 4;
        v = dE == 0 ? kAlways : thr[b * 8 + (dE < 0 ? dE + 4 : dE + 3)];
    }
    ktab[t] = v;
}

template <int MODEL, bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
cudaError_t launch_one(const SweepArgs &a, int blocks, int cpb, size_t smem, cudaStream_t st)
{
    auto kern = MODEL == MUCA_ISING ? ising_fast_kernel<HIST, RECORD, TSMEM, HSMEM, LSMEM>
                                    : potts_fast_kernel<HIST, RECORD, TSMEM, HSMEM, LSMEM>;
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

}  // namespace

cudaError_t launch_fast_sweep(const SweepArgs &a, const SweepPlan &pl, int model, int blocks, bool hist,
                              bool record, cudaStream_t st)
{
    if (model == MUCA_ISING) {
        if (hist && record) return dispatch_staging<MUCA_ISING, true, true>(a, pl, blocks, st);
        if (hist) return dispatch_staging<MUCA_ISING, true, false>(a, pl, blocks, st);
        if (record) return dispatch_staging<MUCA_ISING, false, true>(a, pl, blocks, st);
        return dispatch_staging<MUCA_ISING, false, false>(a, pl, blocks, st);
    }
    if (hist && record) return dispatch_staging<MUCA_POTTS, true, true>(a, pl, blocks, st);
    if (hist) return dispatch_staging<MUCA_POTTS, true, false>(a, pl, blocks, st);
    if (record) return dispatch_staging<MUCA_POTTS, false, true>(a, pl, blocks, st);
    return dispatch_staging<MUCA_POTTS, false, false>(a, pl, blocks, st);
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
