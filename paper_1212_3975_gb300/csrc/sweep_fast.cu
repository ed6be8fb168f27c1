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

// Predicated reductions.  No "memory" clobber: the compiler may move the (unrelated)
// table loads across them; the block's histogram is only read after __syncthreads(),
// whose bar.sync orders all earlier shared-memory operations of the block.
__device__ __forceinline__ void red_add_shared_if(bool p, uint32_t *addr, uint32_t v)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared.add.u32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
        "r"(a), "r"(v));
}

__device__ __forceinline__ void red_add_global_if(bool p, uint64_t *addr, uint64_t v)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.global.add.u64 [%1], %2;\n\t}" ::"r"((uint32_t)p),
        "l"(addr), "l"(v));
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
#define TAB_BYTES(o)                                                         \
    (TSMEM ? *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(s_tab) + (o)) \
           : __ldg(reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(a.ktab) + (o))))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L;
        const int last_bits = L - 32 * (RW - 1);
        int bin = (a.E[c] + 2 * V) >> 2;  // bin after the latest attempt
        uint32_t k1r[10];
        philox_round_keys((uint32_t)c, k1r);
        int M = 0;
        if (RECORD) {
            int up = 0;
            for (int k = 0; k < a.lat_words; ++k) up += __popc(LAT(k));
            M = 2 * up - V;
        }
        // Deferred form of the chain state: the table offset of an attempt is selected
        // between two candidates computed before the previous accept is known.
        uint32_t bin20 = 20u * (uint32_t)bin;  // 4*5*bin before the previous decision
        uint32_t d20p = 0u;                    // its change if the previous attempt was accepted
        bool ap = false;                       // previous attempt accepted
        int run_bin = bin;
        uint32_t run = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            uint4 blk = philox4x32_10_rk(make_uint4(0u, ctr1, a.iteration, a.ctr3), a.key0, k1r);
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;  // row above: updated (old for y = 0)
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;  // row below: old (new for y = L-1)
                uint32_t R = LAT(kr), U = LAT(ku), D = LAT(kd);
                uint32_t lbit = (LAT(kr + RW - 1) >> (last_bits - 1)) & 1u;  // site L-1, old
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
                    // bit-sliced per-site sums of the neighbours that do not depend on
                    // this row's decisions: unequal up, down and right (old) neighbours
                    const uint32_t ua = R ^ U, ub = R ^ D;
                    const uint32_t tr = R ^ ((R >> 1) | ((Rn & 1u) << 31));
                    const uint32_t lo = ua ^ ub ^ tr;
                    const uint32_t hi = (ua & ub) | (tr & (ua ^ ub));
                    // old left neighbour differs from the site (left = site L-1 for x = 0)
                    const uint32_t qw = R ^ ((R << 1) | lbit);
                    uint32_t Rw = R;
                    for (int g = 0; g < nb; g += 4, site += 4) {
                        const uint4 nxt = philox4x32_10_rk(make_uint4(((uint32_t)site >> 2) + 1u, ctr1, a.iteration,
                                                                   a.ctr3),
                                                        a.key0, k1r);
                        const bool lastg = lastw && (g + 4 == nb);
                        const uint32_t log_ = lo >> g, hig = hi >> g, qg = qw >> g;
                        const uint32_t uag = ua >> g, ubg = ub >> g, Rg = R >> g;
                        const uint32_t gbit = 1u << g;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t u = min(k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w,
                                                   0xFFFFFFFEu);  // then u < A decides, A = 2^32-1 included
                            uint32_t pre = ((log_ >> k) & 1u) + ((hig >> k) & 1u) * 2u;
                            if (k == 3) {
                                // last site of the row: its right neighbour is site 0, already updated
                                const uint32_t pre_end =
                                    ((uag >> 3) & 1u) + ((ubg >> 3) & 1u) + (((Rg >> 3) & 1u) ^ first_new);
                                pre = lastg ? pre_end : pre;
                            }
                            const uint32_t q = (qg >> k) & 1u;
                            const bool rowstart = (k == 0) && (w == 0) && (g == 0);
                            const uint32_t n0 = pre + q;                          // previous attempt rejected
                            const uint32_t n1 = rowstart ? n0 : pre + 1u - q;     // previous attempt accepted
                            const uint32_t b1 = bin20 + d20p;
                            const uint32_t off = ap ? b1 + 4u * n1 : bin20 + 4u * n0;
                            const uint32_t A = TAB_BYTES(off);
                            const bool acc = u < A;
                            const uint32_t nneq = ap ? n1 : n0;
                            bin20 = ap ? b1 : bin20;
                            d20p = 40u - 20u * nneq;
                            bin += acc ? 2 - (int)nneq : 0;
                            if (RECORD) M += acc ? 2 - 4 * (int)((Rg >> k) & 1u) : 0;
                            if (k == 0 && w == 0 && g == 0) first_new = (R & 1u) ^ (acc ? 1u : 0u);
                            Rw ^= acc ? (gbit << k) : 0u;
                            if (HIST) {
                                if (HSMEM) {
                                    red_add_shared_if(true, s_hist + bin, 1u);
                                } else {
                                    const bool fl = bin != run_bin;
                                    flush_if<false>(fl, s_hist, a.H, run_bin, run);
                                    run = fl ? 1u : run + 1u;
                                    run_bin = bin;
                                }
                            }
                            ap = acc;
                        }
                        blk = nxt;
                    }
                    LAT(kr + w) = Rw;
                    lbit = R >> 31;
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
#undef TAB_BYTES
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
#define TAB_BYTES(o)                                                         \
    (TSMEM ? *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(s_tab) + (o)) \
           : __ldg(reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(a.ktab) + (o))))

    if (c < a.p) {
        const int L = a.L, RW = a.row_words, V = L * L;
        int bin = a.E[c] + 2 * V;
        uint32_t k1r[10];
        philox_round_keys((uint32_t)c, k1r);
        uint64_t cnt_lo = 0, cnt_hi = 0;
        if (RECORD) {
            uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < a.lat_words; ++k) potts_counts(LAT(k), cnt);
            for (int k = 0; k < 4; ++k) {
                cnt_lo |= (uint64_t)cnt[k] << (16 * k);
                cnt_hi |= (uint64_t)cnt[k + 4] << (16 * k);
            }
        }
        // deferred chain state (see the Ising kernel): offsets in bytes of the
        // [bin][dE+4] kernel table, 36 bytes per bin
        uint32_t bin36 = 36u * (uint32_t)bin;
        uint32_t d36p = 0u;
        bool ap = false;
        int run_bin = bin;
        uint32_t run = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            uint4 b0 = philox4x32_10_rk(make_uint4(0u, ctr1, a.iteration, a.ctr3), a.key0, k1r);
            uint4 b1 = philox4x32_10_rk(make_uint4(1u, ctr1, a.iteration, a.ctr3), a.key0, k1r);
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;
                uint32_t R = LAT(kr), U = LAT(ku), D = LAT(kd);
                // candidates for the left neighbour: previous site unchanged / changed
                uint32_t left0 = LAT(kr + RW - 1) >> 24;  // site L-1, old
                uint32_t left1 = left0;
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w, site += 4) {
                    const bool lastw = (w == RW - 1);
                    uint32_t Rn = 0u, Un = 0u, Dn = 0u;
                    if (!lastw) {
                        Rn = LAT(kr + w + 1);
                        Un = LAT(ku + w + 1);
                        Dn = LAT(kd + w + 1);
                    }
                    // random numbers of the next word, independent of the chain state
                    const uint4 n0 = philox4x32_10_rk(make_uint4(((uint32_t)site >> 1) + 2u, ctr1, a.iteration, a.ctr3),
                                                   a.key0, k1r);
                    const uint4 n1 = philox4x32_10_rk(make_uint4(((uint32_t)site >> 1) + 3u, ctr1, a.iteration, a.ctr3),
                                                   a.key0, k1r);
                    uint32_t Rw = R;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t u = min(k == 0 ? b0.x : k == 1 ? b0.z : k == 2 ? b1.x : b1.z, 0xFFFFFFFEu);
                        const uint32_t pw = k == 0 ? b0.y : k == 1 ? b0.w : k == 2 ? b1.y : b1.w;
                        const uint32_t s = (R >> (8 * k)) & 0xFFu;
                        // right neighbour: next byte; after the word's last site the next word
                        // (old) or, at the row end, site 0 of this row (already updated)
                        const uint32_t r = k < 3 ? (R >> (8 * (k + 1))) & 0xFFu : (lastw ? first_new : (Rn & 0xFFu));
                        const uint32_t sn = (s + 1u + __umulhi(pw, 7u)) & 7u;
                        // up, down, right neighbours as bytes 0..2; byte 3 never matches a state
                        const uint32_t ud = __byte_perm(U, D, (uint32_t)(k | ((k + 4) << 4)));
                        const uint32_t nb3 = __byte_perm(ud, r | 0xFF00u, 0x5410u);
                        const int base = zero_bytes(nb3 ^ (0x01010101u * s)) - zero_bytes(nb3 ^ (0x01010101u * sn));
                        const int dE0 = base + (left0 == s) - (left0 == sn);
                        const int dE1 = base + (left1 == s) - (left1 == sn);
                        const uint32_t b1o = bin36 + d36p;
                        const uint32_t off = ap ? b1o + 4u * (uint32_t)(dE1 + 4) : bin36 + 4u * (uint32_t)(dE0 + 4);
                        const uint32_t A = TAB_BYTES(off);
                        const bool acc = u < A;
                        const int dE = ap ? dE1 : dE0;
                        bin36 = ap ? b1o : bin36;
                        d36p = (uint32_t)(36 * dE);
                        bin += acc ? dE : 0;
                        const uint32_t mask = 0xFFu << (8 * k);
                        Rw = acc ? ((Rw & ~mask) | (sn << (8 * k))) : Rw;
                        if (RECORD && acc) count_move(cnt_lo, cnt_hi, s, sn);
                        if (k == 0 && w == 0) first_new = acc ? sn : s;
                        left0 = s;
                        left1 = sn;
                        if (HIST) {
                            if (HSMEM) {
                                red_add_shared_if(true, s_hist + bin, 1u);
                            } else {
                                const bool fl = bin != run_bin;
                                flush_if<false>(fl, s_hist, a.H, run_bin, run);
                                run = fl ? 1u : run + 1u;
                                run_bin = bin;
                            }
                        }
                        ap = acc;
                    }
                    LAT(kr + w) = Rw;
                    b0 = n0;
                    b1 = n1;
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
#undef TAB_BYTES
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
