// Warp-specialised Ising sweep kernel (L % 4 == 0).
//
// Within one chain every attempt depends on the previous one (the weight depends on
// the global energy), so a chain's speed is set by the length of its own instruction
// stream.  This kernel therefore splits the work of each group of 32 chains over
// three warps of one block, each on its own scheduler:
//   warp 0 (decider): the Markov chain proper -- neighbour sums, threshold load,
//          accept, spin flip.  The table offset for an attempt is chosen between two
//          candidates prepared before the previous accept is known, and both
//          candidate thresholds are loaded speculatively, so only a select and one
//          compare lie between consecutive decisions.
//   warp 1 (producer): the Philox4x32-10 draws (independent of the chain state) of
//          each row word, written to a shared-memory ring ahead of the decider.
//   warp 2 (bookkeeper, iteration and production launches): rebuilds from a
//          per-word snapshot (neighbour sums, flip mask) every attempt's energy bin,
//          fills the block histogram, and writes the (E, M) records.
// Hand-offs use named barriers (bar.sync / bar.arrive) in the classic full/empty
// pattern; every warp runs the same (sweep, row, word) loop nest, so the number of
// arrivals and waits on each barrier match exactly.
// The Markov chain, random numbers and histograms are identical to the oracle's.
#include <algorithm>

#include "muca_internal.cuh"

namespace muca {
namespace {

constexpr int kRingU = 4;   // slots of Philox draws (one row word each)
constexpr int kRingS = 3;   // slots of bookkeeping snapshots
constexpr int kBarFullU = 1, kBarEmptyU = kBarFullU + kRingU;      // ids 1..8
constexpr int kBarFullS = kBarEmptyU + kRingU, kBarEmptyS = kBarFullS + kRingS;  // ids 9..14
static_assert(kBarEmptyS + kRingS <= 16, "named barrier ids");

__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Table loads as explicit instructions: both candidate thresholds must really be
// loaded before the previous accept is known (a compiler may otherwise turn
// "cond ? load(a) : load(b)" into "load(cond ? a : b)", which puts the load back on
// the dependent chain).
__device__ __forceinline__ uint32_t lds_u32(uint32_t saddr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
    return v;
}
__device__ __forceinline__ uint32_t ldg_nc_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void red_shared(uint32_t *addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(addr)), "r"(v));
}

// snapshot of one row word for the bookkeeper (per lane)
struct Snap {
    uint32_t lo, hi;   // bit-sliced sum of the unequal up, down and right neighbours
    uint32_t qw;       // site differs from its old left neighbour
    uint32_t flip;     // sites whose spin flipped (= accepted attempts)
    uint32_t rold;     // spins before the word was swept
    uint32_t pad[3];
};

template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
__global__ void __launch_bounds__(128) ising_ws_kernel(SweepArgs a)
{
    constexpr bool BOOK = HIST || RECORD;
    constexpr int NP = BOOK ? 2 : 3;            // producer warps (one SM sub-partition each)
    constexpr int NT = 128;                     // decider + producers (+ bookkeeper)
    constexpr int NU = 32 * (1 + NP);           // threads on the draw-ring barriers
    constexpr int BOOK_WARP = 1 + NP;
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_tab = a.n_bins * 5;
    uint32_t *s_tab = smem;
    uint32_t *s_hist = smem + (TSMEM ? ((n_tab + 3) & ~3) : 0);
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? ((a.n_bins + 3) & ~3) : 0);
    uint4 *s_ring = reinterpret_cast<uint4 *>(s_lat + (LSMEM ? a.lat_words * 32 : 0));  // [kRingU][8][32]
    Snap *s_snap = reinterpret_cast<Snap *>(s_ring + kRingU * 8 * 32);                   // [kRingS][32]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = blockIdx.x * 32 + lane;
    const bool active = c < a.p;

    if (TSMEM)
        for (int i = tid; i < n_tab; i += NT) s_tab[i] = a.ktab[i];
    if (HIST && HSMEM)
        for (int i = tid; i < a.n_bins; i += NT) s_hist[i] = 0u;
    if (LSMEM && warp == 0)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * 32 + lane] = a.lat[(size_t)k * a.p_pad + c];
    // production launches: magnetisation at the start, read before the decider
    // touches the lattice
    int M_start = 0;
    if (RECORD && warp == BOOK_WARP && active) {
        int up = 0;
        for (int k = 0; k < a.lat_words; ++k) up += __popc(a.lat[(size_t)k * a.p_pad + c]);
        M_start = 2 * up - a.L * a.L;
    }
    __syncthreads();

    const int L = a.L, RW = a.row_words, V = L * L;
    const int last_bits = L - 32 * (RW - 1);
    const int total = a.n_sweeps * L * RW;  // row words per launch, identical for all warps

    if (warp >= 1 && warp <= NP) {
        // ---------------- producers: Philox draws, clamped to 2^32-2 ------------
        // producer pr computes the blocks gi = pr, pr + NP, ... of every row word
        const int pr = warp - 1;
        uint32_t k1r[10];
        philox_round_keys((uint32_t)c, k1r);
        int it = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = a.sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                for (int w = 0; w < RW; ++w, ++it) {
                    const int nb = (w == RW - 1) ? last_bits : 32;
                    const int slot = it % kRingU;
                    if (it >= kRingU) bar_sync(kBarEmptyU + slot, NU);
                    uint4 *dst = s_ring + slot * 8 * 32 + lane;
                    // the word's blocks are independent: unrolled so that their 10-round
                    // dependency chains interleave
#pragma unroll 4
                    for (int gi = pr; gi < (nb >> 2); gi += NP) {
                        uint4 b = philox4x32_10_rk(make_uint4((uint32_t)(site >> 2) + (uint32_t)gi, ctr1, a.iteration,
                                                              a.ctr3),
                                                   a.key0, k1r);
                        // clamped so that u < A decides (A = 2^32-1 always accepts);
                        // padding chains get 2^32-1, which never accepts
                        const uint32_t cap = active ? 0xFFFFFFFEu : 0xFFFFFFFFu;
                        b.x = active ? min(b.x, cap) : cap;
                        b.y = active ? min(b.y, cap) : cap;
                        b.z = active ? min(b.z, cap) : cap;
                        b.w = active ? min(b.w, cap) : cap;
                        dst[gi * 32] = b;
                    }
                    site += nb;
                    bar_arrive(kBarFullU + slot, NU);
                }
            }
        }
    } else if (warp == 0) {
        // ---------------- decider: the Markov chain -----------------------------
        uint32_t *lp = LSMEM ? s_lat + lane : a.lat + c;
        const size_t ls = LSMEM ? (size_t)32 : (size_t)a.p_pad;
#define LAT(k) lp[(size_t)(k) * ls]
        const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(s_tab);
#define TAB_BYTES(o)                 \
    (TSMEM ? lds_u32(tab_s + (o))    \
           : ldg_nc_u32(reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(a.ktab) + (o))))
        const int bin0 = active ? (a.E[c] + 2 * V) >> 2 : (V >> 1);
        uint32_t bin20 = 20u * (uint32_t)bin0;  // 4*5*bin before the previous decision
        uint32_t d20p = 0u;                     // its change if the previous attempt was accepted
        bool ap = false;                        // previous attempt accepted
        int it = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW;
                const int ku = (y == 0 ? L - 1 : y - 1) * RW;  // row above: updated (old for y = 0)
                const int kd = (y == L - 1 ? 0 : y + 1) * RW;  // row below: old (new for y = L-1)
                uint32_t R = LAT(kr), U = LAT(ku), D = LAT(kd);
                uint32_t lbit = (LAT(kr + RW - 1) >> (last_bits - 1)) & 1u;  // site L-1, old
                uint32_t first_new = 0u;
                for (int w = 0; w < RW; ++w, ++it) {
                    const bool lastw = (w == RW - 1);
                    const int nb = lastw ? last_bits : 32;
                    uint32_t Rn = 0u, Un = 0u, Dn = 0u;
                    if (!lastw) {
                        Rn = LAT(kr + w + 1);
                        Un = LAT(ku + w + 1);
                        Dn = LAT(kd + w + 1);
                    }
                    const uint32_t ua = R ^ U, ub = R ^ D;
                    const uint32_t tr = R ^ ((R >> 1) | ((Rn & 1u) << 31));
                    uint32_t lo = ua ^ ub ^ tr;
                    uint32_t hi = (ua & ub) | (tr & (ua ^ ub));
                    const uint32_t qw = R ^ ((R << 1) | lbit);
                    const int slot = it % kRingU;
                    bar_sync(kBarFullU + slot, NU);
                    const uint4 *src = s_ring + slot * 8 * 32 + lane;
                    uint32_t Rw = R;
                    if (nb == 32) {
                        // Full word, software-pipelined: while site j decides, the two
                        // candidate thresholds of site j+1 are loaded (their offsets are
                        // resolved by site j-1's decision).  State: P0/P1 = 20 * bin
                        // before this site's decision if the previous attempt was
                        // rejected / accepted.
                        uint32_t P0 = bin20, P1 = bin20 + d20p;
                        uint32_t K0n, K1n, D0n, D1n;  // of the next site
                        auto site_consts = [&](int j, uint32_t &K0, uint32_t &K1, uint32_t &D0, uint32_t &D1) {
                            uint32_t pre = ((lo >> j) & 1u) + ((hi >> j) & 1u) * 2u;
                            if (j == 31) {
                                // row end (last word): right neighbour is site 0, already updated
                                const uint32_t pre_end =
                                    ((ua >> 31) & 1u) + ((ub >> 31) & 1u) + ((R >> 31) ^ first_new);
                                pre = lastw ? pre_end : pre;
                            }
                            const uint32_t q = (qw >> j) & 1u;
                            const uint32_t n0 = pre + q;
                            const uint32_t n1 = (j == 0 && w == 0) ? n0 : pre + 1u - q;
                            K0 = tab_s + 4u * n0;
                            K1 = tab_s + 4u * n1;
                            D0 = 40u - 20u * n0;
                            D1 = 40u - 20u * n1;
                        };
                        uint32_t K0, K1, D0, D1;
                        site_consts(0, K0, K1, D0, D1);
                        uint32_t A0 = TSMEM ? lds_u32(P0 + K0) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                                      reinterpret_cast<const char *>(a.ktab) + P0 + K0 - tab_s));
                        uint32_t A1 = TSMEM ? lds_u32(P1 + K1) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                                      reinterpret_cast<const char *>(a.ktab) + P1 + K1 - tab_s));
                        uint4 blk = src[0];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int k = j & 3;
                            if (k == 0 && j > 0) blk = src[(j >> 2) * 32];
                            const uint32_t u = k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w;
                            // Issue order matters (a warp issues in order): first the loads
                            // of site j+1, whose offsets need only the previous decision,
                            // then the decision of site j, which waits for its own loads.
                            uint32_t A0n = 0u, A1n = 0u;
                            if (j < 31) {
                                site_consts(j + 1, K0n, K1n, D0n, D1n);
                                const uint32_t o0 = ap ? P1 + K0n : P0 + K0n;
                                const uint32_t o1 = ap ? P1 + D1 + K1n : P0 + D0 + K1n;
                                A0n = TSMEM ? lds_u32(o0) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                               reinterpret_cast<const char *>(a.ktab) + o0 - tab_s));
                                A1n = TSMEM ? lds_u32(o1) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                               reinterpret_cast<const char *>(a.ktab) + o1 - tab_s));
                            }
                            const uint32_t A = ap ? A1 : A0;
                            const bool acc = u < A;
                            const uint32_t nP0 = ap ? P1 : P0;
                            const uint32_t nP1 = ap ? P1 + D1 : P0 + D0;
                            A0 = A0n;
                            A1 = A1n;
                            P0 = nP0;
                            P1 = nP1;
                            D0 = D0n;
                            D1 = D1n;
                            Rw ^= acc ? (1u << j) : 0u;
                            if (j == 0 && w == 0) first_new = (R & 1u) ^ (acc ? 1u : 0u);
                            ap = acc;
                        }
                        // back to the (bin20, d20p) form at the word boundary
                        bin20 = P0;
                        d20p = P1 - P0;
                    } else
                    for (int g = 0; g < nb; g += 4) {
                        uint4 blk = src[(g >> 2) * 32];
                        const uint4 nxt = (g + 4 < nb) ? src[((g >> 2) + 1) * 32] : blk;
                        const bool lastg = lastw && (g + 4 == nb);
                        const uint32_t log_ = lo >> g, hig = hi >> g, qg = qw >> g;
                        const uint32_t uag = ua >> g, ubg = ub >> g, Rg = R >> g;
                        const uint32_t gbit = 1u << g;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t u = k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w;
                            uint32_t pre = ((log_ >> k) & 1u) + ((hig >> k) & 1u) * 2u;
                            if (k == 3) {
                                // row end: the right neighbour is site 0, already updated
                                const uint32_t pre_end =
                                    ((uag >> 3) & 1u) + ((ubg >> 3) & 1u) + (((Rg >> 3) & 1u) ^ first_new);
                                pre = lastg ? pre_end : pre;
                            }
                            const uint32_t q = (qg >> k) & 1u;
                            const bool rowstart = (k == 0) && (w == 0) && (g == 0);
                            const uint32_t n0 = pre + q;
                            const uint32_t n1 = rowstart ? n0 : pre + 1u - q;
                            const uint32_t b1o = bin20 + d20p;
                            const uint32_t A0 = TAB_BYTES(bin20 + 4u * n0);
                            const uint32_t A1 = TAB_BYTES(b1o + 4u * n1);
                            const uint32_t A = ap ? A1 : A0;
                            const bool acc = active && (u < A);
                            const uint32_t nneq = ap ? n1 : n0;
                            bin20 = ap ? b1o : bin20;
                            d20p = 40u - 20u * nneq;
                            Rw ^= acc ? (gbit << k) : 0u;
                            if (k == 0 && w == 0 && g == 0) first_new = (R & 1u) ^ (acc ? 1u : 0u);
                            ap = acc;
                        }
                        blk = nxt;
                    }
                    if (it < total - kRingU) bar_arrive(kBarEmptyU + slot, NU);
                    LAT(kr + w) = Rw;
                    if (BOOK) {
                        if (lastw) {
                            // the row's last site saw the updated site 0 as its right neighbour
                            const uint32_t bitm = 1u << (nb - 1);
                            const uint32_t tr2 = (tr & ~bitm) | ((((R >> (nb - 1)) & 1u) ^ first_new) << (nb - 1));
                            lo = ua ^ ub ^ tr2;
                            hi = (ua & ub) | (tr2 & (ua ^ ub));
                        }
                        const int ss = it % kRingS;
                        if (it >= kRingS) bar_sync(kBarEmptyS + ss, 64);
                        Snap *sn = s_snap + ss * 32 + lane;
                        sn->lo = lo;
                        sn->hi = hi;
                        sn->qw = qw;
                        sn->flip = R ^ Rw;
                        sn->rold = R;
                        bar_arrive(kBarFullS + ss, 64);
                    }
                    lbit = R >> 31;
                    R = Rn;
                    U = Un;
                    D = Dn;
                }
            }
        }
        if (active && !BOOK) {
            // no bookkeeper: apply the pending decision and recount M
            const uint32_t bin_end = (ap ? bin20 + d20p : bin20) / 20u;
            a.E[c] = 4 * (int)bin_end - 2 * V;
            int up = 0;
            for (int k = 0; k < a.lat_words; ++k) up += __popc(LAT(k));
            a.M[c] = 2 * up - V;
        }
#undef TAB_BYTES
        if (LSMEM)
            for (int k = 0; k < a.lat_words; ++k) a.lat[(size_t)k * a.p_pad + c] = s_lat[k * 32 + lane];
#undef LAT
    } else if (BOOK && warp == BOOK_WARP) {
        // ---------------- bookkeeper: bins, histogram, records -------------------
        int bin = active ? (a.E[c] + 2 * V) >> 2 : (V >> 1);
        int M = M_start;
        int run_bin = bin;
        uint32_t run = 0;
        int it = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            for (int y = 0; y < L; ++y) {
                uint32_t pflip = 0u;  // flip of the previous site in this row
                for (int w = 0; w < RW; ++w, ++it) {
                    const int nb = (w == RW - 1) ? last_bits : 32;
                    const int ss = it % kRingS;
                    bar_sync(kBarFullS + ss, 64);
                    const Snap sn = s_snap[ss * 32 + lane];
                    if (it < total - kRingS) bar_arrive(kBarEmptyS + ss, 64);
                    // left neighbour as seen by each site: old left, flipped if the
                    // previous site flipped (not across the row start)
                    const uint32_t lf = (sn.flip << 1) | pflip;
                    const uint32_t qn = sn.qw ^ lf;
                    auto book_site = [&](int j) {
                        const int nneq = (int)(((sn.lo >> j) & 1u) + 2u * ((sn.hi >> j) & 1u) + ((qn >> j) & 1u));
                        const bool acc = (sn.flip >> j) & 1u;
                        bin += acc ? 2 - nneq : 0;
                        if (HIST && active) {
                            if (HSMEM) {
                                red_shared(s_hist + bin, 1u);
                            } else {
                                if (bin != run_bin) {
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]),
                                              (unsigned long long)run);
                                    run_bin = bin;
                                    run = 0;
                                }
                                ++run;
                            }
                        }
                    };
                    if (nb == 32) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) book_site(j);
                    } else {
                        for (int j = 0; j < nb; ++j) book_site(j);
                    }
                    if (RECORD) {
                        const uint32_t f = sn.flip;
                        M += 2 * (__popc(f & ~sn.rold) - __popc(f & sn.rold));
                    }
                    pflip = (sn.flip >> (nb - 1)) & 1u;
                }
            }
            if (RECORD && active) {
                const int E = 4 * bin - 2 * V;
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
        }
        if (active) {
            if (HIST && !HSMEM && run)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]), (unsigned long long)run);
            a.E[c] = 4 * bin - 2 * V;
            if (RECORD) a.M[c] = M;
        }
    }
    __syncthreads();
    if (BOOK && !RECORD && warp == 0 && active) {
        // iteration launches: magnetisation recount from the final lattice
        int up = 0;
        for (int k = 0; k < a.lat_words; ++k) up += __popc(a.lat[(size_t)k * a.p_pad + c]);
        a.M[c] = 2 * up - V;
    }
    if (HIST && HSMEM) {
        for (int i = tid; i < a.n_bins; i += NT) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}

template <bool HIST, bool RECORD, bool TSMEM, bool HSMEM, bool LSMEM>
cudaError_t launch_ws(const SweepArgs &a, int blocks, size_t smem, cudaStream_t st)
{
    auto kern = ising_ws_kernel<HIST, RECORD, TSMEM, HSMEM, LSMEM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, 128, smem, st>>>(a);
    return cudaGetLastError();
}

template <bool HIST, bool RECORD>
cudaError_t ws_staging(const SweepArgs &a, const SweepPlan &pl, int blocks, size_t smem, cudaStream_t st)
{
    const int key = (pl.table_smem ? 4 : 0) | ((HIST && pl.hist_smem) ? 2 : 0) | (pl.lattice_smem ? 1 : 0);
    switch (key) {
    case 0: return launch_ws<HIST, RECORD, false, false, false>(a, blocks, smem, st);
    case 1: return launch_ws<HIST, RECORD, false, false, true>(a, blocks, smem, st);
    case 2: return launch_ws<HIST, RECORD, false, true, false>(a, blocks, smem, st);
    case 3: return launch_ws<HIST, RECORD, false, true, true>(a, blocks, smem, st);
    case 4: return launch_ws<HIST, RECORD, true, false, false>(a, blocks, smem, st);
    case 5: return launch_ws<HIST, RECORD, true, false, true>(a, blocks, smem, st);
    case 6: return launch_ws<HIST, RECORD, true, true, false>(a, blocks, smem, st);
    default: return launch_ws<HIST, RECORD, true, true, true>(a, blocks, smem, st);
    }
}

}  // namespace

// shared memory of the warp-specialised kernel beyond the staging of the plan
size_t ws_extra_smem() { return (size_t)kRingU * 8 * 32 * sizeof(uint4) + (size_t)kRingS * 32 * sizeof(Snap); }

cudaError_t launch_ising_ws(const SweepArgs &a, const SweepPlan &pl, int blocks, bool hist, bool record,
                            cudaStream_t st)
{
    const size_t smem = pl.smem_bytes + ws_extra_smem();
    if (hist && record) return ws_staging<true, true>(a, pl, blocks, smem, st);
    if (hist) return ws_staging<true, false>(a, pl, blocks, smem, st);
    if (record) return ws_staging<false, true>(a, pl, blocks, smem, st);
    return ws_staging<false, false>(a, pl, blocks, smem, st);
}

}  // namespace muca
