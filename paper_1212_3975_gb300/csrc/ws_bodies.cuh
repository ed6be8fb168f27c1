// Warp-specialised sweep bodies (L % 4 == 0), shared by the standalone kernels
// and the persistent batched kernel.
//
// Ising:
//
// Within one chain every attempt depends on the previous one (the weight depends on
// the global energy), so a chain's speed is set by the length of its own instruction
// stream.  This kernel therefore splits the work of each group of 32 chains over the
// four warps of one block, each on its own scheduler:
//   warp 0 (decider): the Markov chain proper -- neighbour sums, threshold load,
//          accept, spin flip.  The table offset for an attempt is chosen between two
//          candidates prepared before the previous accept is known, and both
//          candidate thresholds are loaded speculatively, so only a select and one
//          compare lie between consecutive decisions.
//   warps 1..3 (producers; 1..2 when warp 3 keeps the books): the Philox4x32-10
//          draws (independent of the chain state) of each row word, written to a
//          shared-memory ring ahead of the decider.
//   warp 3 (bookkeeper, iteration and production launches): rebuilds from
//          snapshots (neighbour sums, flip mask; two row words per hand-off) every
//          attempt's energy bin, fills the block histogram (one count per attempt, per
//          pair of consecutive attempts, or 16-bit counts flushed by rows), and writes
//          the (E, M) records.
// A group holds up to 32 chains (fewer when small p is spread over every SM); the
// stagings of the table, histogram and lattices range from everything in shared
// memory (one block per SM) over the compact staging (two blocks per SM) to the
// table of 16-bit threshold halves (three blocks per SM, ties replayed exactly).
//
// 8-state Potts (further below): decider, three producers (draws, proposals and the
// byte-parallel column counts of the neighbours fixed in advance) and, for iterations
// and production, a bookkeeper; rows of whole ring slots run the slot decider.
//
// Hand-offs use named barriers (bar.sync / bar.arrive) in the classic full/empty
// pattern; every warp runs the same (sweep, row, word) loop nest, so the number of
// arrivals and waits on each barrier match exactly.
// The Markov chain, random numbers and histograms are identical to the oracle's.
#pragma once
#include <algorithm>

#include "muca_internal.cuh"

namespace muca {
namespace ws {

constexpr int kRingU = 4;   // slots of Philox draws (one row word each)
constexpr int kRingS = 3;   // slots of bookkeeping snapshots
constexpr int kSnapWords = 2;  // Ising: row words per snapshot slot (one hand-off per pair)
constexpr int kCompactRing = 3;  // draw-ring slots of the compact Ising staging
constexpr int kHistDummy = 32;   // histogram slots of inactive lanes (one per lane)
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
__device__ __forceinline__ uint32_t lds_u16(uint32_t saddr)
{
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(saddr));
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
};  // 20 bytes: a lane stride of 5 words, so a warp's accesses of one field hit 32 banks
static_assert(sizeof(Snap) == 20, "snapshot layout");

// Neighbour planes of one row word: lo/hi = bit-sliced count of the unequal up, down
// and right neighbours, qw = site differs from its old left neighbour.
struct WordCtx {
    uint32_t R, Rn;        // the word and its right neighbour word (old values)
    uint32_t ua, ub, tr;   // unequal up / down / right
    uint32_t lo, hi, qw;
};

__device__ __forceinline__ WordCtx word_ctx(uint32_t R, uint32_t U, uint32_t D, uint32_t Rn, uint32_t lbit)
{
    WordCtx x;
    x.R = R;
    x.Rn = Rn;
    x.ua = R ^ U;
    x.ub = R ^ D;
    x.tr = R ^ ((R >> 1) | ((Rn & 1u) << 31));
    x.lo = x.ua ^ x.ub ^ x.tr;
    x.hi = (x.ua & x.ub) | (x.tr & (x.ua ^ x.ub));
    x.qw = R ^ ((R << 1) | lbit);
    return x;
}

// Byte k of x, zero-extended / sign-extended (prmt: a selector nibble with its top bit
// set replicates the sign of the byte it names).
__device__ __forceinline__ uint32_t ubyte(uint32_t x, int k)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "r"(0x4440u | (uint32_t)k));
    return d;
}
__device__ __forceinline__ uint32_t sbyte(uint32_t x, int k)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "r"((uint32_t)k | (8u | (uint32_t)k) * 0x1110u));
    return d;
}

// Site constants of four consecutive sites of a word, one site per byte: the table
// offsets 4 n0 / 4 n1 (n = number of unequal neighbours with the left neighbour old /
// flipped) and the bin changes 40 - 20 n0 / 40 - 20 n1 (bytes of the table, 20 per
// bin) as signed bytes.
struct Quad {
    uint32_t K0, K1, D0, D1;
};

// bits 4g..4g+3 of x, bit i to bit 8i + s
__device__ __forceinline__ uint32_t spread4(uint32_t x, int g, int s)
{
    return (((x >> (4 * g)) & 0xFu) * (0x00204081u << s)) & (0x01010101u << s);
}

__device__ __forceinline__ Quad site_quad(const WordCtx &x, int g, bool rowstart)
{
    const uint32_t pre4 = spread4(x.lo, g, 2) + spread4(x.hi, g, 3);  // 4 x (up + down + right)
    const uint32_t q4 = spread4(x.qw, g, 2);
    Quad r;
    r.K0 = pre4 + q4;
    r.K1 = pre4 + 0x04040404u - q4;
    // site 0 of a row: its left neighbour (site L-1) is not visited yet
    if (rowstart) r.K1 = (r.K1 & 0xFFFFFF00u) | (r.K0 & 0xFFu);
    // per byte 168 - 5 K >= 88: no borrow; xor 0x80 recentres to 40 - 20 n
    r.D0 = (0xA8A8A8A8u - 5u * r.K0) ^ 0x80808080u;
    r.D1 = (0xA8A8A8A8u - 5u * r.K1) ^ 0x80808080u;
    return r;
}

// The same constants for the table of 16-bit entries (threshold upper halves): offsets
// 2 n0 / 2 n1 and bin changes 20 - 10 n (10 bytes per bin row).
__device__ __forceinline__ Quad site_quad16(const WordCtx &x, int g, bool rowstart)
{
    const uint32_t pre2 = spread4(x.lo, g, 1) + spread4(x.hi, g, 2);  // 2 x (up + down + right)
    const uint32_t q2 = spread4(x.qw, g, 1);
    Quad r;
    r.K0 = pre2 + q2;
    r.K1 = pre2 + 0x02020202u - q2;
    if (rowstart) r.K1 = (r.K1 & 0xFFFFFF00u) | (r.K0 & 0xFFu);
    // per byte 148 - 5 K >= 108: no borrow; xor 0x80 recentres to 20 - 10 n
    r.D0 = (0x94949494u - 5u * r.K0) ^ 0x80808080u;
    r.D1 = (0x94949494u - 5u * r.K1) ^ 0x80808080u;
    return r;
}

// Ising decider for rows of whole words (L % 32 == 0, at least two words per row).
// The sites of consecutive words form one software pipeline: while word it is decided,
// the lattice words and neighbour planes of word it+1 are prepared, its first draws
// are loaded (site 28) and the candidate thresholds of its site 0 are loaded with the
// offsets resolved by site 30's decision (site 31), exactly as between sites of one
// word.  (With one word per row the next word's upper neighbours are this word's new
// spins, so that case keeps the per-word form.)  The site constants come four sites
// at a time in byte-parallel form, so a site costs four byte extractions, three
// selects on the previous decision, three adds, the two loads and the compare.
// CTX: site of the current word at which the next word's neighbour planes are formed
// from its lattice words (loaded at the start of the current word): early when the
// lattices are in shared memory, later when they come from L2.
//
// T16: the table in shared memory holds the upper 16 bits of every threshold (10 bytes
// per bin row), and a site compares the upper 16 bits of its draw with it.  That
// decides exactly unless the two halves are equal (probability ~2^-16 per attempt), in
// which case the fast path rejects, which always leaves a valid bin.  A lane that met
// such a tie marks it, and at the end of the word, if any lane did, the warp replays the
// word from the state it started it in, reading the 32-bit threshold from global memory
// where a draw ties its entry, and reloads the next site's candidates: every decision
// is the exact one.
// bin20 / d20p are in row bytes: 20 per bin, 10 per bin with T16.
template <bool BOOK, bool TSMEM, int RU, int RS, int CTX, bool T16 = false>
__device__ __forceinline__ void ising_decide_stream(const SweepArgs &a, uint32_t *lp, const size_t ls,
                                                    const uint32_t tab_s, const uint4 *s_ring, Snap *s_snap,
                                                    const int NU, const int lane, const int total, uint32_t &bin20,
                                                    uint32_t &d20p, bool &ap, const bool active)
{
#define LAT(k) lp[(size_t)(k) * ls]
    static_assert(!T16 || TSMEM, "the 16-bit table lives in shared memory");
    const int L = a.L, RW = a.row_words;
    // (fields of `a` are read once here: in the batched kernel `a` lives in shared memory,
    // and every named barrier would make the compiler read it again)
    const char *const ktab_b = reinterpret_cast<const char *>(a.ktab) - tab_s;
    const uint32_t *const ktab32 = a.ktab;
    auto tload = [&](uint32_t o) -> uint32_t {
        return T16 ? lds_u16(o) : TSMEM ? lds_u32(o) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(ktab_b + o));
    };
    auto quad = [&](const WordCtx &x, int g, bool rowstart) {
        return T16 ? site_quad16(x, g, rowstart) : site_quad(x, g, rowstart);
    };
    constexpr uint32_t ROW = T16 ? 10u : 20u;  // bytes per bin row
    bool tie = false;                          // a lane met an undecided 16-bit compare
    auto row_up = [&](int y) { return (y == 0 ? L - 1 : y - 1) * RW; };    // row above: updated
    auto row_down = [&](int y) { return (y == L - 1 ? 0 : y + 1) * RW; };  // row below: old (new for y = L-1)

    // ---- word 0
    int y = 0, w = 0;
    WordCtx cur = word_ctx(LAT(0), LAT(row_up(0)), LAT(row_down(0)), LAT(1), (LAT(RW - 1) >> 31) & 1u);
    uint32_t first_new = 0u;
    // P0 / P1: table address of the current site's bin (tab_s + 20 bin) if the previous
    // attempt was rejected / accepted
    uint32_t P0 = tab_s + bin20, P1 = P0 + d20p;
    Quad q0 = quad(cur, 0, true);
    uint32_t A0 = tload(P0 + ubyte(q0.K0, 0)), A1 = tload(P1 + ubyte(q0.K1, 0));
    bar_sync(kBarFullU + 0, NU);
    uint4 blk = s_ring[lane], blk_next = s_ring[32 + lane];

    for (int it = 0; it < total; ++it) {
        const bool lastw = (w == RW - 1);
        const bool has_next = it + 1 < total;
        const int slot = it % RU;
        const uint4 *src = s_ring + slot * 8 * 32 + lane;
        if (lastw) {
            // the row's last site sees the updated site 0 as its right neighbour
            const uint32_t tr2 = (cur.tr & 0x7FFFFFFFu) | (((cur.R >> 31) ^ first_new) << 31);
            cur.lo = cur.ua ^ cur.ub ^ tr2;
            cur.hi = (cur.ua & cur.ub) | (tr2 & (cur.ua ^ cur.ub));
        }
        // next word: (y1, w1)
        int y1 = y, w1 = w + 1;
        if (w1 == RW) {
            w1 = 0;
            y1 = (y + 1 == L) ? 0 : y + 1;
        }
        const int slot1 = (it + 1) % RU;
        const uint4 *src1 = s_ring + slot1 * 8 * 32 + lane;
        // its lattice words: all old, except the row above (finished: at least two words
        // per row) and, for the last row, the row below (row 0, finished)
        uint32_t R1 = 0u, U1 = 0u, D1w = 0u, Rn1 = 0u, lb1 = 0u;
        if (has_next) {
            const int kr1 = y1 * RW;
            R1 = (w1 == 0) ? LAT(kr1) : cur.Rn;
            U1 = LAT(row_up(y1) + w1);
            D1w = LAT(row_down(y1) + w1);
            Rn1 = (w1 + 1 < RW) ? LAT(kr1 + w1 + 1) : 0u;
            lb1 = (w1 == 0) ? ((LAT(kr1 + RW - 1) >> 31) & 1u) : (cur.R >> 31);
        }
        WordCtx nx;
        uint4 nblk = make_uint4(0u, 0u, 0u, 0u), nblk_next = nblk;
        uint32_t Rw = cur.R;
        const uint32_t P0s = P0, P1s = P1;  // state at the start of the word (replay)
        const bool aps = ap;
        Quad q1 = quad(cur, 1, false);  // constants of the next four sites
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int k = j & 3;
            if (k == 0 && j > 0) {
                blk = blk_next;
                if (j < 28) blk_next = src[((j >> 2) + 1) * 32];
                q0 = q1;
                if (j < 28)
                    q1 = quad(cur, (j >> 2) + 1, false);
                else
                    q1 = quad(nx, 0, w1 == 0);  // site 0 of the next word
            }
            if (j == CTX) nx = word_ctx(R1, U1, D1w, Rn1, lb1);
            if (j == 28 && has_next) {
                // first draws of the next word
                bar_sync(kBarFullU + slot1, NU);
                nblk = src1[0];
                nblk_next = src1[32];
            }
            const uint32_t u = k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w;
            // this site's bin and its change if accepted, resolved by the previous decision
            const uint32_t Pc = ap ? P1 : P0;
            const uint32_t DD = ap ? sbyte(q0.D1, k) : sbyte(q0.D0, k);
            const uint32_t nP1 = Pc + DD;
            // loads of the next site first (offsets resolved by the previous decision),
            // then the decision of this site
            uint32_t A0n = 0u, A1n = 0u;
            if ((j < 31) || has_next) {
                const uint32_t K0n = k == 3 ? ubyte(q1.K0, 0) : ubyte(q0.K0, k + 1);
                const uint32_t K1n = k == 3 ? ubyte(q1.K1, 0) : ubyte(q0.K1, k + 1);
                A0n = tload(Pc + K0n);
                A1n = tload(nP1 + K1n);
            }
            const uint32_t A = ap ? A1 : A0;
            bool acc;
            if (T16) {
                const uint32_t uh = u >> 16;
                acc = uh < A;
                tie |= uh == A;
            } else {
                acc = u < A;
            }
            A0 = A0n;
            A1 = A1n;
            P0 = Pc;
            P1 = nP1;
            Rw ^= acc ? (1u << j) : 0u;
            if (j == 0 && w == 0) first_new = (cur.R & 1u) ^ (acc ? 1u : 0u);
            ap = acc;
        }
        q0 = q1;
        if (T16 && __any_sync(0xffffffffu, tie && active)) {
            // exact replay of the word from its start: the 16-bit entries decide again,
            // and a draw that ties its entry reads the 32-bit threshold
            uint32_t bin = ((aps ? P1s : P0s) - tab_s) / ROW;
            bool apr = aps;
            uint32_t Rr = cur.R, b31 = 0u, n31 = 0u;
            for (int g = 0; g < 8; ++g) {
                const Quad qq = quad(cur, g, w == 0 && g == 0);
                const uint4 bl = src[g * 32];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t n = (apr ? ubyte(qq.K1, k) : ubyte(qq.K0, k)) >> 1;
                    const uint32_t u = k == 0 ? bl.x : k == 1 ? bl.y : k == 2 ? bl.z : bl.w;
                    const uint32_t uh = u >> 16, Ah = lds_u16(tab_s + ROW * bin + 2u * n);
                    bool acc = uh < Ah;
                    if (uh == Ah) acc = u < __ldg(ktab32 + bin * 5u + n);
                    if (g == 7 && k == 3) {
                        b31 = bin;
                        n31 = n;
                    }
                    if (acc) {
                        bin = bin + 2u - n;
                        Rr ^= 1u << (4 * g + k);
                    }
                    if (g == 0 && k == 0 && w == 0) first_new = (cur.R & 1u) ^ (acc ? 1u : 0u);
                    apr = acc;
                }
            }
            Rw = Rr;
            ap = apr;
            P0 = tab_s + ROW * b31;      // bin before site 31
            P1 = P0 + ROW * (2u - n31);  // ... and after it if it was accepted
            if (has_next) {              // the next site's candidates
                A0 = tload(P0 + ubyte(q0.K0, 0));
                A1 = tload(P1 + ubyte(q0.K1, 0));
            }
        }
        tie = false;
        if (it < total - RU) bar_arrive(kBarEmptyU + slot, NU);
        LAT(y * RW + w) = Rw;
        if (BOOK) {
            // snapshots are handed over in pairs of words (a launch has an even number
            // of words: L is even), one barrier hand-off per pair
            const int pw = it >> 1, half = it & 1, ss = pw % RS;
            if (half == 0 && pw >= RS) bar_sync(kBarEmptyS + ss, 64);
            Snap *sn = s_snap + (ss * kSnapWords + half) * 32 + lane;
            sn->lo = cur.lo;
            sn->hi = cur.hi;
            sn->qw = cur.qw;
            sn->flip = cur.R ^ Rw;
            sn->rold = cur.R;
            if (half == 1) bar_arrive(kBarFullS + ss, 64);
        }
        if (lastw) first_new = 0u;
        cur = nx;
        blk = nblk;
        blk_next = nblk_next;
        y = y1;
        w = w1;
    }
    bin20 = P0 - tab_s;
    d20p = P1 - P0;
#undef LAT
}

// HMODE: block histogram in global memory (0), in shared memory with one count per
// attempt (1), or in shared memory with one count per pair of consecutive attempts
// (2): C[b][d + 2] counts the pairs whose first attempt ends in bin b and whose second
// ends in bin b + d (|d| <= 2), and the histogram is H[b] = sum_d C[b][d + 2] +
// sum_d C[b - d][d + 2].  Mode 2 halves the shared-memory atomics, which otherwise
// delay the decider's table loads.  Mode 3 (lattices whose 32-bit histogram does not
// fit in shared memory, e.g. 256 x 256): 16-bit counts, two bins per word, added to the
// global histogram and cleared by the bookkeeper every floor(65535 / (32 L)) rows, before
// any count can reach 2^16 (a row adds at most 32 L counts to one bin).
// RU: slots of the draw ring (4; 3 in the compact staging that fits two blocks per SM)
// T16: the shared table holds the upper 16 bits of the thresholds (compact staging of
// three blocks per SM; rows of whole words, at least two per row: the stream decider)
template <bool HIST, bool RECORD, bool TSMEM, int HMODE, bool LSMEM, int RU = kRingU, bool T16 = false>
__device__ __forceinline__ void ising_ws_body(const SweepArgs &a, const int cblk, uint32_t *smem)
{
    __syncthreads();  // smem may still be read by a previous work unit of this block
    constexpr bool HSMEM = HMODE != 0;
    constexpr bool HPAIR = HIST && HMODE == 2;
    constexpr bool BOOK = HIST || RECORD;
    constexpr int NP = BOOK ? 2 : 3;            // producer warps (one SM sub-partition each)
    constexpr int NT = 128;                     // decider + producers (+ bookkeeper)
    constexpr int NU = 32 * (1 + NP);           // threads on the draw-ring barriers
    constexpr int BOOK_WARP = 1 + NP;
    static_assert(!T16 || (TSMEM && !LSMEM && HMODE != 2), "16-bit table: compact staging only");
    const int n_tab = a.n_bins * 5;
    constexpr uint32_t ROWB = T16 ? 10u : 20u;  // table bytes per bin
    uint32_t *s_tab = smem;
    constexpr bool H16 = HIST && HMODE == 3;
    const int n_hist = HPAIR ? a.n_bins * 5 : H16 ? (a.n_bins + 1) >> 1 : a.n_bins;
    const int tab_words = T16 ? (n_tab + 1) >> 1 : n_tab;
    uint32_t *s_hist = smem + (TSMEM ? ((tab_words + 3) & ~3) : 0);
    // the histogram is followed by one slot per lane (kHistDummy) for inactive lanes
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? ((n_hist + 3) & ~3) + kHistDummy : 0);
    static_assert(RU >= 2 && RU <= kRingU, "draw ring slots");
    uint4 *s_ring = reinterpret_cast<uint4 *>(s_lat + (LSMEM ? a.lat_words * 32 : 0));  // [RU][8][32]
    Snap *s_snap = reinterpret_cast<Snap *>(s_ring + RU * 8 * 32);  // [kRingS][kSnapWords][32]

    const int tid = threadIdx.x, lane = tid & 31;
    // chain of this lane: group cblk holds chains cblk * cpg ..; lanes beyond cpg take
    // padding columns after the last group (never read back)
    const int cpg = a.cpg;
    const int c = lane < cpg ? cblk * cpg + lane : (a.p_pad >> 5) * cpg + cblk * (32 - cpg) + (lane - cpg);
    const bool active = lane < cpg && c < a.p;
    // inactive lanes add their histogram counts into a slot of their own past the
    // histogram, so that every histogram atomic is a full-warp one (a red.shared issued
    // by part of a warp only is far slower)
    uint32_t *const s_hdummy = s_hist + ((n_hist + 3) & ~3) + lane;
    // Roles: 0 decider, 1..NP producers, NP+1 bookkeeper.  A warp issues on the SM
    // sub-partition of its warp slot mod 4, and a block's four warps take the four slots
    // of one aligned group, one per sub-partition.  In the compact staging two blocks
    // share an SM; there each decider gets the other block's bookkeeper (the warp that
    // issues least) as its neighbour on the same sub-partition: the block in an even
    // slot group puts its decider on sub-partition 0 and its bookkeeper on 3, the other
    // one the other way round, and the producers take 1 and 2 (measured 3% faster than
    // the slot order at p = 9728, 64 x 64).  With one block per SM the role is the warp
    // index, read back from shared memory (measured 5% faster at p = 1024 than taking
    // it from the thread index directly: the compiler lays the role branches out
    // differently).  With three blocks per SM (T16) the block in slot group g puts its
    // decider on sub-partition g mod 4 and its bookkeeper on (g + 3) mod 4, so that the
    // three deciders issue from three sub-partitions.  If a block's four sub-partitions
    // are not distinct the role is the warp index.
    constexpr bool PAIR_ROLES = RU != kRingU;
    __shared__ int s_sub[4], s_par;
    if (lane == 0) {
        uint32_t slot = 0u;
        if (PAIR_ROLES) asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
        s_sub[tid >> 5] = PAIR_ROLES ? (int)(slot & 3u) : (tid >> 5);
        if (tid == 0) s_par = (int)((slot >> 2) & (T16 ? 3u : 1u));
    }
    __syncthreads();
    int warp = s_sub[tid >> 5];
    if (PAIR_ROLES) {
        if (((1 << s_sub[0]) | (1 << s_sub[1]) | (1 << s_sub[2]) | (1 << s_sub[3])) == 0xF) {
            // sub-partitions of the decider and of the bookkeeper (role 3: the third
            // producer in launches without one); the producers take the other two in order
            const int dsub = T16 ? s_par : s_par ? 3 : 0;
            const int bsub = T16 ? (s_par + 3) & 3 : 3 - dsub;
            const int sub = warp;
            if (sub == dsub) {
                warp = 0;
            } else if (sub == bsub) {
                warp = 3;
            } else {
                warp = 1;
                for (int t = 0; t < sub; ++t) warp += (t != dsub && t != bsub) ? 1 : 0;
            }
        } else {
            warp = tid >> 5;
        }
    }

    if (T16) {
        uint16_t *s_tab16 = reinterpret_cast<uint16_t *>(s_tab);
        for (int i = tid; i < n_tab; i += NT) s_tab16[i] = (uint16_t)(a.ktab[i] >> 16);
    } else if (TSMEM) {
        for (int i = tid; i < n_tab; i += NT) s_tab[i] = a.ktab[i];
    }
    if (HIST && HSMEM)
        for (int i = tid; i < n_hist; i += NT) s_hist[i] = 0u;
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
        const uint32_t key0 = a.key0, iter = a.iteration, ctr3 = a.ctr3, sweep0 = a.sweep0;
        const int n_sweeps = a.n_sweeps;
        int it = 0;
        for (int sw = 0; sw < n_sweeps; ++sw) {
            const uint32_t ctr1 = sweep0 + (uint32_t)sw;
            int site = 0;
            for (int y = 0; y < L; ++y) {
                for (int w = 0; w < RW; ++w, ++it) {
                    const int nb = (w == RW - 1) ? last_bits : 32;
                    const int slot = it % RU;
                    if (it >= RU) bar_sync(kBarEmptyU + slot, NU);
                    uint4 *dst = s_ring + slot * 8 * 32 + lane;
                    // the word's blocks are independent: unrolled so that their 10-round
                    // dependency chains interleave
#pragma unroll 4
                    for (int gi = pr; gi < (nb >> 2); gi += NP) {
                        uint4 b = philox4x32_10_rk(make_uint4((uint32_t)(site >> 2) + (uint32_t)gi, ctr1, iter, ctr3),
                                                   key0, k1r);
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
        // table addresses: shared-memory addresses, or byte offsets into the global table
        const uint32_t tab_s = TSMEM ? (uint32_t)__cvta_generic_to_shared(s_tab) : 0u;
        const char *const ktab_g = reinterpret_cast<const char *>(a.ktab);
#define TAB_BYTES(o) (TSMEM ? lds_u32(tab_s + (o)) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(ktab_g + (o))))
        const int bin0 = active ? (a.E[c] + 2 * V) >> 2 : (V >> 1);
        uint32_t bin20 = ROWB * (uint32_t)bin0;  // table row of the bin before the previous decision
        uint32_t d20p = 0u;                      // its change if the previous attempt was accepted
        bool ap = false;                         // previous attempt accepted
        if (T16 || (last_bits == 32 && RW >= 2)) {
            ising_decide_stream<BOOK, TSMEM, RU, kRingS, LSMEM ? 8 : 20, T16>(a, lp, ls, tab_s, s_ring, s_snap, NU, lane,
                                                                             total, bin20, d20p, ap, active);
        } else {
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
                    const int slot = it % RU;
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
                                                                      ktab_g + P0 + K0 - tab_s));
                        uint32_t A1 = TSMEM ? lds_u32(P1 + K1) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                                      ktab_g + P1 + K1 - tab_s));
                        // draws of the word: group g+1 is loaded while group g is decided
                        uint4 blk = src[0], blk_next = src[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int k = j & 3;
                            if (k == 0 && j > 0) {
                                blk = blk_next;
                                if (j < 28) blk_next = src[((j >> 2) + 1) * 32];
                            }
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
                                                               ktab_g + o0 - tab_s));
                                A1n = TSMEM ? lds_u32(o1) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(
                                                               ktab_g + o1 - tab_s));
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
                    if (it < total - RU) bar_arrive(kBarEmptyU + slot, NU);
                    LAT(kr + w) = Rw;
                    if (BOOK) {
                        if (lastw) {
                            // the row's last site saw the updated site 0 as its right neighbour
                            const uint32_t bitm = 1u << (nb - 1);
                            const uint32_t tr2 = (tr & ~bitm) | ((((R >> (nb - 1)) & 1u) ^ first_new) << (nb - 1));
                            lo = ua ^ ub ^ tr2;
                            hi = (ua & ub) | (tr2 & (ua ^ ub));
                        }
                        const int pw = it >> 1, half = it & 1, ss = pw % kRingS;  // pairs of words
                        if (half == 0 && pw >= kRingS) bar_sync(kBarEmptyS + ss, 64);
                        Snap *sn = s_snap + (ss * kSnapWords + half) * 32 + lane;
                        sn->lo = lo;
                        sn->hi = hi;
                        sn->qw = qw;
                        sn->flip = R ^ Rw;
                        sn->rold = R;
                        if (half == 1) bar_arrive(kBarFullS + ss, 64);
                    }
                    lbit = R >> 31;
                    R = Rn;
                    U = Un;
                    D = Dn;
                }
            }
        }
        }
        if (active && !BOOK) {
            // no bookkeeper: apply the pending decision and recount M
            const uint32_t bin_end = (ap ? bin20 + d20p : bin20) / ROWB;
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
        // mode 3: rows between flushes of the 16-bit counts into the global histogram
        const int flush_rows = max(1, 65535 / (32 * L));
        int rows = 0;
        auto flush16 = [&]() {
            __syncwarp();  // every lane's counts of the flushed rows are in place
            for (int i = lane; i < n_hist; i += 32) {
                const uint32_t v = s_hist[i];
                if (v) {
                    s_hist[i] = 0u;
                    unsigned long long *Hg = reinterpret_cast<unsigned long long *>(a.H) + 2 * i;
                    if (v & 0xFFFFu) atomicAdd(Hg, (unsigned long long)(v & 0xFFFFu));
                    if (v >> 16) atomicAdd(Hg + 1, (unsigned long long)(v >> 16));
                }
            }
            __syncwarp();
        };
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            for (int y = 0; y < L; ++y) {
                uint32_t pflip = 0u;  // flip of the previous site in this row
                for (int w = 0; w < RW; ++w, ++it) {
                    const int nb = (w == RW - 1) ? last_bits : 32;
                    const int pw = it >> 1, half = it & 1, ss = pw % kRingS;  // pairs of words
                    if (half == 0) bar_sync(kBarFullS + ss, 64);
                    const Snap sn = s_snap[(ss * kSnapWords + half) * 32 + lane];
                    if (half == 1 && pw < (total >> 1) - kRingS) bar_arrive(kBarEmptyS + ss, 64);
                    // left neighbour as seen by each site: old left, flipped if the
                    // previous site flipped (not across the row start)
                    const uint32_t lf = (sn.flip << 1) | pflip;
                    const uint32_t qn = sn.qw ^ lf;
                    auto book_site = [&](int j) {
                        const int nneq = (int)(((sn.lo >> j) & 1u) + 2u * ((sn.hi >> j) & 1u) + ((qn >> j) & 1u));
                        const bool acc = (sn.flip >> j) & 1u;
                        bin += acc ? 2 - nneq : 0;
                        if (H16) {
                            red_shared(active ? s_hist + (bin >> 1) : s_hdummy, 1u << ((bin & 1) << 4));
                        } else if (HIST && HSMEM) {
                            red_shared(active ? s_hist + bin : s_hdummy, 1u);
                        } else if (HIST && active) {
                            if (bin != run_bin) {
                                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]), (unsigned long long)run);
                                run_bin = bin;
                                run = 0;
                            }
                            ++run;
                        }
                    };
                    if (HPAIR) {
                        // one count per pair of attempts (nb is a multiple of 4)
                        auto delta = [&](int j) {
                            const int nneq =
                                (int)(((sn.lo >> j) & 1u) + 2u * ((sn.hi >> j) & 1u) + ((qn >> j) & 1u));
                            return ((sn.flip >> j) & 1u) ? 2 - nneq : 0;
                        };
                        auto book_pair = [&](int j) {
                            bin += delta(j);
                            const int d = delta(j + 1);
                            red_shared(active ? s_hist + 5 * bin + 2 + d : s_hdummy, 1u);
                            bin += d;
                        };
                        if (nb == 32) {
#pragma unroll
                            for (int j = 0; j < 32; j += 2) book_pair(j);
                        } else {
                            for (int j = 0; j < nb; j += 2) book_pair(j);
                        }
                    } else if (nb == 32) {
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
                if (H16 && ++rows == flush_rows) {
                    flush16();
                    rows = 0;
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
    if (HPAIR) {
        // first attempts of the pairs in bin b, then second attempts (from bin b - d)
        for (int b = tid; b < a.n_bins; b += NT) {
            uint32_t v = 0u;
#pragma unroll
            for (int d = -2; d <= 2; ++d) {
                v += s_hist[5 * b + 2 + d];
                if (b - d >= 0 && b - d < a.n_bins) v += s_hist[5 * (b - d) + 2 + d];
            }
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[b]), (unsigned long long)v);
        }
    } else if (H16) {
        // the counts since the last flush
        for (int i = tid; i < n_hist; i += NT) {
            const uint32_t v = s_hist[i];
            unsigned long long *Hg = reinterpret_cast<unsigned long long *>(a.H) + 2 * i;
            if (v & 0xFFFFu) atomicAdd(Hg, (unsigned long long)(v & 0xFFFFu));
            if (v >> 16) atomicAdd(Hg + 1, (unsigned long long)(v >> 16));
        }
    } else if (HIST && HSMEM) {
        for (int i = tid; i < a.n_bins; i += NT) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}


// ===========================================================================
// 8-state Potts: warp 0 decides (and fills the histogram / records), warps 1..3
// produce.  A ring slot holds up to 8 words (32 sites) of one row; the ring has three
// slots and slot s always belongs to producer s, so each hand-off barrier has two
// parties (the decider and that producer) and the producers run independently of
// each other.  Per word of 4 sites the producer writes the four clamped
// acceptance draws, the proposed spins and, byte-parallel, each site's table column
// (dE + 4) for the previous attempt rejected / accepted, counted over the neighbours
// whose values are fixed before the decider reaches the site: the old spins below, to
// the right and to the left, and the left neighbour's proposal.  The decider adds the
// upper neighbour (the row above is already updated), the right neighbour of a row's
// last site (site 0, updated at the start of the row) and the left neighbour of a slot
// that starts mid-row.
// ===========================================================================
constexpr int kPottsSlotWords = 8;
constexpr int kPottsRing = 3;  // = number of producers

__device__ __forceinline__ int zero_bytes_ws(uint32_t x)
{
    const uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    return __popc(~t & 0x80808080u);
}

// 0x01 in every byte where x and y are equal, 0x00 elsewhere
__device__ __forceinline__ uint32_t eq_bytes(uint32_t x, uint32_t y)
{
    const uint32_t t = x ^ y;
    return (~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u) >> 7;
}

__device__ __forceinline__ uint32_t byte_of(uint32_t x, int k) { return __byte_perm(x, 0u, 0x4440u | (uint32_t)k); }

__device__ __forceinline__ void potts_count_move(uint64_t &lo, uint64_t &hi, uint32_t from, uint32_t to)
{
    const uint64_t df = 1ull << (16 * (from & 3u)), dt = 1ull << (16 * (to & 3u));
    if (from < 4) lo -= df; else hi -= df;
    if (to < 4) lo += dt; else hi += dt;
}

__device__ __forceinline__ int potts_count_max(uint64_t lo, uint64_t hi)
{
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        m = max(m, (int)((lo >> (16 * k)) & 0xFFFFu));
        m = max(m, (int)((hi >> (16 * k)) & 0xFFFFu));
    }
    return m;
}

__device__ __forceinline__ void potts_count_word(uint32_t word, uint32_t (&cnt)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt[k] += zero_bytes_ws(word ^ (0x01010101u * (uint32_t)k));
}

// Potts decider for rows of whole ring slots (RW a multiple of 8: L % 32 == 0).  The 32
// sites of a slot are one unrolled block, so every word index in it is a constant:
// the next word's records and upper neighbour are read while the current word is
// decided (the next slot's first word while a slot's last word is), and what is left
// per word is the upper neighbour's column correction, byte-parallel.  Per site, as in
// the per-word form: two byte extractions, two bin changes, three selects, the two
// table loads and the compare.  With the bookkeeper (BOOKW) the decider hands over,
// per word, the corrected column words, the accepted-byte mask and the old spins (and
// the proposals, for records), one snapshot block per slot, from which the bookkeeper
// rebuilds every attempt's bin for its histogram (BHIST; without a histogram it gets
// the bin at each word's end instead); without the bookkeeper the decider counts the
// shared histogram itself (HIST).  Returns the state after the last attempt in P0 /
// P1 / ap.
constexpr int kPSnapSlots = 2;  // snapshot blocks of the slot form (one ring slot each)

// byte-wise "not zero" of words whose bytes are below 8 (no masking needed)
__device__ __forceinline__ uint32_t nz_bytes8(uint32_t x) { return ((x + 0x7F7F7F7Fu) >> 7) & 0x01010101u; }

template <bool BOOKW, bool HIST, bool RECORD, bool TSMEM, bool LSMEM, bool BHIST>
__device__ __forceinline__ void potts_decide_slots(const SweepArgs &a, const uint4 *s_ring, uint4 *s_snap,
                                                   uint32_t *s_snsn, uint32_t *s_hist, uint32_t *s_hdummy,
                                                   const uint32_t tab_s, uint32_t *lp, const size_t ls,
                                                   const int lane, const bool active, uint32_t &P0, uint32_t &P1,
                                                   bool &ap)
{
    static_assert(!RECORD || BOOKW, "records come from the bookkeeper");
    static_assert(!(HIST && BOOKW), "one histogram owner");
#define LAT(k) lp[(size_t)(k) * ls]
    constexpr int NU = 64, RD = kPottsRing;
    const int L = a.L, RW = a.row_words, spr = RW >> 3;
    const int total = a.n_sweeps * L * spr;  // slots per launch
    const char *const tab_g = reinterpret_cast<const char *>(a.ktab) - tab_s;
    auto tload = [&](uint32_t o) -> uint32_t {
        return TSMEM ? lds_u32(o) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(tab_g + o));
    };
    // bin of a table row address: (P - tab_s) / 36 = ((P - tab_s) / 4) * 9^-1 mod 2^32
    auto bin_of = [&](uint32_t P) { return (int)(((P - tab_s) >> 2) * 0x38E38E39u); };
    struct Word {
        uint4 u;                 // acceptance draws
        uint32_t R, SN, C0, C1;  // old spins, proposals, column words (previous attempt rejected / accepted)
    };
    // a word's columns: the producer's counts plus the upper neighbour U (row above,
    // final): + [U == s] - [U == s'] = nz(U ^ s') - nz(U ^ s) per byte
    auto columns = [](Word &x, const uint4 &r1, uint32_t U) {
        x.R = r1.w;
        x.SN = r1.x;
        const uint32_t d = nz_bytes8(U ^ r1.x) - nz_bytes8(U ^ r1.w);
        x.C0 = r1.y + d;  // every byte of the result is a count in 0..8: the borrows cancel
        x.C1 = r1.z + d;
    };
    auto up_row = [&](int y) { return (y == 0 ? L - 1 : y - 1) * RW; };

    int y = 0, sl = 0;  // row and slot in the row
    uint32_t first_new = 0u;
    Word cur;
    bar_sync(kBarFullU + 0, NU);
    {
        cur.u = s_ring[lane];
        const uint4 r1 = s_ring[32 + lane];
        columns(cur, r1, LAT(up_row(0)));
    }
    uint32_t K0 = byte_of(cur.C0, 0), K1 = byte_of(cur.C1, 0);
    uint32_t D0 = 36u * K0 - 144u, D1 = 36u * K1 - 144u;
    uint32_t A0 = tload(P0 + 4u * K0), A1 = tload(P1 + 4u * K1);

    for (int s = 0; s < total; ++s) {
        const bool has_next = s + 1 < total;
        int y1 = y, sl1 = sl + 1;
        if (sl1 == spr) {
            sl1 = 0;
            y1 = (y + 1 == L) ? 0 : y + 1;
        }
        const bool row_start = sl == 0, row_end = sl == spr - 1;
        const uint4 *src = s_ring + (s % RD) * 16 * 32 + lane;
        const int kr = y * RW + sl * 8, ku = up_row(y) + sl * 8;
        const int b = s % kPSnapSlots;
        if (BOOKW && s >= kPSnapSlots) bar_sync(kBarEmptyS + b, 64);
        uint4 *snap = s_snap + b * 8 * 32 + lane;
        uint32_t Fm = 0u;  // bytes of accepted sites of the current word
        Word nx = cur;
        uint4 nr1 = make_uint4(0u, 0u, 0u, 0u);
        uint32_t nU = 0u;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int w = j >> 2, k = j & 3;
            if (k == 0) {
                // records of the next word: in this slot, or the next slot's first
                if (w < 7) {
                    nx.u = src[(2 * w + 2) * 32];
                    nr1 = src[(2 * w + 3) * 32];
                    nU = LAT(ku + w + 1);
                } else if (has_next) {
                    bar_sync(kBarFullU + (s + 1) % RD, NU);
                    const uint4 *src1 = s_ring + ((s + 1) % RD) * 16 * 32 + lane;
                    nx.u = src1[0];
                    nr1 = src1[32];
                    nU = LAT(up_row(y1) + sl1 * 8);
                }
            }
            if (k == 1 && (w < 7 || has_next)) {
                columns(nx, nr1, nU);
                if (w == 7 && sl1 != 0) {
                    // the next slot starts mid-row: its first site's left neighbour is this
                    // slot's last site (old spin if that attempt is rejected, else proposal)
                    const uint32_t lold = cur.R >> 24, lsn = cur.SN >> 24;
                    const uint32_t s0 = nx.R & 0xFFu, sn0 = nx.SN & 0xFFu;
                    nx.C0 = nx.C0 + (lold == s0 ? 1u : 0u) - (lold == sn0 ? 1u : 0u);
                    nx.C1 = nx.C1 + (lsn == s0 ? 1u : 0u) - (lsn == sn0 ? 1u : 0u);
                }
            }
            if (w == 7 && k == 1 && row_end) {
                // the row's last site: its right neighbour is site 0 of the row, updated
                const uint32_t s3 = cur.R >> 24, sn3 = cur.SN >> 24;
                const uint32_t dK = ((first_new == s3 ? 1u : 0u) - (first_new == sn3 ? 1u : 0u)) << 24;
                cur.C0 += dK;
                cur.C1 += dK;
            }
            // 1. candidates of the next site (offsets resolved by the previous decision)
            const uint32_t Kn0 = k < 3 ? byte_of(cur.C0, k + 1) : byte_of(nx.C0, 0);
            const uint32_t Kn1 = k < 3 ? byte_of(cur.C1, k + 1) : byte_of(nx.C1, 0);
            const uint32_t Dn0 = 36u * Kn0 - 144u, Dn1 = 36u * Kn1 - 144u;
            const uint32_t Pb = ap ? P1 : P0;
            const uint32_t PbD = Pb + (ap ? D1 : D0);
            uint32_t A0n = 0u, A1n = 0u;
            if (j < 31 || has_next) {
                A0n = tload(Pb + 4u * Kn0);
                A1n = tload(PbD + 4u * Kn1);
            }
            // 2. decision of this site
            const uint32_t u = k == 0 ? cur.u.x : k == 1 ? cur.u.y : k == 2 ? cur.u.z : cur.u.w;
            const bool acc = u < (ap ? A1 : A0);
            Fm |= acc ? (0xFFu << (8 * k)) : 0u;
            if (j == 0 && row_start) first_new = acc ? (cur.SN & 0xFFu) : (cur.R & 0xFFu);
            if (HIST) red_shared(active ? s_hist + bin_of(acc ? PbD : Pb) : s_hdummy, 1u);
            // 3. state of the next site
            P0 = Pb;
            P1 = PbD;
            D0 = Dn0;
            D1 = Dn1;
            A0 = A0n;
            A1 = A1n;
            ap = acc;
            if (k == 3) {
                LAT(kr + w) = (cur.R & ~Fm) | (cur.SN & Fm);
                if (BOOKW) {
                    // the bookkeeper rebuilds every attempt's bin from the column words
                    // for its histogram (BHIST), else it needs the bin at the word's end
                    snap[w * 32] = make_uint4(BHIST ? cur.C0 : (ap ? P1 : P0), cur.C1, Fm, cur.R);
                    if (RECORD) s_snsn[(b * 8 + w) * 32 + lane] = cur.SN;
                }
                Fm = 0u;
                cur = nx;
            }
        }
        // the slot's records are all read: release it
        if (s < total - RD) bar_arrive(kBarEmptyU + s % RD, NU);
        if (BOOKW) bar_arrive(kBarFullS + b, 64);
        y = y1;
        sl = sl1;
    }
#undef LAT
}

// Bookkeeper of the slot form: every attempt's bin from the snapshot block of a slot
// (column words, accepted bytes, old spins, proposals) for the histogram (single
// attempts, or pairs of attempts: HPAIR), and for records the state counts and the
// (E, M) records.  The state counts live in shared memory, one 32-bit counter per
// (state, lane) and a ninth row for rejected attempts, updated with red.shared (no
// result, so consecutive updates do not wait on one another): an accepted site moves
// one count from its old state to its new one.
template <bool HIST, bool HPAIR, bool RECORD>
__device__ __forceinline__ void potts_book_slots(const SweepArgs &a, const uint4 *s_snap, const uint32_t *s_snsn,
                                                 uint32_t *s_hist, uint32_t *s_hdummy, uint32_t *s_cnt,
                                                 const uint32_t tab_s, const int lane, const bool active, const int c,
                                                 int bin)
{
    const int L = a.L, RW = a.row_words, V = L * L, spr = RW >> 3;
    const int total = a.n_sweeps * L * spr;
    const int per_sweep = L * spr;
    uint32_t *const cl = s_cnt + lane;  // [9][32]: counters of states 0..7, rejected
    bool ap = false;                    // previous attempt accepted
    uint32_t last_row = 0u;             // bin row after the slot (without a histogram)
    for (int s = 0; s < total; ++s) {
        const int b = s % kPSnapSlots;
        bar_sync(kBarFullS + b, 64);
        const uint4 *snap = s_snap + b * 8 * 32 + lane;
#pragma unroll 2
        for (int w = 0; w < 8; ++w) {
            const uint4 sn = snap[w * 32];  // (C0 or bin row, C1, Fm, R)
            if (HIST) {
                int bk[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool acc = (sn.z >> (8 * k)) & 1u;
                    const int col = (int)(ap ? byte_of(sn.y, k) : byte_of(sn.x, k));
                    bin += acc ? col - 4 : 0;
                    bk[k] = bin;
                    ap = acc;
                    if (!HPAIR) red_shared(active ? s_hist + bin : s_hdummy, 1u);
                }
                if (HPAIR) {
                    // one count per pair of attempts: (0, 1) and (2, 3)
                    red_shared(active ? s_hist + 9 * bk[0] + 4 + (bk[1] - bk[0]) : s_hdummy, 1u);
                    red_shared(active ? s_hist + 9 * bk[2] + 4 + (bk[3] - bk[2]) : s_hdummy, 1u);
                }
            } else {
                last_row = sn.x;
            }
            if (RECORD) {
                const uint32_t SN = s_snsn[(b * 8 + w) * 32 + lane];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool acc = (sn.z >> (8 * k)) & 1u;
                    red_shared(cl + 32u * (acc ? byte_of(sn.w, k) : 8u), 0xFFFFFFFFu);  // - 1
                    red_shared(cl + 32u * (acc ? byte_of(SN, k) : 8u), 1u);
                }
            }
        }
        if (s < total - kPSnapSlots) bar_arrive(kBarEmptyS + b, 64);
        if (RECORD && (s + 1) % per_sweep == 0) {
            if (!HIST) bin = (int)(((last_row - tab_s) >> 2) * 0x38E38E39u);  // row / 36
            if (active) {
                const int sw = s / per_sweep;
                const int E = bin - 2 * V;
                uint32_t mx = 0u;
#pragma unroll
                for (int v = 0; v < 8; ++v) mx = max(mx, cl[32 * v]);
                const int M = 8 * (int)mx - V;
                if (a.E_rec) a.E_rec[(size_t)sw * a.rec_stride + c] = E;
                if (a.M_rec) a.M_rec[(size_t)sw * a.rec_stride + c] = M;
                if (a.samples) {
                    const unsigned long long am = (unsigned long long)(M < 0 ? -M : M);
                    unsigned long long *sp = reinterpret_cast<unsigned long long *>(a.samples);
                    atomicAdd(&sp[bin], 1ull);
                    atomicAdd(&sp[a.n_bins + bin], am);
                    atomicAdd(&sp[2 * a.n_bins + bin], am * am);
                }
            }
        }
    }
}

// PBOOK: a fifth warp, the bookkeeper, takes the histogram, the state counts and the
// records from per-word snapshots (iteration and production launches of the
// standalone kernel); the decider then runs on warp 1, alone on its SM sub-partition,
// and the bookkeeper shares one with producer warp 0.
// HMODE as for Ising; in mode 2 (bookkeeper only) C[b][d + 4] counts the pairs of
// consecutive attempts ending in bins b and b + d (|d| <= 4).
template <bool HIST, bool RECORD, bool TSMEM, int HMODE, bool LSMEM, bool PBOOK = false>
__device__ __forceinline__ void potts_ws_body(const SweepArgs &a, const int cblk, uint32_t *smem)
{
    constexpr bool HSMEM = HMODE != 0;
    constexpr bool BOOKW = PBOOK && (HIST || RECORD);
    constexpr bool HPAIR = BOOKW && HIST && HMODE == 2;
    constexpr int NT = BOOKW ? 160 : 128;  // decider + one producer warp per ring slot (+ bookkeeper)
    constexpr int NU = 64;                 // decider + the slot's producer
    __syncthreads();  // smem may still be read by a previous work unit of this block
    const int n_tab = a.n_bins * 9;
    uint32_t *s_tab = smem;
    const int n_hist = HPAIR ? a.n_bins * 9 : a.n_bins;
    uint32_t *s_hist = smem + (TSMEM ? ((n_tab + 3) & ~3) : 0);
    // the histogram is followed by one slot per lane (kHistDummy) for inactive lanes
    uint32_t *s_lat = s_hist + ((HIST && HSMEM) ? ((n_hist + 3) & ~3) + kHistDummy : 0);
    uint4 *s_ring = reinterpret_cast<uint4 *>(s_lat + (LSMEM ? a.lat_words * 32 : 0));  // [ring][8 words][2][32]
    uint4 *s_psnap = s_ring + kPottsRing * 16 * 32;  // [kRingS][2][32]; slot form: [kPSnapSlots][8][32]
    uint32_t *s_snsn = reinterpret_cast<uint32_t *>(s_psnap + kPSnapSlots * 8 * 32);  // [kPSnapSlots][8][32]
    // slot form of the decider (and bookkeeper): rows of whole slots, with the
    // histogram in shared memory or kept by the bookkeeper, records by the bookkeeper
    constexpr bool SLOTS_OK = (BOOKW || !RECORD) && (!HIST || HSMEM);
    const bool slots = SLOTS_OK && (a.row_words % kPottsSlotWords) == 0;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int vw = BOOKW ? (warp == 0 ? 1 : warp == 1 ? 0 : warp) : warp;  // role: 0 decider, 1..3 producers, 4 bookkeeper
    // chain of this lane (groups of cpg chains; lanes beyond cpg on padding columns)
    const int cpg = a.cpg;
    const int c = lane < cpg ? cblk * cpg + lane : (a.p_pad >> 5) * cpg + cblk * (32 - cpg) + (lane - cpg);
    const bool active = lane < cpg && c < a.p;
    uint32_t *const s_hdummy = s_hist + ((n_hist + 3) & ~3) + lane;  // inactive lanes' histogram slot

    if (TSMEM)
        for (int i = tid; i < n_tab; i += NT) s_tab[i] = a.ktab[i];
    if (HIST && HSMEM)
        for (int i = tid; i < n_hist; i += NT) s_hist[i] = 0u;
    if (LSMEM && vw == 0)
        for (int k = 0; k < a.lat_words; ++k) s_lat[k * 32 + lane] = a.lat[(size_t)k * a.p_pad + c];
    // bookkeeper of a production launch: state counts of the starting lattice, read
    // before the decider changes it (16-bit counters, four per register)
    const int bk_bin0 = active ? a.E[c] + 2 * a.L * a.L : a.L * a.L;  // bin at the start
    uint64_t bk_lo = 0, bk_hi = 0;
    if (BOOKW && RECORD && vw == 4) {
        uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < a.lat_words; ++k) potts_count_word(a.lat[(size_t)k * a.p_pad + c], cnt);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bk_lo |= (uint64_t)cnt[k] << (16 * k);
            bk_hi |= (uint64_t)cnt[k + 4] << (16 * k);
        }
    }
    __syncthreads();

    const int L = a.L, RW = a.row_words, V = L * L;
    const int spr = (RW + kPottsSlotWords - 1) / kPottsSlotWords;  // slots per row
    const int total = a.n_sweeps * L * spr;                          // slots per launch
    // A producer reads row y+1 (old) and, for the last row, row 0 of the current sweep
    // (new), so it may run at most L - 1 rows of slots ahead: 3 <= spr * (L - 1) for L >= 4.
    constexpr int RD = kPottsRing;
    uint32_t *const glat = a.lat + c;
    const size_t gstride = (size_t)a.p_pad;
#define LAT(k) (*(LSMEM ? &s_lat[(k) * 32 + lane] : &glat[(size_t)(k) * gstride]))

    if (vw >= 1 && vw <= kPottsRing) {
        // ---------------- producers ----------------------------------------------
        const int pr = vw - 1;
        uint32_t k1r[10];
        philox_round_keys((uint32_t)c, k1r);
        const uint32_t cap = active ? 0xFFFFFFFEu : 0xFFFFFFFFu;
        const uint32_t key0 = a.key0, iter = a.iteration, ctr3 = a.ctr3, sweep0 = a.sweep0;
        auto draw = [&](uint32_t x) { return active ? min(x, cap) : cap; };
        // proposal offset floor(7 w / 2^32) in 0..6, exactly: 7w = 8w - w
        auto offset7 = [](uint32_t x) { return (x >> 29) - ((x << 3) < x ? 1u : 0u); };
        int it = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            const uint32_t ctr1 = sweep0 + (uint32_t)sw;
            for (int y = 0; y < L; ++y) {
                const int kr = y * RW, kd = (y == L - 1 ? 0 : y + 1) * RW;
                for (int w0 = 0; w0 < RW; w0 += kPottsSlotWords, ++it) {
                    if (it % RD != pr) continue;  // another producer's slot
                    const int nw = min(kPottsSlotWords, RW - w0);
                    const int slot = pr;
                    if (it >= RD) bar_sync(kBarEmptyU + slot, NU);
                    {
                        uint4 *dst = s_ring + slot * 16 * 32 + lane;
                        // left neighbour of the slot's first site: site L-1 (old) at a row
                        // start; mid-row it is added by the decider (0xFF matches no spin)
                        uint32_t lprev = (w0 == 0) ? (LAT(kr + RW - 1) >> 24) : 0xFFu;
                        uint32_t snprev = 0xFFu;
                        uint32_t R = LAT(kr + w0);
#pragma unroll 2
                        for (int w = w0; w < w0 + nw; ++w) {
                            const bool lastw = (w == RW - 1);
                            // right word (old); at the row end the decider adds site 0
                            const uint32_t Rn = lastw ? 0xFFu : LAT(kr + w + 1);
                            const uint32_t D = LAT(kd + w);
                            const uint32_t g = (uint32_t)(y * L + 4 * w) >> 1;
                            const uint4 b0 = philox4x32_10_rk(make_uint4(g, ctr1, iter, ctr3), key0, k1r);
                            const uint4 b1 = philox4x32_10_rk(make_uint4(g + 1u, ctr1, iter, ctr3), key0, k1r);
                            const uint32_t off = offset7(b0.y) | (offset7(b0.w) << 8) | (offset7(b1.y) << 16) |
                                                 (offset7(b1.w) << 24);
                            const uint32_t SN = (R + 0x01010101u + off) & 0x07070707u;  // (s + 1 + off) mod 8
                            const uint32_t Rr = (R >> 8) | (Rn << 24);
                            const uint32_t Ll = (R << 8) | lprev;
                            const uint32_t SNl = (SN << 8) | snprev;
                            const uint32_t base = 0x04040404u + eq_bytes(D, R) + eq_bytes(Rr, R) - eq_bytes(D, SN) -
                                                  eq_bytes(Rr, SN);
                            const uint32_t c0 = base + eq_bytes(Ll, R) - eq_bytes(Ll, SN);
                            uint32_t c1 = base + eq_bytes(SNl, R) - eq_bytes(SNl, SN);
                            // a row's first site: its left neighbour is not the previous attempt
                            if (w == 0) c1 = (c1 & 0xFFFFFF00u) | (c0 & 0xFFu);
                            dst[(2 * (w - w0)) * 32] = make_uint4(draw(b0.x), draw(b0.z), draw(b1.x), draw(b1.z));
                            dst[(2 * (w - w0) + 1) * 32] = make_uint4(SN, c0, c1, R);  // R: old spins
                            lprev = R >> 24;
                            snprev = SN >> 24;
                            R = Rn;
                        }
                    }
                    bar_arrive(kBarFullU + slot, NU);
                }
            }
        }
    } else if (vw == 0) {
        // ---------------- decider ------------------------------------------------
        // table addresses: shared-memory addresses, or byte offsets into the global table
        const uint32_t tab_s = TSMEM ? (uint32_t)__cvta_generic_to_shared(s_tab) : 0u;
        const char *tab_g = reinterpret_cast<const char *>(a.ktab) - tab_s;
#define TABLOAD(o) (TSMEM ? lds_u32(o) : ldg_nc_u32(reinterpret_cast<const uint32_t *>(tab_g + (o))))
        const int bin0 = active ? a.E[c] + 2 * V : V;
        uint64_t cnt_lo = 0, cnt_hi = 0;
        if (RECORD && !BOOKW && active) {
            uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < a.lat_words; ++k) potts_count_word(LAT(k), cnt);
            for (int k = 0; k < 4; ++k) {
                cnt_lo |= (uint64_t)cnt[k] << (16 * k);
                cnt_hi |= (uint64_t)cnt[k + 4] << (16 * k);
            }
        }
        // P0/P1 = table address of the row of the bin before this attempt if the previous
        // attempt was rejected / accepted (36 bytes per bin)
        uint32_t P0 = tab_s + 36u * (uint32_t)bin0, P1 = P0;
        bool ap = false;
        int run_bin = bin0;
        uint32_t run = 0;
        // bin of a table row address: (P - tab_s) / 36 = ((P - tab_s) / 4) * 9^-1 mod 2^32
        auto bin_of = [&](uint32_t P) { return (int)(((P - tab_s) >> 2) * 0x38E38E39u); };

        // word context: old spins, proposals, draws and the two column words x 4
        struct PW {
            uint32_t R, SN, C0, C1;
            uint4 u;
        };
        // columns of a word: the producer's counts plus the upper neighbour; a slot that
        // starts mid-row also gets its first site's left neighbour (old spin, proposal)
        auto columns = [&](PW &x, const uint4 &r1, uint32_t U, bool slot_mid, uint32_t lold, uint32_t lsn) {
            x.SN = r1.x;
            const uint32_t up = eq_bytes(U, x.R), un = eq_bytes(U, x.SN);
            uint32_t c0 = r1.y + up - un, c1 = r1.z + up - un;
            if (slot_mid) {
                const uint32_t s0 = x.R & 0xFFu, sn0 = x.SN & 0xFFu;
                c0 = c0 + (lold == s0 ? 1u : 0u) - (lold == sn0 ? 1u : 0u);
                c1 = c1 + (lsn == s0 ? 1u : 0u) - (lsn == sn0 ? 1u : 0u);
            }
            x.C0 = c0 << 2;
            x.C1 = c1 << 2;
        };

        if (slots) {
            potts_decide_slots<BOOKW, HIST && !BOOKW && SLOTS_OK, RECORD && BOOKW, TSMEM, LSMEM, BOOKW && HIST>(
                a, s_ring, s_psnap, s_snsn, s_hist, s_hdummy, tab_s, LSMEM ? s_lat + lane : glat,
                LSMEM ? (size_t)32 : gstride, lane, active, P0, P1, ap);
        } else {
        const int total_words = a.n_sweeps * L * RW;
        // the first word
        bar_sync(kBarFullU + 0, NU);
        PW cur;
        {
            cur.R = LAT(0);
            cur.u = s_ring[lane];
            columns(cur, s_ring[32 + lane], LAT((L - 1) * RW), false, 0u, 0u);
        }
        uint32_t K0 = cur.C0 & 0xFFu, K1 = cur.C1 & 0xFFu;
        uint32_t D0 = 9u * K0 - 144u, D1 = 9u * K1 - 144u;
        uint32_t A0 = TABLOAD(P0 + K0), A1 = TABLOAD(P1 + K1);
        int y = 0, w = 0, sw = 0, it = 0;
        uint32_t first_new = 0u;
        for (int q = 0; q < total_words; ++q) {
            const bool lastw = (w == RW - 1);
            const bool has_next = q + 1 < total_words;
            int y1 = y, w1 = w + 1;
            if (w1 == RW) {
                w1 = 0;
                y1 = (y + 1 == L) ? 0 : y + 1;
            }
            const bool new_slot = (w1 % kPottsSlotWords) == 0;  // the next word opens a slot
            const int it1 = it + (new_slot ? 1 : 0);
            // next word: its slot, records, old spins and row above (new)
            PW nx;
            nx.R = 0u;
            nx.SN = nx.C0 = nx.C1 = 0u;
            nx.u = make_uint4(0u, 0u, 0u, 0u);
            uint4 nr1 = nx.u;
            uint32_t nU = 0u;
            if (has_next) {
                if (new_slot) bar_sync(kBarFullU + it1 % RD, NU);
                const uint4 *src1 = s_ring + (it1 % RD) * 16 * 32 + (2 * (w1 % kPottsSlotWords)) * 32 + lane;
                nx.u = src1[0];
                nr1 = src1[32];
                nx.R = nr1.w;
                nU = LAT((y1 == 0 ? L - 1 : y1 - 1) * RW + w1);
            }
            uint32_t Fm = 0u;  // bytes of accepted sites
            uint32_t Pw[4];    // bin rows after each attempt of the word (bookkeeper)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t u = k == 0 ? cur.u.x : k == 1 ? cur.u.y : k == 2 ? cur.u.z : cur.u.w;
                if (k == 1 && RW > 1 && has_next)
                    columns(nx, nr1, nU, new_slot && w1 != 0, cur.R >> 24, cur.SN >> 24);
                if (k == 3 && RW == 1 && has_next) {
                    // one word per row: the row above of the next word is this word, whose
                    // sites 0..2 are final here (site 0 is all the next site needs)
                    nU = (cur.R & ~Fm) | (cur.SN & Fm);
                    columns(nx, nr1, nU, false, 0u, 0u);
                }
                // 1. candidates of the next site
                uint32_t Kn0 = 0u, Kn1 = 0u;
                if (k < 3) {
                    Kn0 = byte_of(cur.C0, k + 1);
                    Kn1 = byte_of(cur.C1, k + 1);
                    if (k == 2 && lastw) {
                        // row end: the right neighbour of site 3 is site 0 of the row, new
                        const uint32_t s3 = cur.R >> 24, sn3 = cur.SN >> 24;
                        const uint32_t dK = (first_new == s3 ? 4u : 0u) - (first_new == sn3 ? 4u : 0u);
                        Kn0 += dK;
                        Kn1 += dK;
                    }
                } else {
                    Kn0 = nx.C0 & 0xFFu;
                    Kn1 = nx.C1 & 0xFFu;
                }
                const uint32_t Dn0 = 9u * Kn0 - 144u, Dn1 = 9u * Kn1 - 144u;
                const uint32_t Pb = ap ? P1 : P0;
                const uint32_t PbD = ap ? P1 + D1 : P0 + D0;
                uint32_t A0n = 0u, A1n = 0u;
                if (k < 3 || has_next) {
                    A0n = TABLOAD(Pb + Kn0);
                    A1n = TABLOAD(PbD + Kn1);
                }
                // 2. decision of this site
                const uint32_t A = ap ? A1 : A0;
                const bool acc = u < A;
                Fm |= acc ? (0xFFu << (8 * k)) : 0u;
                if (k == 0 && w == 0) first_new = acc ? (cur.SN & 0xFFu) : (cur.R & 0xFFu);
                const uint32_t Pa = acc ? PbD : Pb;  // bin row after this attempt
                Pw[k] = Pa;
                if (RECORD && !BOOKW && acc) potts_count_move(cnt_lo, cnt_hi, byte_of(cur.R, k), byte_of(cur.SN, k));
                if (HIST && !BOOKW) {
                    const int bin = bin_of(Pa);
                    if (HSMEM) {
                        red_shared(active ? s_hist + bin : s_hdummy, 1u);
                    } else {
                        if (bin != run_bin) {
                            if (active)
                                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]),
                                          (unsigned long long)run);
                            run_bin = bin;
                            run = 0;
                        }
                        ++run;
                    }
                }
                // 3. state of the next site
                P0 = Pb;
                P1 = PbD;
                D0 = Dn0;
                D1 = Dn1;
                A0 = A0n;
                A1 = A1n;
                ap = acc;
            }
            LAT(y * RW + w) = (cur.R & ~Fm) | (cur.SN & Fm);
            // one word per row: now that this word is final, the next word's columns
            // (its sites 1..3) get their upper neighbours
            if (RW == 1 && has_next) columns(nx, nr1, (cur.R & ~Fm) | (cur.SN & Fm), false, 0u, 0u);
            // the slot's records are all read: release it
            if (new_slot && it < total - RD) bar_arrive(kBarEmptyU + it % RD, NU);
            if (BOOKW) {
                const int ss = q % kRingS;
                if (q >= kRingS) bar_sync(kBarEmptyS + ss, 64);
                uint4 *sn = s_psnap + ss * 2 * 32 + lane;
                if (HIST) sn[0] = make_uint4(Pw[0], Pw[1], Pw[2], Pw[3]);
                if (RECORD) sn[32] = make_uint4(Pw[3], cur.R, cur.SN, Fm);
                bar_arrive(kBarFullS + ss, 64);
            }
            if (lastw && y == L - 1) {
                if (RECORD && !BOOKW && active) {
                    const int bin = bin_of(ap ? P1 : P0);
                    const int E = bin - 2 * V;
                    const int M = 8 * potts_count_max(cnt_lo, cnt_hi) - V;
                    if (a.E_rec) a.E_rec[(size_t)sw * a.rec_stride + c] = E;
                    if (a.M_rec) a.M_rec[(size_t)sw * a.rec_stride + c] = M;
                    if (a.samples) {
                        const unsigned long long am = (unsigned long long)(M < 0 ? -M : M);
                        unsigned long long *sp = reinterpret_cast<unsigned long long *>(a.samples);
                        atomicAdd(&sp[bin], 1ull);
                        atomicAdd(&sp[a.n_bins + bin], am);
                        atomicAdd(&sp[2 * a.n_bins + bin], am * am);
                    }
                }
                ++sw;
            }
            cur = nx;
            y = y1;
            w = w1;
            it = it1;
        }
        }
        if (active) {
            if (HIST && !BOOKW && !HSMEM && run)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]), (unsigned long long)run);
            if (!RECORD) {
                uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int k = 0; k < a.lat_words; ++k) potts_count_word(LAT(k), cnt);
                cnt_lo = cnt_hi = 0;
                for (int k = 0; k < 4; ++k) {
                    cnt_lo |= (uint64_t)cnt[k] << (16 * k);
                    cnt_hi |= (uint64_t)cnt[k + 4] << (16 * k);
                }
            }
            a.E[c] = bin_of(ap ? P1 : P0) - 2 * V;
            if (!(RECORD && BOOKW)) {
                a.M[c] = 8 * potts_count_max(cnt_lo, cnt_hi) - V;
                a.cnt[c] = cnt_lo;
                a.cnt[a.p_pad + c] = cnt_hi;
            }
        }
#undef TABLOAD
        if (LSMEM)
            for (int k = 0; k < a.lat_words; ++k) a.lat[(size_t)k * a.p_pad + c] = s_lat[k * 32 + lane];
    } else if (BOOKW && vw == 4 && slots) {
        uint32_t *const s_cnt = s_snsn + kPSnapSlots * 8 * 32;  // [9][32] state counters
        if (RECORD) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                s_cnt[32 * v + lane] = (uint32_t)(bk_lo >> (16 * v)) & 0xFFFFu;
                s_cnt[32 * (v + 4) + lane] = (uint32_t)(bk_hi >> (16 * v)) & 0xFFFFu;
            }
            s_cnt[32 * 8 + lane] = 0u;
        }
        const uint32_t tab_s = TSMEM ? (uint32_t)__cvta_generic_to_shared(s_tab) : 0u;
        potts_book_slots<HIST, HPAIR, RECORD>(a, s_psnap, s_snsn, s_hist, s_hdummy, s_cnt, tab_s, lane, active, c,
                                             bk_bin0);
        if (active && RECORD) {
            uint64_t lo = 0, hi = 0;
            uint32_t mx = 0u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint32_t n0 = s_cnt[32 * v + lane], n1 = s_cnt[32 * (v + 4) + lane];
                lo |= (uint64_t)n0 << (16 * v);
                hi |= (uint64_t)n1 << (16 * v);
                mx = max(mx, max(n0, n1));
            }
            a.M[c] = 8 * (int)mx - V;
            a.cnt[c] = lo;
            a.cnt[a.p_pad + c] = hi;
        }
    } else if (BOOKW && vw == 4) {
        // ---------------- bookkeeper: histogram, state counts, records -----------
        // table addresses: shared-memory addresses, or byte offsets into the global table
        const uint32_t tab_s = TSMEM ? (uint32_t)__cvta_generic_to_shared(s_tab) : 0u;
        auto bin_of = [&](uint32_t P) { return (int)(((P - tab_s) >> 2) * 0x38E38E39u); };
        int run_bin = bk_bin0;
        uint32_t run = 0;
        const int total_words = a.n_sweeps * L * RW;
        const int words_per_sweep = L * RW;
        for (int q = 0; q < total_words; ++q) {
            const int ss = q % kRingS;
            bar_sync(kBarFullS + ss, 64);
            const uint4 *sn = s_psnap + ss * 2 * 32 + lane;
            uint4 pb = make_uint4(0u, 0u, 0u, 0u), rs = pb;
            if (HIST) pb = sn[0];
            if (RECORD) rs = sn[32];
            if (q < total_words - kRingS) bar_arrive(kBarEmptyS + ss, 64);
            if (HPAIR) {
                // one count per pair of attempts: (0, 1) and (2, 3)
                const int b0 = bin_of(pb.x), b1 = bin_of(pb.y), b2 = bin_of(pb.z), b3 = bin_of(pb.w);
                red_shared(active ? s_hist + 9 * b0 + 4 + (b1 - b0) : s_hdummy, 1u);
                red_shared(active ? s_hist + 9 * b2 + 4 + (b3 - b2) : s_hdummy, 1u);
            } else if (HIST) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int bin = bin_of(k == 0 ? pb.x : k == 1 ? pb.y : k == 2 ? pb.z : pb.w);
                    if (HSMEM) {
                        red_shared(active ? s_hist + bin : s_hdummy, 1u);
                    } else {
                        if (bin != run_bin) {
                            if (active)
                                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]),
                                          (unsigned long long)run);
                            run_bin = bin;
                            run = 0;
                        }
                        ++run;
                    }
                }
            }
            if (RECORD) {
                // rs = (bin row after the word's last attempt, old spins, proposals, accepted bytes)
                // accepted sites move one count from the old state to the new one; a
                // rejected site moves one from state 0 to state 0 (no branch)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool acc = (rs.w >> (8 * k)) & 1u;
                    potts_count_move(bk_lo, bk_hi, acc ? byte_of(rs.y, k) : 0u, acc ? byte_of(rs.z, k) : 0u);
                }
                if ((q + 1) % words_per_sweep == 0 && active) {
                    const int sw = q / words_per_sweep;
                    const int bin = bin_of(rs.x);
                    const int E = bin - 2 * V;
                    const int M = 8 * potts_count_max(bk_lo, bk_hi) - V;
                    if (a.E_rec) a.E_rec[(size_t)sw * a.rec_stride + c] = E;
                    if (a.M_rec) a.M_rec[(size_t)sw * a.rec_stride + c] = M;
                    if (a.samples) {
                        const unsigned long long am = (unsigned long long)(M < 0 ? -M : M);
                        unsigned long long *sp = reinterpret_cast<unsigned long long *>(a.samples);
                        atomicAdd(&sp[bin], 1ull);
                        atomicAdd(&sp[a.n_bins + bin], am);
                        atomicAdd(&sp[2 * a.n_bins + bin], am * am);
                    }
                }
            }
        }
        if (active) {
            if (HIST && !HSMEM && run)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[run_bin]), (unsigned long long)run);
            if (RECORD) {
                a.M[c] = 8 * potts_count_max(bk_lo, bk_hi) - V;
                a.cnt[c] = bk_lo;
                a.cnt[a.p_pad + c] = bk_hi;
            }
        }
    }
#undef LAT
    __syncthreads();
    if (HPAIR) {
        // first attempts of the pairs in bin b, then second attempts (from bin b - d)
        for (int b = tid; b < a.n_bins; b += NT) {
            uint32_t v = 0u;
#pragma unroll
            for (int d = -4; d <= 4; ++d) {
                v += s_hist[9 * b + 4 + d];
                if (b - d >= 0 && b - d < a.n_bins) v += s_hist[9 * (b - d) + 4 + d];
            }
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[b]), (unsigned long long)v);
        }
    } else if (HIST && HSMEM) {
        for (int i = tid; i < a.n_bins; i += NT) {
            const uint32_t v = s_hist[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&a.H[i]), (unsigned long long)v);
        }
    }
}

// shared memory of the Potts body beyond the staging: the draw/column ring and, with
// the bookkeeper (histogram or records), its snapshots: the larger of the word form
// ([kRingS][2][32] uint4) and the slot form ([kPSnapSlots][8][32] uint4, and for
// records the proposals [kPSnapSlots][8][32] and the state counters [9][32])
__host__ __device__ constexpr size_t potts_ws_extra_smem(bool hist, bool record)
{
    return (size_t)kPottsRing * 16 * 32 * sizeof(uint4) +
           (!(hist || record) ? 0
            : (size_t)kRingS * 2 * 32 * sizeof(uint4) >
                      (size_t)kPSnapSlots * 8 * 32 * sizeof(uint4) +
                          (record ? (size_t)kPSnapSlots * 8 * 32 * sizeof(uint32_t) + 9 * 32 * sizeof(uint32_t) : 0)
                ? (size_t)kRingS * 2 * 32 * sizeof(uint4)
                : (size_t)kPSnapSlots * 8 * 32 * sizeof(uint4) +
                      (record ? (size_t)kPSnapSlots * 8 * 32 * sizeof(uint32_t) + 9 * 32 * sizeof(uint32_t) : 0));
}
}  // namespace ws
}  // namespace muca
