/*
 * muca_oracle.c -- plain CPU oracle for the parallel multicanonical (MUCA) method
 * of Zierenberg, Marenz and Janke, "Scaling Properties of a Parallel Implementation
 * of the Multicanonical Algorithm" (arXiv:1212.3975).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct statement of
 * what the GPU path computes.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and it never calls it.
 *
 * What it covers (the weight recursion and the reweighting live in oracle/*.py):
 *   - the Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
 *     the source of every random number a chain draws;
 *   - the two Hamiltonians of Sec. 3 (Eq. 3 Ising, Eq. 4 q-state Potts) on a periodic
 *     L x L square lattice;
 *   - the start at infinite temperature (Sec. 3: "start at ... beta = 0");
 *   - typewriter sweeps of V = L*L single-spin updates (Sec. 3, last sentence) with
 *     the multicanonical acceptance min(1, W(E')/W(E)) implied by Eq. 1, realised as
 *     an integer threshold test on a raw 32-bit draw;
 *   - the per-chain energy histograms H_i(E) of the parallel version (Sec. 2,
 *     "Parallel Version"), and the (E, M) records of the production run (Sec. 5).
 *
 * Readings where the paper is silent (each one is also listed in the design notes):
 *   - periodic boundaries; site i = y*L + x, x fastest; sweep order = i ascending;
 *   - Philox key = (low 32 bits of seed, chain id); counter = (site group, sweep,
 *     iteration, (high 32 bits of seed << 2) | phase), phase 0 init, 1 weight
 *     iteration, 2 thermalisation, 3 production;
 *     Ising: group = i >> 2, acceptance draw u = word[i & 3];
 *     Potts: group = i >> 1, u = word[2*(i & 1)], proposal draw = word[2*(i & 1) + 1];
 *     init:  group = i >> 2, word[i & 3]; Ising s = +1 iff its top bit is set,
 *            Potts s = (word * q) >> 32;
 *   - Potts proposal s' = (s + 1 + ((word * (q - 1)) >> 32)) mod q (uniform over the
 *     q - 1 other states);
 *   - acceptance: dE = 0 always accepted; otherwise the threshold A for the current
 *     bin and dE is read from a table and the move is accepted iff
 *     A == 0xFFFFFFFF or u < A;
 *   - after every attempt (accepted or not) the chain histogram at the current
 *     energy is incremented, so one sweep adds exactly V entries per chain.
 *
 * Energies and bins: Ising E = -sum_<ij> s_i s_j in [-2V, 2V] step 4, bin (E + 2V)/4;
 * Potts E = -sum_<ij> delta(s_i, s_j) in [-2V, 0], bin E + 2V.
 * Magnetisation: Ising M = sum_i s_i; Potts M = q * max_k N_k - V (N_k = sites in
 * state k).
 *
 * Spin storage here is one byte per site, chain-major: spins[c * V + i]; Ising spins
 * are stored as +1 / -1 (int8), Potts spins as 0 .. q-1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ISING 0
#define ORC_POTTS 1

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-P network with */
/* multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,      */
/* 0xBB67AE85 applied between rounds.                                          */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 4-word Philox block for (chain, site group, sweep, iteration, phase). */
static void draw_block(uint64_t seed, int64_t chain, uint32_t group, uint32_t sweep,
                       uint32_t iteration, uint32_t phase, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = group;
    ctr[1] = sweep;
    ctr[2] = iteration;
    ctr[3] = ((uint32_t)(seed >> 32) << 2) | (phase & 3u);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)chain;
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------- */
/* Lattice and Hamiltonians (Sec. 3, Eqs. 3 and 4)                            */
/* ------------------------------------------------------------------------- */
static int site_of(int L, int x, int y) { return y * L + x; }

/* Full energy of one configuration: every bond counted once through the right and
 * the down neighbour of each site. */
int64_t orc_energy(int model, int L, const int8_t *s)
{
    int64_t E = 0;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int i = site_of(L, x, y);
            int r = site_of(L, (x + 1) % L, y);
            int d = site_of(L, x, (y + 1) % L);
            if (model == ORC_ISING) {
                E -= (int64_t)s[i] * s[r];
                E -= (int64_t)s[i] * s[d];
            } else {
                E -= (s[i] == s[r]);
                E -= (s[i] == s[d]);
            }
        }
    }
    return E;
}

/* Ising: M = sum of spins.  Potts: M = q * max_k N_k - V. */
int64_t orc_magnetization(int model, int L, int q, const int8_t *s)
{
    int V = L * L;
    if (model == ORC_ISING) {
        int64_t M = 0;
        for (int i = 0; i < V; ++i) M += s[i];
        return M;
    }
    int64_t count[256];
    for (int k = 0; k < q; ++k) count[k] = 0;
    for (int i = 0; i < V; ++i) count[(uint8_t)s[i]] += 1;
    int64_t mx = 0;
    for (int k = 0; k < q; ++k) if (count[k] > mx) mx = count[k];
    return (int64_t)q * mx - V;
}

int orc_n_bins(int model, int L) { int V = L * L; return model == ORC_ISING ? V + 1 : 2 * V + 1; }
int orc_n_de(int model) { return model == ORC_ISING ? 4 : 8; }

static int64_t bin_of(int model, int L, int64_t E)
{
    int64_t V = (int64_t)L * L;
    return model == ORC_ISING ? (E + 2 * V) / 4 : E + 2 * V;
}

/* Column of the threshold table for an energy change dE != 0.
 * Ising: dE in {-8, -4, 4, 8}   -> columns 0..3 (ascending dE).
 * Potts: dE in {-4..-1, 1..4}   -> columns 0..7 (ascending dE). */
static int column_of(int model, int dE)
{
    if (model == ORC_ISING) {
        int k = dE / 4;                 /* -2, -1, 1, 2 */
        return k < 0 ? k + 2 : k + 1;
    }
    return dE < 0 ? dE + 4 : dE + 3;
}

/* ------------------------------------------------------------------------- */
/* Start at infinite temperature (Sec. 3): i.i.d. uniform spins.              */
/* ------------------------------------------------------------------------- */
int orc_init(int model, int L, int q, uint64_t seed, int64_t chain0, int n_chains,
             int8_t *spins, int64_t *E, int64_t *M)
{
    int V = L * L;
    for (int c = 0; c < n_chains; ++c) {
        int8_t *s = spins + (int64_t)c * V;
        for (int i = 0; i < V; ++i) {
            uint32_t w[4];
            draw_block(seed, chain0 + c, (uint32_t)(i >> 2), 0u, 0u, 0u, w);
            uint32_t word = w[i & 3];
            if (model == ORC_ISING)
                s[i] = (word >> 31) ? (int8_t)1 : (int8_t)-1;
            else
                s[i] = (int8_t)(((uint64_t)word * (uint64_t)q) >> 32);
        }
        E[c] = orc_energy(model, L, s);
        M[c] = orc_magnetization(model, L, q, s);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One chain, n_sweeps typewriter sweeps (Sec. 3: a sweep is V spin updates).  */
/* thr: [n_bins][n_de] acceptance thresholds (uint32), the integer form of      */
/*      W(E')/W(E).                                                            */
/* H:   [n_bins] per-chain histogram, incremented after every attempt (or NULL).*/
/* E_rec/M_rec: one record per sweep with stride rec_stride (or NULL).          */
/* Returns 0, or -1 if the running E/M ever disagree with a full recomputation.*/
/* ------------------------------------------------------------------------- */
static int run_chain(int model, int L, int q, uint64_t seed, uint32_t phase,
                     uint32_t iteration, uint32_t sweep0, int n_sweeps, int64_t chain,
                     int8_t *s, int64_t *E_io, int64_t *M_io, const uint32_t *thr,
                     uint64_t *H, int32_t *E_rec, int32_t *M_rec, int64_t rec_stride)
{
    int V = L * L;
    int n_de = orc_n_de(model);
    int64_t E = *E_io, M = *M_io;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint32_t sweep = sweep0 + (uint32_t)sw;
        for (int i = 0; i < V; ++i) {
            int x = i % L, y = i / L;
            int nb[4];
            nb[0] = site_of(L, (x + 1) % L, y);
            nb[1] = site_of(L, (x + L - 1) % L, y);
            nb[2] = site_of(L, x, (y + 1) % L);
            nb[3] = site_of(L, x, (y + L - 1) % L);
            uint32_t w[4];
            uint32_t u, proposal_word = 0;
            if (model == ORC_ISING) {
                draw_block(seed, chain, (uint32_t)(i >> 2), sweep, iteration, phase, w);
                u = w[i & 3];
            } else {
                draw_block(seed, chain, (uint32_t)(i >> 1), sweep, iteration, phase, w);
                u = w[2 * (i & 1)];
                proposal_word = w[2 * (i & 1) + 1];
            }
            int old = s[i], neu;
            int dE;
            if (model == ORC_ISING) {
                neu = -old;
                int sum = s[nb[0]] + s[nb[1]] + s[nb[2]] + s[nb[3]];
                dE = 2 * old * sum;             /* E' - E for s_i -> -s_i (Eq. 3) */
            } else {
                int shift = (int)(((uint64_t)proposal_word * (uint64_t)(q - 1)) >> 32);
                neu = (old + 1 + shift) % q;
                int same_old = 0, same_new = 0;
                for (int k = 0; k < 4; ++k) {
                    same_old += (s[nb[k]] == old);
                    same_new += (s[nb[k]] == neu);
                }
                dE = same_old - same_new;       /* E' - E (Eq. 4) */
            }
            int accept;
            if (dE == 0) {
                accept = 1;
            } else {
                int64_t b = bin_of(model, L, E);
                uint32_t A = thr[b * n_de + column_of(model, dE)];
                accept = (A == 0xFFFFFFFFu) || (u < A);
            }
            if (accept) {
                s[i] = (int8_t)neu;
                E += dE;
                if (model == ORC_ISING) M += neu - old;
            }
            if (H) H[bin_of(model, L, E)] += 1;
        }
        /* Invariant: incremental energy (and Ising magnetisation) equal a recount. */
        if (orc_energy(model, L, s) != E) return -1;
        if (model == ORC_ISING) {
            if (orc_magnetization(model, L, q, s) != M) return -1;
        } else {
            M = orc_magnetization(model, L, q, s);
        }
        if (E_rec) E_rec[(int64_t)sw * rec_stride] = (int32_t)E;
        if (M_rec) M_rec[(int64_t)sw * rec_stride] = (int32_t)M;
    }
    *E_io = E;
    *M_io = M;
    return 0;
}

/* n_chains chains with global ids chain0 .. chain0 + n_chains - 1.
 * spins: [n_chains][V]; E, M: [n_chains];
 * H: [n_chains][n_bins] per-chain histograms (added to) or NULL;
 * E_rec, M_rec: [n_sweeps][n_chains] records or NULL.
 * Chains are independent; OpenMP runs them on the host cores. */
int orc_sweeps(int model, int L, int q, uint64_t seed, int phase, uint32_t iteration,
               uint32_t sweep0, int n_sweeps, int64_t chain0, int n_chains,
               int8_t *spins, int64_t *E, int64_t *M, const uint32_t *thr,
               uint64_t *H, int32_t *E_rec, int32_t *M_rec)
{
    int V = L * L;
    int nb = orc_n_bins(model, L);
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:status)
    for (int c = 0; c < n_chains; ++c) {
        status |= run_chain(model, L, q, seed, (uint32_t)phase, iteration, sweep0, n_sweeps,
                            chain0 + c, spins + (int64_t)c * V, &E[c], &M[c], thr,
                            H ? H + (int64_t)c * nb : NULL,
                            E_rec ? E_rec + c : NULL, M_rec ? M_rec + c : NULL,
                            (int64_t)n_chains);
    }
    return status ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Multimagnetic Ising (Sec. 4, Fig. 6): weights in the magnetisation M at a    */
/* fixed inverse temperature beta, i.e. the chain samples W(M) exp(-beta E).    */
/* Readings: bin of M = (M + V) / 2 (all V + 1 bins reachable); the threshold   */
/* table has 10 columns per bin, column 5 * (s == +1) + n for the flipped spin  */
/* s and its n unequal neighbours (0..4), so that E' - E = 8 - 4n and the bin    */
/* moves to (M - 2s + V) / 2; the random streams, the sweep order and the        */
/* acceptance test are those of the Ising chain above; after every attempt the   */
/* chain histogram at the current M bin is incremented.                          */
/* ------------------------------------------------------------------------- */
static int run_muma_chain(int L, uint64_t seed, uint32_t phase, uint32_t iteration, uint32_t sweep0,
                          int n_sweeps, int64_t chain, int8_t *s, int64_t *E_io, int64_t *M_io,
                          const uint32_t *thr, uint64_t *H, int32_t *E_rec, int32_t *M_rec,
                          int64_t rec_stride)
{
    int V = L * L;
    int64_t E = *E_io, M = *M_io;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint32_t sweep = sweep0 + (uint32_t)sw;
        for (int i = 0; i < V; ++i) {
            int x = i % L, y = i / L;
            int nb[4];
            nb[0] = site_of(L, (x + 1) % L, y);
            nb[1] = site_of(L, (x + L - 1) % L, y);
            nb[2] = site_of(L, x, (y + 1) % L);
            nb[3] = site_of(L, x, (y + L - 1) % L);
            uint32_t w[4];
            draw_block(seed, chain, (uint32_t)(i >> 2), sweep, iteration, phase, w);
            uint32_t u = w[i & 3];
            int old = s[i];
            int unequal = 0;
            for (int k = 0; k < 4; ++k) unequal += (s[nb[k]] != old);
            int64_t b = (M + V) / 2;
            uint32_t A = thr[b * 10 + 5 * (old == 1) + unequal];
            if ((A == 0xFFFFFFFFu) || (u < A)) {
                s[i] = (int8_t)(-old);
                E += 8 - 4 * unequal;
                M -= 2 * old;
            }
            if (H) H[(M + V) / 2] += 1;
        }
        if (orc_energy(ORC_ISING, L, s) != E) return -1;
        if (orc_magnetization(ORC_ISING, L, 2, s) != M) return -1;
        if (E_rec) E_rec[(int64_t)sw * rec_stride] = (int32_t)E;
        if (M_rec) M_rec[(int64_t)sw * rec_stride] = (int32_t)M;
    }
    *E_io = E;
    *M_io = M;
    return 0;
}

/* As orc_sweeps for the multimagnetic Ising chain; thr: [V + 1][10]; H: [n_chains][V + 1]. */
int orc_muma_sweeps(int L, uint64_t seed, int phase, uint32_t iteration, uint32_t sweep0, int n_sweeps,
                    int64_t chain0, int n_chains, int8_t *spins, int64_t *E, int64_t *M, const uint32_t *thr,
                    uint64_t *H, int32_t *E_rec, int32_t *M_rec)
{
    int V = L * L;
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:status)
    for (int c = 0; c < n_chains; ++c) {
        status |= run_muma_chain(L, seed, (uint32_t)phase, iteration, sweep0, n_sweeps, chain0 + c,
                                 spins + (int64_t)c * V, &E[c], &M[c], thr,
                                 H ? H + (int64_t)c * (V + 1) : NULL,
                                 E_rec ? E_rec + c : NULL, M_rec ? M_rec + c : NULL, (int64_t)n_chains);
    }
    return status ? -1 : 0;
}

/* Threads of the OpenMP loops over chains (the CPU-baseline timing runs 1 and all). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
