// Internal declarations of libmuca (not part of the C ABI).
//
// Device data layout (chain-interleaved, so that the 32 chains of a warp touch 32
// consecutive words at every step of their lockstep typewriter sweep):
//   Ising: one bit per site, bit j of word w of row y holds site x = 32 w + j
//          (1 = spin +1); row_words = ceil(L / 32).
//   Potts: one byte per site, byte j of word w of row y holds site x = 4 w + j;
//          row_words = ceil(L / 4).
//   word k = y * row_words + w of chain c lives at lat[k * p_pad + c].
// The warp-specialised sweep kernels give each block a group of cpg <= 32 chains (fewer
// than 32 when there are fewer than 32 chains per SM, so that every SM runs some):
// p_pad = ceil(p / cpg) * 32, lanes beyond cpg work on padding columns past
// ceil(p / cpg) * cpg, and padding chains are never read back.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>

#include "muca.h"

namespace muca {

constexpr uint32_t kAlways = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the 4 x 32-bit
// S-P network, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key bumps 0x9E3779B9 /
// 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * ctr.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
    }
    return ctr;
}

// Same generator with the per-round second key word precomputed by the caller
// (k1r[r] = k1 + r * 0xBB67AE85); the first key word is warp-uniform (the seed).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 ctr, uint32_t k0, const uint32_t (&k1r)[10])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t kr0 = k0 + (uint32_t)round * 0x9E3779B9u;
        const uint32_t lo0 = 0xD2511F53u * ctr.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ kr0, lo1, hi0 ^ ctr.w ^ k1r[round], lo0);
    }
    return ctr;
}

__device__ __forceinline__ void philox_round_keys(uint32_t k1, uint32_t (&k1r)[10])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) k1r[round] = k1 + (uint32_t)round * 0xBB67AE85u;
}

// counter word 3: (seed >> 32) << 2 | phase
enum Phase : uint32_t { kPhaseInit = 0, kPhaseIterate = 1, kPhaseThermalize = 2, kPhaseProduce = 3 };

__host__ __device__ inline int n_bins_of(int model, int L)
{
    return model == MUCA_ISING ? L * L + 1 : 2 * L * L + 1;
}
__host__ __device__ inline int n_de_of(int model) { return model == MUCA_ISING ? 4 : 8; }

// Arguments of one sweep launch (plain values and device pointers).
struct SweepArgs {
    uint32_t *lat;        // [lat_words][p_pad]
    int32_t *E;           // [p_pad] running energy
    int32_t *M;           // [p_pad] running magnetisation (Ising) / record scratch
    uint64_t *cnt;        // Potts packed state counts [2][p_pad]
    const uint32_t *thr;  // [n_bins][n_de]
    const uint32_t *ktab; // kernel table: Ising [n_bins][5] by unequal neighbours, Potts [n_bins][9] by dE+4
    uint64_t *H;          // merged histogram [n_bins] (uint64, atomically added)
    int32_t *E_rec;       // [n_sweeps][rec_stride] or null
    int32_t *M_rec;
    uint64_t *samples;    // [3][n_bins] production sums (n, sum|M|, sum M^2) or null
    int L, q, p, p_pad, row_words, lat_words, n_bins;
    int cpg;              // chains per block of the warp-specialised bodies (<= 32)
    int n_sweeps;
    uint32_t sweep0;      // counter word 1 of the first sweep
    uint32_t iteration;   // counter word 2
    uint32_t ctr3;        // counter word 3 = (seed_hi << 2) | phase
    uint32_t key0;        // low 32 bits of the seed
    int rec_stride;       // records row stride (= p)
};

// staging flags of a sweep launch
struct SweepPlan {
    bool table_smem, hist_smem, lattice_smem;
    bool hist_pairs;        // warp-specialised: shared histogram of attempt pairs
    bool warp_specialized;  // decider / producer / bookkeeper warps per 32 chains
    bool compact;           // warp-specialised Ising: two blocks per SM (3-slot draw ring)
    bool t16;               // compact with a table of 16-bit threshold halves: three blocks per SM
    bool hist16;            // histogram of 16-bit counts, two bins per word, flushed by rows
    int chains_per_block;
    size_t smem_bytes;      // staging of the plan (table, histogram, lattices)
    size_t table_bytes, hist_bytes, lat_bytes;  // its parts (0: not staged)
};

// Device view of one lattice of a batch (pointers into its context).
struct BatchJob {
    int model, L, q, p, p_pad, row_words, lat_words, n_bins, n_de, V;
    int accumulated, width;
    uint32_t key0, ctr3_iter;   // seed low word; counter word 3 of weight iterations
    uint32_t *lat;
    int32_t *E, *M;
    uint64_t *cnt;
    double *lnw, *P, *wscratch;
    uint8_t *acc;
    uint32_t *thr, *ktab;
    uint64_t *H;
    muca_iter_stats *stats;
    uint32_t *iteration;        // device counter of weight iterations (counter word 2)
    int flags;                  // staging of the sweep body: 4 table, 2 histogram, 1 lattice in smem
    int *active;                // 0: the lattice is frozen (converged) and every batch kernel skips it
    int *conv;                  // iteration at which the lattice converged, -1 before
    uint32_t ctr3_therm;        // counter word 3 of thermalisation sweeps
    uint32_t *therm;            // device counter of thermalisation sweeps (counter word 1)
};

}  // namespace muca

// Host-side context (opaque to callers).
struct muca_ctx {
    int model, L, q, p, V, n_bins, n_de;
    uint64_t seed;
    muca_config cfg;
    cudaStream_t stream;
    int device;
    int cpg;                  // chains per group of the warp-specialised sweep kernels (<= 32)
    int n_sm;                 // streaming multiprocessors of the device (queried at init)
    int smem_per_sm;          // shared memory per SM and reserved per block (bytes, queried)
    int smem_reserved;
    int row_words, lat_words, p_pad;
    // device state
    uint32_t *d_lat;
    int32_t *d_E, *d_M;
    uint64_t *d_cnt;
    double *d_lnw, *d_P, *d_lnw_prod, *d_wscratch;
    uint8_t *d_acc;
    uint32_t *d_thr;
    uint32_t *d_ktab;         // thresholds re-indexed for the sweep kernels
    int ktab_dirty;
    uint64_t *d_H;
    uint64_t *d_samples;      // [3][n_bins]
    muca_iter_stats *d_stats;
    muca_iter_stats *h_stats; // pinned
    // production series scratch (used when the caller passes host or null buffers)
    int32_t *d_series;        // [2][series_cap]
    size_t series_cap;        // records per array
    // reweighting scratch: per-bin table inputs, and outputs/betas of one call
    void *d_rw;
    size_t rw_bytes;
    double *d_rwout;
    size_t rwout_cap;         // doubles
    void *d_rwtile;           // per-call tile scratch of the reweighting (grown on demand)
    size_t rwtile_bytes;
    // counters and flags
    uint32_t iteration;
    uint32_t sweeps_therm, sweeps_prod;
    int have_hist;
    int samples_active;
    uint64_t lnw_version, samples_lnw_version;
    // metric log: host clock at the start of the last iteration's sweeps, its attempts
    double it_t0, it_attempts;
};

namespace muca {

// error plumbing (thread-local message)
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
void note_launches(uint64_t n);

// NVTX range around an entry point (visible in profilers; free without one attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define MUCA_RANGE(name) ::muca::NvtxRange muca_range_(name)

// Test hook: with the environment variable MUCA_TEST_FAIL_ALLOC=k the k-th allocation
// of the process (device or pinned host memory, counting from 1) fails as if no memory
// were left, so that the clean-up of every allocation path can be tested without a GPU
// fault.
bool alloc_should_fail();

#define MUCA_CUDA_TRY(call)                                           \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::muca::cuda_fail(e_, #call);   \
    } while (0)

// launches (defined in the kernel translation units)
int launch_init_lattice(muca_ctx *ctx);
int launch_recount(muca_ctx *ctx);
int launch_sweeps(muca_ctx *ctx, uint32_t phase, int n_sweeps, uint32_t sweep0,
                  uint32_t iteration, bool hist, int32_t *E_rec, int32_t *M_rec,
                  bool samples);
int launch_unpack_spins(muca_ctx *ctx, int8_t *d_out);
int launch_thresholds(muca_ctx *ctx);
int launch_update(muca_ctx *ctx);
int launch_stats(muca_ctx *ctx);
int launch_reweight(muca_ctx *ctx, const double *d_betas, int n_beta, int precision,
                    double *const out[4] /* e, C, absm, chi: device [n_beta] each */);
SweepPlan plan_sweeps(const muca_ctx *ctx, bool allow_pairs = true, bool allow_compact = true);
int plan_flags(const SweepPlan &pl);  // MUCA_PLAN_* bit mask
cudaError_t launch_batch_update(const BatchJob *d_jobs, int n_jobs, int max_thr, cudaStream_t st);
int launch_ktab(muca_ctx *ctx);
// Scratch of the tiled reweighting kernels (reweight_kernels.cu): a per-bin part (five
// FP64 arrays, a float copy of ln Omega, the sampled range) and a per-call part for
// n_beta betas (tile parameters, shifts, item offsets, partial sums), 256-byte aligned
// pieces.
constexpr int kRwTile = 8;          // betas per tile
constexpr int kRwMaxChunks = 32;    // bin chunks per tile at most
constexpr size_t kRwTileParamsBytes = 72;
constexpr size_t rw_align256(size_t b) { return (b + 255) & ~(size_t)255; }
// per-bin part: five FP64 arrays, five float arrays (ln Omega and mean |M| as float
// pairs, the within-bin variance), the sampled range of every block of the preparation
// kernel (256 bins each), and the completion counter of the setup kernel (zero between
// calls: zeroed with the scratch, reset by its last user)
constexpr size_t rw_bin_part_bytes(size_t nb)
{
    return rw_align256(5 * nb * 8) + 5 * rw_align256(nb * 4) + rw_align256(8 * ((nb + 255) / 256)) + 256;
}
// per-call part: tile parameters, shifts (FP64, and the float constants of every beta),
// every beta's reference bin (mean |M| in FP64 and as a float pair),
// item offsets, the tiles' completion counters (each zeroed by its setup block), the
// tile of every item, partial sums
constexpr size_t rw_tile_part_bytes(size_t n_beta)
{
    return rw_align256(kRwTileParamsBytes * ((n_beta + kRwTile - 1) / kRwTile)) + rw_align256(8 * n_beta) +
           rw_align256(16 * n_beta) + rw_align256(8 * n_beta) + rw_align256(8 * n_beta) +
           rw_align256(4 * ((n_beta + kRwTile - 1) / kRwTile + 1)) +
           rw_align256(4 * ((n_beta + kRwTile - 1) / kRwTile + 1)) +
           rw_align256(4 * ((n_beta + kRwTile - 1) / kRwTile) * kRwMaxChunks) +
           8 * ((n_beta + kRwTile - 1) / kRwTile) * kRwMaxChunks * kRwTile * 6;
}
// allocation-free reweighting (reweight_noalloc.cu): the bins and betas per pass it
// serves, its fixed scratch and the launch on caller buffers
constexpr int kNoallocMaxBins = 16385;       // Ising L <= 128, 8-Potts L <= 90
constexpr int kNoallocBetasPerPass = 512;
constexpr size_t kNoallocScratchBytes = rw_bin_part_bytes(kNoallocMaxBins) + rw_tile_part_bytes(kNoallocBetasPerPass);
cudaError_t launch_reweight_buffers(double *scratch, const uint64_t *samples, const double *lnw, int model, int L,
                                    int q, const double *d_betas, int n_beta, int precision, double *d_out, int n_sm,
                                    cudaStream_t st);
// shared memory of a warp-specialised launch beyond its staging, for launches with a
// histogram and / or records (the defaults: the largest)
size_t ws_extra_smem(int model, bool compact = false, bool hist = true, bool record = true);
// multimagnetic Ising ensemble (muma.cu)
int launch_muma_thresholds(muca_ctx *ctx);
int launch_muma_sweeps(muca_ctx *ctx, uint32_t phase, int n_sweeps, uint32_t sweep0, uint32_t iteration, bool hist,
                       int32_t *E_rec, int32_t *M_rec);
cudaError_t launch_ws_sweep(const SweepArgs &a, const SweepPlan &pl, int model, int blocks, bool hist, bool record,
                            cudaStream_t st);

}  // namespace muca
