/*
 * muca.h -- C ABI of the GB300 (sm_103a) parallel multicanonical library, libmuca.so.
 *
 * Method: Zierenberg, Marenz and Janke, "Scaling Properties of a Parallel
 * Implementation of the Multicanonical Algorithm" (arXiv:1212.3975).  p independent
 * Markov chains share one set of logarithmic weights ln W(E) (Sec. 2, Parallel
 * Version); each runs single-spin-flip sweeps of the 2D Ising model (Eq. 3) or the
 * 8-state Potts model (Eq. 4) on a periodic L x L lattice with acceptance
 * min(1, W(E')/W(E)) (Eq. 1); their energy histograms are merged, H = sum_i H_i, and
 * feed the recursive ln W update with boundary correction and convergence test
 * (Secs. 2-3); a production run then records (E, M) per sweep, and Eq. 2 reweights
 * the records to many inverse temperatures (Sec. 5 for C_V).
 *
 * Conventions shared by every entry point:
 *  - Return value: MUCA_OK (0) or a negative MUCA_ERR_* code; muca_last_error()
 *    then returns a message (thread-local, valid until the next call on the thread).
 *  - Memory: the context owns the lattices, weights, tables, histograms and scratch
 *    buffers on the GPU; the caller owns every pointer it passes in.  A caller buffer
 *    may be host or device memory: device pointers (cudaMalloc, torch tensors) are
 *    read/written asynchronously on the context's stream; host pointers are read or
 *    written before the call returns (the call synchronises the stream).
 *  - Streams: all work of a context runs in order on the stream given to muca_init.
 *  - Thread safety: a context may be used by one host thread at a time.
 *  - Energies/bins: Ising E = -sum_<ij> s_i s_j in [-2V, 2V] step 4, bin (E+2V)/4,
 *    n_bins = V+1; Potts E = -sum_<ij> delta(s_i, s_j) in [-2V, 0], bin E+2V,
 *    n_bins = 2V+1 (V = L*L).  Inaccessible bins (Ising E = +-(2V-4); Potts 1, 2, 3
 *    and 5 broken bonds) keep ln W = 0 and are never entered.
 *  - Random numbers: Philox4x32-10 with key (low 32 bits of seed, chain id) and
 *    counter (site group, sweep, iteration, (seed >> 32) << 2 | phase); a chain's
 *    trajectory therefore depends only on (seed, chain id, weights), never on p.
 */
#ifndef MUCA_H
#define MUCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* models (Sec. 3) */
#define MUCA_ISING 0
#define MUCA_POTTS 1

/* status codes */
#define MUCA_OK 0
#define MUCA_ERR_ARG (-1)     /* invalid argument or size */
#define MUCA_ERR_CUDA (-2)    /* a CUDA call failed (message names it) */
#define MUCA_ERR_OOM (-3)     /* device allocation failed */
#define MUCA_ERR_TIMEOUT (-4) /* a bounded device wait gave up */
#define MUCA_ERR_STATE (-5)   /* call not valid in the context's current state */
#define MUCA_ERR_IO (-6)      /* checkpoint file could not be read or written */

/* reweighting arithmetic for the beta x E table and its contraction */
#define MUCA_FP64 0
#define MUCA_FP32 1
#define MUCA_BF16 2

/* weight recursions (Sec. 2) */
#define MUCA_RECURSION_ACCUMULATED 0 /* error-weighted, uses all past iterations */
#define MUCA_RECURSION_SIMPLE 1      /* W^(n+1) = W^(n) / H^(n) */

/* lattice staging of the sweep kernels */
#define MUCA_STAGING_AUTO 0
#define MUCA_STAGING_SHARED 1 /* lattices copied into shared memory for a launch */
#define MUCA_STAGING_GLOBAL 2 /* lattices stay in global memory (L2 / HBM) */

/* ensembles: weights in the energy (multicanonical, Secs. 2-3) or, for the Ising
 * model, in the magnetisation at a fixed inverse temperature (multimagnetic, Sec. 4
 * and Fig. 6: the chain samples W(M) exp(-beta E); bins M = -V..V in steps of 2) */
#define MUCA_ENSEMBLE_ENERGY 0
#define MUCA_ENSEMBLE_MAGNETIZATION 1

typedef struct muca_config {
    int recursion;        /* MUCA_RECURSION_*; default accumulated */
    int correction_width; /* bins for the boundary slope (Sec. 3); 0 -> L */
    int chains_per_block; /* multiple of 32, <= 256; 0 -> automatic */
    int staging;          /* MUCA_STAGING_*; 0 -> automatic */
    int ensemble;         /* MUCA_ENSEMBLE_*; 0 -> energy */
    double beta;          /* inverse temperature of the multimagnetic ensemble */
} muca_config;

/* Convergence statistics of one merged histogram over the accessible bins (Sec. 3:
 * full range covered and every entry within [1/2, 2] of the mean). */
typedef struct muca_iter_stats {
    int32_t covered;       /* every accessible bin has H > 0 */
    int32_t flat;          /* covered and 0.5*mean <= H <= 2*mean everywhere */
    int32_t lo, hi;        /* lowest / highest sampled accessible bin, -1 if none */
    int64_t n_sampled;     /* accessible bins with H > 0 */
    double min_over_mean;  /* min H / mean H */
    double max_over_mean;  /* max H / mean H */
    uint64_t total;        /* sum of H */
} muca_iter_stats;

typedef struct muca_ctx muca_ctx;

/* Message of the last failing call on this host thread ("" if none). */
const char *muca_last_error(void);

/* Number of kernels this library has launched in the process (all contexts). */
uint64_t muca_kernel_launches(void);

/* Create p chains of the given model on an L x L periodic lattice (Sec. 3) and start
 * them at infinite temperature: i.i.d. uniform spins, ln W = 0 (Sec. 3).
 * With cfg->ensemble = MUCA_ENSEMBLE_MAGNETIZATION (Ising only) the weights, the
 * histograms and the convergence test are over the V+1 magnetisation bins
 * (M + V)/2 and the acceptance includes exp(-cfg->beta dE); production then records
 * (E, M) per sweep but keeps no energy sums, so the reweighting and interface-tension
 * calls return MUCA_ERR_STATE, and batches reject such contexts.
 *  model: MUCA_ISING (q must be 2, L even, 4 <= L <= 1024) or MUCA_POTTS (q must
 *         be 8, 3 <= L <= 255); p: 1 <= p <= 2^24 chains; seed: seed >> 32 < 2^30.
 *  cfg:   NULL for defaults; cuda_stream: a cudaStream_t, NULL = legacy default.
 * On success *out owns device memory until muca_destroy.
 * Errors: MUCA_ERR_ARG, MUCA_ERR_OOM, MUCA_ERR_CUDA. */
int muca_init(muca_ctx **out, int model, int L, int q, int p, uint64_t seed,
              const muca_config *cfg, void *cuda_stream);

/* Release every device buffer of the context (synchronises its stream). */
int muca_destroy(muca_ctx *ctx);

/* Start the same chains again at infinite temperature with a new seed (Sec. 3):
 * fresh i.i.d. spins, ln W = 0, recursion accumulator, histogram, production sums
 * and all counters cleared.  No allocation; asynchronous on the context's stream.
 * Errors: MUCA_ERR_ARG (seed >> 32 >= 2^30), MUCA_ERR_CUDA. */
int muca_reset(muca_ctx *ctx, uint64_t seed);

int muca_n_bins(const muca_ctx *ctx); /* V+1 (Ising) or 2V+1 (Potts); <0 on error */
int muca_n_de(const muca_ctx *ctx);   /* threshold-table columns: 4 or 8 */
int muca_num_chains(const muca_ctx *ctx);

/* One weight iteration's sampling (Sec. 2, Parallel Version): every chain continues
 * from its last state (Sec. 4) and runs n_sweeps typewriter sweeps of V updates with
 * the current weights; after every attempt the energy bin is histogrammed.  The
 * per-chain histograms are merged into H(E) = sum_i H_i(E) (uint64), kept in the
 * context for muca_update_weights and copied to H_out[n_bins] when non-NULL.
 * The iteration counter of the random streams advances by one.
 * Errors: MUCA_ERR_ARG (n_sweeps < 1), MUCA_ERR_CUDA. */
int muca_iterate(muca_ctx *ctx, int n_sweeps, uint64_t *H_out);

/* Estimate the next weights from the last merged histogram (Secs. 2-3): the
 * configured recursion in log form, then the boundary correction that extends
 * ln W linearly beyond the sampled range with the slope of the innermost
 * correction_width bins, then ln W -= max over accessible bins; the acceptance
 * thresholds are rebuilt from the new ln W.  Convergence statistics of the histogram
 * are written to *out when non-NULL (host pointer).
 * Errors: MUCA_ERR_STATE (no histogram since the last update), MUCA_ERR_CUDA. */
int muca_update_weights(muca_ctx *ctx, muca_iter_stats *out);

/* Weight iterations until convergence (Sec. 3; the study of Sec. 4 counts them):
 * muca_iterate(n_sweeps) + muca_update_weights, repeated until the merged histogram
 * of an iteration is covered and flat, or max_iterations were run.  The update of
 * the converged iteration is applied, so the context holds the weights that follow
 * it.  therm_sweeps > 0: after every update that did not converge (and is not the
 * last allowed iteration) the chains are thermalised for that many sweeps with the
 * new weights (muca_thermalize), the intermediate thermalisation of Sec. 4.
 * *n_iter_out (host, may be NULL) = the number of iterations run when the last one
 * converged (the paper's N_iter), -1 if none did; *last (host, may be NULL) = the
 * statistics of the last iteration.  Synchronises once per iteration.
 * Errors: MUCA_ERR_ARG (n_sweeps < 1, therm_sweeps < 0 or max_iterations < 1),
 * MUCA_ERR_CUDA. */
int muca_converge(muca_ctx *ctx, int n_sweeps, int therm_sweeps, int max_iterations, int *n_iter_out,
                  muca_iter_stats *last);

/* Thermalise every chain with the current weights for n_sweeps sweeps (Sec. 3:
 * "thermalized again" before production); nothing is recorded. */
int muca_thermalize(muca_ctx *ctx, int n_sweeps);

/* Production run (Sec. 5): n_sweeps sweeps per chain at the current weights; after
 * each sweep the chain's energy E and magnetisation M are recorded (Ising M = sum s;
 * Potts M = q max_k N_k - V) into E_out / M_out laid out [n_sweeps][p] (int32),
 * which may be NULL.  The records are also accumulated into per-bin exact sums
 * (count, sum |M|, sum M^2) that muca_reweight uses.  The weights in force at the
 * first production call after muca_init / muca_reset_samples are the ones the
 * records are reweighted with; changing the weights in between is MUCA_ERR_STATE. */
int muca_produce(muca_ctx *ctx, int n_sweeps, int32_t *E_out, int32_t *M_out);

/* Forget the accumulated production sums. */
int muca_reset_samples(muca_ctx *ctx);

/* Replace the production sums by caller-supplied ones (n, sum |M|, sum M^2 per bin,
 * [n_bins] uint64 each, host or device; e.g. sums saved from an earlier run or test
 * inputs) and take the context's current ln W as the weights they were produced with;
 * muca_reweight and the interface-tension calls then use them, and later production
 * records add to them.  Errors: MUCA_ERR_ARG, MUCA_ERR_STATE (multimagnetic ensemble). */
int muca_set_samples(muca_ctx *ctx, const uint64_t *n, const uint64_t *sum_abs_m, const uint64_t *sum_m2);

/* Time-series reweighting of all production records (Eq. 2) to n_beta inverse
 * temperatures betas[] (host or device, FP64).  Per beta it writes
 *   e    = <E>/V,  C = beta^2 (<E^2> - <E>^2)/V  (C_V of Sec. 5),
 *   absm = <|M|>/Mnorm,  chi = beta V (<m^2> - <|m|>^2),  m = M/Mnorm,
 * Mnorm = V (Ising) or (q-1) V (Potts); any output pointer may be NULL.
 * precision selects the arithmetic of the beta x E weight table and its contraction:
 *  MUCA_FP64  exponents, weights and sums in FP64 (terms below e^-100 of a beta's
 *             largest skipped);
 *  MUCA_FP32  exponents and sums as float pairs (compensated), partial sums combined in
 *             FP64: within ~2e-7 of FP64 on the configurations' beta grids;
 *  MUCA_BF16  tensor cores: weights and columns split into three BF16 terms, FP32
 *             accumulation flushed to FP64 per 16 bins.
 * FP64 and FP32 centre every beta's columns on its own reference bin (the bin where its
 * weights peak), so scattered or far betas are fine; BF16 centres each tile of 16
 * consecutive betas on one bin (the columns are the shared operand of the product), so
 * its C and chi are accurate only where a tile's betas peak close together, as on a
 * dense sorted grid: use MUCA_FP32 otherwise.  Observables are formed in FP64.
 * Errors: MUCA_ERR_STATE (no records), MUCA_ERR_ARG. */
int muca_reweight(muca_ctx *ctx, const double *betas, int n_beta, int precision,
                  double *e, double *C, double *absm, double *chi);

/* Reweighting without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * want observables -- e.g. an application whose framework allocator already holds
 * the free device memory, or a latency-critical loop that must not stall on
 * cudaMalloc/cudaFree (cudaFree synchronises the device).
 * In FP64 or FP32 it computes what muca_reweight computes (Eq. 2, same outputs, same
 * kernels; BF16 is not offered here) from
 * caller-owned DEVICE buffers, without a context:
 *   samples [3][n_bins] uint64 (count, sum |M|, sum M^2 per bin, as muca_get_samples),
 *   lnw [n_bins] FP64 (the weights the samples were produced with), betas [n_beta],
 *   out [4][n_beta] FP64 (rows e, C, absm, chi); precision MUCA_FP64 or MUCA_FP32;
 *   work is queued on cuda_stream (NULL = legacy default stream).
 * Its scratch is one fixed array inside the library's device image, 1,806,336 bytes:
 * per-bin arrays for up to 16385 bins and the tile sums of 512 betas (more betas are
 * taken 512 at a time); lattices with more than 16385 bins (Ising L > 128, 8-Potts
 * L > 90) are rejected with MUCA_ERR_ARG.  The image, and with it the array, is
 * loaded onto a GPU by the first call on that device (CUDA loads modules lazily by
 * default), so that first call needs 1,806,336 bytes of free device memory once and
 * can fail with MUCA_ERR_CUDA when none is left: make it at start-up, before any
 * stream capture.  From then on the GPU holds the array until the process exits.
 * Every call looks the array's address up for the current device and context
 * (cudaGetSymbolAddress), so a device reset is harmless.  All calls share the array:
 * calls that overlap on the GPU (e.g. on two streams) race and give wrong results;
 * serialise them.  Each call writes or clears every scratch entry it reads, so nothing
 * needs clearing between calls.  Only MUCA_FP64 and MUCA_FP32 are supported.
 * Errors: MUCA_ERR_ARG (bad model/size, precision, host pointers or buffers of
 * another device, too many bins), MUCA_ERR_CUDA. */
int muca_reweight_noalloc(int model, int L, int q, const uint64_t *samples, const double *lnw,
                          const double *betas, int n_beta, int precision, double *out,
                          void *cuda_stream);

/* State access (host or device buffers).
 * lnw: [n_bins] FP64; thresholds: [n_bins][n_de] uint32, column j = ascending dE
 * (Ising dE = -8,-4,4,8; Potts dE = -4..-1,1..4), A = 0xFFFFFFFF or u < A accepts;
 * spins: [p][V] int8 (Ising +1/-1, Potts 0..q-1), site i = y*L + x;
 * E, M: [p] int64 (host only); H: [n_bins] uint64 (last merged histogram);
 * samples: n, sum|M|, sum M^2 each [n_bins] uint64. */
int muca_get_lnw(muca_ctx *ctx, double *lnw);
int muca_set_lnw(muca_ctx *ctx, const double *lnw); /* also rebuilds thresholds */
int muca_get_thresholds(muca_ctx *ctx, uint32_t *thr);
int muca_set_thresholds(muca_ctx *ctx, const uint32_t *thr); /* until next update */
int muca_get_spins(muca_ctx *ctx, int8_t *spins);
int muca_get_energies(muca_ctx *ctx, int64_t *E, int64_t *M);
int muca_get_histogram(muca_ctx *ctx, uint64_t *H);
int muca_get_samples(muca_ctx *ctx, uint64_t *n, uint64_t *sum_abs_m, uint64_t *sum_m2);
int muca_get_iteration(const muca_ctx *ctx); /* weight iterations done */

/* How the sweep kernels stage this context's chains (introspection for tests and
 * tuning; the choice depends on L, p, the device and cfg->staging): a bit mask of
 *  MUCA_PLAN_LATTICE_SMEM   lattices in shared memory (else global memory, L1/L2),
 *  MUCA_PLAN_HIST_SMEM      block histogram in shared memory (else global atomics),
 *  MUCA_PLAN_TABLE_SMEM     threshold table in shared memory (else global memory),
 *  MUCA_PLAN_PAIR_HIST      histogram of pairs of consecutive attempts,
 *  MUCA_PLAN_COMPACT        compact staging, two blocks per SM (more groups of 32
 *                           chains than SMs),
 *  MUCA_PLAN_WARP_SPECIALIZED  decider / producer / bookkeeper warps (L % 4 == 0),
 *  MUCA_PLAN_TABLE16        compact staging with the upper 16 bits of the thresholds
 *                           in shared memory, three blocks per SM (Ising, L % 32 == 0,
 *                           L >= 64, more than two groups of 32 chains per SM); a
 *                           draw whose upper half ties the table entry replays its
 *                           word from the 32-bit table, so results are unchanged,
 *  MUCA_PLAN_HIST16         block histogram of 16-bit counts in shared memory, two bins
 *                           per word, added to the merged histogram every
 *                           floor(65535 / (32 L)) rows (Ising histograms too large for
 *                           32-bit counts in shared memory, e.g. 256 x 256).
 * Errors: MUCA_ERR_ARG (null context). */
#define MUCA_PLAN_LATTICE_SMEM 1
#define MUCA_PLAN_HIST_SMEM 2
#define MUCA_PLAN_TABLE_SMEM 4
#define MUCA_PLAN_PAIR_HIST 8
#define MUCA_PLAN_COMPACT 16
#define MUCA_PLAN_WARP_SPECIALIZED 32
#define MUCA_PLAN_TABLE16 64
#define MUCA_PLAN_HIST16 128
int muca_sweep_plan(const muca_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Batched form (not in the paper): many independent lattices -- uneven L, both
 * models -- advance together.  Each lattice is a full context (its own chains,
 * weights, histogram) and follows exactly the trajectory it would follow alone
 * (same random streams, same updates); only the scheduling differs:
 *  - one persistent kernel sweeps every lattice's chains: work units of 32 chains,
 *    longest first, taken from an atomic counter by a fixed grid;
 *  - one launch updates every lattice's weights (Secs. 2-3), one rebuilds all
 *    threshold tables;
 *  - the whole loop of n_iterations can be captured once as a CUDA graph and
 *    replayed with a single launch.
 * ------------------------------------------------------------------------- */
typedef struct muca_job {
    int model, L, q, p; /* as muca_init */
    uint64_t seed;
} muca_job;

typedef struct muca_batch muca_batch;

/* Create n_jobs contexts (1 <= n_jobs <= 4096) sharing cfg and the stream (NULL:
 * the batch creates its own non-blocking stream, needed for graph capture).
 * Errors: as muca_init; MUCA_ERR_ARG for an empty job list. */
int muca_batch_create(muca_batch **out, const muca_job *jobs, int n_jobs, const muca_config *cfg,
                      void *cuda_stream);
int muca_batch_destroy(muca_batch *b);

/* n_iterations weight iterations of every lattice, each of n_sweeps sweeps per
 * chain followed by the weight update (equivalent to muca_iterate +
 * muca_update_weights on every context).  use_graph != 0 replays a captured CUDA
 * graph (built once per (n_iterations, n_sweeps) and cached); returns when the work
 * is queued.  Errors: MUCA_ERR_ARG, MUCA_ERR_CUDA. */
int muca_batch_iterate(muca_batch *b, int n_iterations, int n_sweeps, int use_graph);

/* Weight iterations of every lattice until each converges (as muca_converge on each
 * context with the same arguments, and bit-identical to it): a lattice whose merged
 * histogram is covered and flat freezes in that iteration -- no further sweeps,
 * thermalisation, updates or counter advances -- while the others go on, up to
 * max_iterations.  n_iter_out[n_jobs] (host, may be NULL) receives each lattice's
 * N_iter, -1 for one that did not converge.  Afterwards every lattice runs again in
 * later calls.  Synchronises every few iterations.
 * Errors: MUCA_ERR_ARG, MUCA_ERR_CUDA. */
int muca_batch_converge(muca_batch *b, int n_sweeps, int therm_sweeps, int max_iterations, int *n_iter_out);

/* The context of job j (owned by the batch; use it for state access). */
muca_ctx *muca_batch_job(muca_batch *b, int j);

/* How the persistent sweep kernel stages job j (as configured by muca_batch_create
 * or the last muca_batch_autotune): a MUCA_PLAN_* bit mask (see muca_sweep_plan).
 * Errors: MUCA_ERR_ARG (no such job). */
int muca_batch_plan(const muca_batch *b, int j);

/* Pick the persistent grid size, the lattice staging and the number of sweep
 * launches per iteration by timing one iteration of n_sweeps on a scratch copy of
 * the batch (the batch's own chains are not touched).  Results are cached in a JSON
 * file keyed by the job list and the device name: cache_path, else the environment
 * variable MUCA_AUTOTUNE_CACHE, else no cache.  *chosen (may be NULL) receives
 * grid, staging (MUCA_STAGING_*) and launches per iteration. */
int muca_batch_autotune(muca_batch *b, int n_sweeps, const char *cache_path, int chosen[3]);

/* ---------------------------------------------------------------------------
 * Order-disorder interface tension (Sec. 5)
 * ------------------------------------------------------------------------- */

/* Reweighted energy distribution of the production sums (Eq. 2 applied to the energy
 * histogram): lnP_out[k][b] = ln n_b - ln W_b - beta_k E_b - ln sum_b'(...), FP64,
 * -inf where the production run never visited bin b; W = the production weights.
 * betas[n_beta] and lnP_out[n_beta][n_bins] may be host or device memory (caller-
 * owned); the call allocates device scratch and synchronises.
 * Errors: MUCA_ERR_ARG, MUCA_ERR_STATE (no production sums), MUCA_ERR_OOM, MUCA_ERR_CUDA. */
int muca_energy_distribution(muca_ctx *ctx, const double *betas, int n_beta, double *lnP_out);

/* sigma_od of Sec. 5 from the production sums: the inverse temperature beta_eqh at
 * which the two peaks of ln P_beta (ordered, low energy; disordered, high energy) are
 * equally high, and ln(P_max / P_min) there (mean peak height minus the minimum
 * between them); sigma_od(L) = ln_ratio / (2 L).  Peaks at a beta: split the sampled
 * bins at s (first: mid-range), highest bin on each side (first on ties), s moved to
 * the lowest bin between them until it stays (<= 64 rounds); they count only with the
 * dip strictly inside and below both.  beta_eqh: first interval of an n_grid-point
 * uniform grid on [beta_lo, beta_hi] where ln P(low peak) - ln P(high peak) turns
 * from negative to non-negative, then n_bisect bisection steps.  Outputs (host, may
 * be NULL): *beta_eqh, *ln_ratio (NaN if no such beta), peaks[3] = (low peak, high
 * peak, dip) bins (-1 if none).  Errors: as muca_energy_distribution. */
int muca_interface_tension(muca_ctx *ctx, double beta_lo, double beta_hi, int n_grid, int n_bisect,
                           double *beta_eqh, double *ln_ratio, int *peaks);

/* Checkpoint / resume: the complete state (spins, E, M, Potts counts, ln W, the
 * recursion accumulator, thresholds, counters, seed, production sums) in one file
 * (format version 3: a header, then the arrays; the per-chain arrays hold the p
 * chains only, so a file loads on a device of any SM count).  Philox is
 * counter-based, so a resumed run continues bit-identically.
 * muca_load: *out = a new context on cuda_stream (NULL: the legacy default stream),
 * owned by the caller (muca_destroy).  Errors: MUCA_ERR_ARG (null argument),
 * MUCA_ERR_IO (missing or foreign file, another format version, a truncated file,
 * spins outside the model, or E / M / counts that are not those of the spins: they
 * are recounted on the device and compared), MUCA_ERR_OOM / MUCA_ERR_CUDA (device);
 * on error *out is NULL and nothing is left allocated. */
int muca_save(muca_ctx *ctx, const char *path);
int muca_load(muca_ctx **out, const char *path, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MUCA_H */
