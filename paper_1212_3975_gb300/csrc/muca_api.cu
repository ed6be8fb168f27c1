// C ABI of libmuca: argument checks, context memory, host/device pointer handling,
// and the order of kernel launches for each call of the parallel multicanonical
// method (arXiv:1212.3975).  No arithmetic of the method lives here.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "muca_internal.cuh"

namespace muca {

namespace {
thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
}  // namespace

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA;
}

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool alloc_should_fail()
{
    static std::atomic<long> remaining{[] {
        const char *v = std::getenv("MUCA_TEST_FAIL_ALLOC");
        return v ? std::atol(v) : 0L;
    }()};
    if (remaining.load() <= 0) return false;
    return remaining.fetch_sub(1) == 1;
}

namespace {

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Per-iteration metric lines: with MUCA_METRICS_LOG=<path> every weight update appends
// one JSON line (iteration, sampled bin range, coverage, min/mean and max/mean of H,
// convergence flag, attempts/ns of the iteration's sweeps by host clock).  The update
// then synchronises once to read its statistics.
FILE *metrics_log()
{
    static FILE *f = [] {
        const char *v = std::getenv("MUCA_METRICS_LOG");
        return v && *v ? std::fopen(v, "a") : (FILE *)nullptr;
    }();
    return f;
}

template <typename T>
int dalloc(T **p, size_t count, const char *what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (alloc_should_fail()) return fail(MUCA_ERR_OOM, std::string("device allocation failed (test hook): ") + what);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MUCA_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    return MUCA_OK;
}

// Copy count elements from device src into a caller buffer (host or device).
int copy_out(muca_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    if (!dst) return MUCA_OK;
    if (is_device_ptr(dst)) {
        MUCA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        MUCA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return MUCA_OK;
}

int copy_in(muca_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    if (is_device_ptr(src)) {
        MUCA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        MUCA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return MUCA_OK;
}

void free_ctx(muca_ctx *c)
{
    if (!c) return;
    void *ptrs[] = {c->d_lat, c->d_E, c->d_M, c->d_cnt, c->d_lnw, c->d_P, c->d_lnw_prod, c->d_acc, c->d_thr,
                    c->d_H, c->d_samples, c->d_stats, c->d_series, c->d_rw, c->d_wscratch,
                    c->d_rwout, c->d_ktab, c->d_rwtile};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    delete c;
}

std::vector<uint8_t> accessible_bins(int model, int L)
{
    const int nb = n_bins_of(model, L);
    std::vector<uint8_t> acc(nb, 1);
    if (model == MUCA_ISING) {
        acc[1] = 0;
        acc[nb - 2] = 0;
    } else {
        for (int k : {1, 2, 3, 5})
            if (k < nb) acc[k] = 0;
    }
    return acc;
}

int check_ctx(const muca_ctx *ctx)
{
    if (!ctx) return fail(MUCA_ERR_ARG, "null context");
    return MUCA_OK;
}

int alloc_buffers(muca_ctx *c)
{
    const size_t nb = c->n_bins;
    int rc;
    if ((rc = dalloc(&c->d_lat, (size_t)c->lat_words * c->p_pad, "lattice"))) return rc;
    if ((rc = dalloc(&c->d_E, c->p_pad, "E"))) return rc;
    if ((rc = dalloc(&c->d_M, c->p_pad, "M"))) return rc;
    if ((rc = dalloc(&c->d_cnt, 2 * (size_t)c->p_pad, "counts"))) return rc;
    if ((rc = dalloc(&c->d_lnw, nb, "lnW"))) return rc;
    if ((rc = dalloc(&c->d_P, nb, "recursion accumulator"))) return rc;
    if ((rc = dalloc(&c->d_lnw_prod, nb, "production lnW"))) return rc;
    if ((rc = dalloc(&c->d_wscratch, nb, "update scratch"))) return rc;
    if ((rc = dalloc(&c->d_acc, nb, "accessible bins"))) return rc;
    if ((rc = dalloc(&c->d_thr, nb * c->n_de, "thresholds"))) return rc;
    if ((rc = dalloc(&c->d_ktab, nb * 9, "kernel thresholds"))) return rc;
    if ((rc = dalloc(&c->d_H, nb, "histogram"))) return rc;
    if ((rc = dalloc(&c->d_samples, 3 * nb, "production sums"))) return rc;
    if ((rc = dalloc(&c->d_stats, 1, "stats"))) return rc;
    // per-bin part of the reweighting scratch (its setup counter must start at zero)
    c->rw_bytes = rw_bin_part_bytes(nb);
    if ((rc = dalloc(reinterpret_cast<uint8_t **>(&c->d_rw), c->rw_bytes, "reweight scratch"))) return rc;
    if (cudaMemset(c->d_rw, 0, c->rw_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(MUCA_ERR_CUDA, "reweight scratch initialisation");
    }
    if (alloc_should_fail() ||
        cudaMallocHost(reinterpret_cast<void **>(&c->h_stats), sizeof(muca_iter_stats)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MUCA_ERR_OOM, "pinned allocation failed");
    }
    return MUCA_OK;
}

int ensure_series(muca_ctx *ctx, size_t records)
{
    if (ctx->series_cap >= records) return MUCA_OK;
    if (ctx->d_series) {
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->d_series);
        ctx->d_series = nullptr;
        ctx->series_cap = 0;
    }
    int rc = dalloc(&ctx->d_series, 2 * records, "production series");
    if (rc) return rc;
    ctx->series_cap = records;
    return MUCA_OK;
}

}  // namespace
}  // namespace muca

using namespace muca;

extern "C" {

const char *muca_last_error(void) { return g_last_error.c_str(); }

uint64_t muca_kernel_launches(void) { return g_launches.load(); }

int muca_init(muca_ctx **out, int model, int L, int q, int p, uint64_t seed, const muca_config *cfg,
              void *cuda_stream)
{
    MUCA_RANGE("muca_init");
    if (!out) return fail(MUCA_ERR_ARG, "out is null");
    *out = nullptr;
    if (model == MUCA_ISING) {
        if (q != 2) return fail(MUCA_ERR_ARG, "Ising requires q = 2");
        if (L < 4 || L > 1024 || (L & 1)) return fail(MUCA_ERR_ARG, "Ising requires even L in [4, 1024]");
    } else if (model == MUCA_POTTS) {
        if (q != 8) return fail(MUCA_ERR_ARG, "Potts requires q = 8");
        if (L < 3 || L > 255) return fail(MUCA_ERR_ARG, "Potts requires L in [3, 255]");
    } else {
        return fail(MUCA_ERR_ARG, "unknown model");
    }
    if (p < 1 || p > (1 << 24)) return fail(MUCA_ERR_ARG, "p must be in [1, 2^24]");
    if ((seed >> 32) >= (1ull << 30)) return fail(MUCA_ERR_ARG, "seed >> 32 must be < 2^30");
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
        cudaGetLastError();
        return fail(MUCA_ERR_CUDA, "no CUDA device available");
    }
    muca_config c0{MUCA_RECURSION_ACCUMULATED, 0, 0, MUCA_STAGING_AUTO, MUCA_ENSEMBLE_ENERGY, 0.0};
    if (cfg) {
        c0 = *cfg;
        if (c0.recursion != MUCA_RECURSION_ACCUMULATED && c0.recursion != MUCA_RECURSION_SIMPLE)
            return fail(MUCA_ERR_ARG, "unknown recursion");
        if (c0.correction_width < 0) return fail(MUCA_ERR_ARG, "correction_width < 0");
        if (c0.chains_per_block < 0 || c0.chains_per_block > 256 || (c0.chains_per_block % 32))
            return fail(MUCA_ERR_ARG, "chains_per_block must be 0 or a multiple of 32 up to 256");
        if (c0.staging < 0 || c0.staging > 2) return fail(MUCA_ERR_ARG, "unknown staging");
        if (c0.ensemble != MUCA_ENSEMBLE_ENERGY && c0.ensemble != MUCA_ENSEMBLE_MAGNETIZATION)
            return fail(MUCA_ERR_ARG, "unknown ensemble");
        if (c0.ensemble == MUCA_ENSEMBLE_MAGNETIZATION && (model != MUCA_ISING || !std::isfinite(c0.beta)))
            return fail(MUCA_ERR_ARG, "the multimagnetic ensemble needs the Ising model and a finite beta");
    }
    muca_ctx *c = new muca_ctx();
    std::memset(static_cast<void *>(c), 0, sizeof(muca_ctx));
    c->model = model;
    c->L = L;
    c->q = q;
    c->p = p;
    c->V = L * L;
    c->n_bins = n_bins_of(model, L);
    c->n_de = c0.ensemble == MUCA_ENSEMBLE_MAGNETIZATION ? 10 : n_de_of(model);
    c->seed = seed;
    c->cfg = c0;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->n_sm < 1 ||
        cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&c->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(MUCA_ERR_CUDA, "cannot query the multiprocessor count and shared memory");
    }
    c->row_words = model == MUCA_ISING ? (L + 31) / 32 : (L + 3) / 4;
    c->lat_words = L * c->row_words;
    // Fewer groups of 32 chains than SMs: the warp-specialised kernels (L % 4 == 0,
    // energy ensemble, automatic block size) spread the chains over every SM, cpg per
    // block.  A chain's attempts are sequential, so at small p the chains' own latency
    // bounds the rate, and fewer chains per SM contend less for its shared memory.
    // Only where the plan stages the lattices in shared memory: a block's chains then
    // span part of a cache line of the chain-interleaved lattice, which in global
    // memory costs more lines per warp access than it gains (8-Potts 128x128 at
    // p = 4096: 35 attempts/ns spread against 70 with 32 chains per block).
    c->cpg = 32;
    c->p_pad = (p + 31) / 32 * 32;
    if (L % 4 == 0 && c0.ensemble == MUCA_ENSEMBLE_ENERGY && c0.chains_per_block == 0 && (p + 31) / 32 < c->n_sm &&
        plan_sweeps(c).lattice_smem) {
        c->cpg = (p + c->n_sm - 1) / c->n_sm;
        c->p_pad = (p + c->cpg - 1) / c->cpg * 32;
    }
    int rc = alloc_buffers(c);
    if (rc) {
        free_ctx(c);
        return rc;
    }
    std::vector<uint8_t> acc = accessible_bins(model, L);
    if (c0.ensemble == MUCA_ENSEMBLE_MAGNETIZATION) acc.assign(c->n_bins, 1);  // every M = -V..V step 2
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->d_acc, acc.data(), acc.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_lnw, 0, sizeof(double) * c->n_bins, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_P, 0, sizeof(double) * c->n_bins, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_H, 0, sizeof(uint64_t) * c->n_bins, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_samples, 0, sizeof(uint64_t) * 3 * c->n_bins, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_cnt, 0, sizeof(uint64_t) * 2 * c->p_pad, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_E, 0, sizeof(int32_t) * c->p_pad, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_M, 0, sizeof(int32_t) * c->p_pad, c->stream)) != cudaSuccess) {
        rc = cuda_fail(e, "context initialisation");
        free_ctx(c);
        return rc;
    }
    if ((rc = launch_init_lattice(c)) || (rc = launch_thresholds(c))) {
        free_ctx(c);
        return rc;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        rc = cuda_fail(e, "muca_init");
        free_ctx(c);
        return rc;
    }
    *out = c;
    return MUCA_OK;
}

int muca_destroy(muca_ctx *ctx)
{
    if (!ctx) return MUCA_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return MUCA_OK;
}

int muca_reset(muca_ctx *ctx, uint64_t seed)
{
    MUCA_RANGE("muca_reset");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if ((seed >> 32) >= (1ull << 30)) return fail(MUCA_ERR_ARG, "seed >> 32 must be < 2^30");
    ctx->seed = seed;
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_lnw, 0, sizeof(double) * ctx->n_bins, ctx->stream));
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_P, 0, sizeof(double) * ctx->n_bins, ctx->stream));
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_H, 0, sizeof(uint64_t) * ctx->n_bins, ctx->stream));
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_samples, 0, sizeof(uint64_t) * 3 * ctx->n_bins, ctx->stream));
    ctx->iteration = 0;
    ctx->sweeps_therm = ctx->sweeps_prod = 0;
    ctx->have_hist = 0;
    ctx->samples_active = 0;
    ctx->lnw_version += 1;
    if ((rc = launch_init_lattice(ctx))) return rc;
    return launch_thresholds(ctx);
}

int muca_n_bins(const muca_ctx *ctx) { return ctx ? ctx->n_bins : fail(MUCA_ERR_ARG, "null context"); }
int muca_n_de(const muca_ctx *ctx) { return ctx ? ctx->n_de : fail(MUCA_ERR_ARG, "null context"); }
int muca_num_chains(const muca_ctx *ctx) { return ctx ? ctx->p : fail(MUCA_ERR_ARG, "null context"); }
int muca_get_iteration(const muca_ctx *ctx) { return ctx ? (int)ctx->iteration : fail(MUCA_ERR_ARG, "null context"); }
int muca_sweep_plan(const muca_ctx *ctx)
{
    if (!ctx) return fail(MUCA_ERR_ARG, "null context");
    return plan_flags(plan_sweeps(ctx));
}

int muca_iterate(muca_ctx *ctx, int n_sweeps, uint64_t *H_out)
{
    MUCA_RANGE("muca_iterate");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (n_sweeps < 1) return fail(MUCA_ERR_ARG, "n_sweeps must be >= 1");
    if (metrics_log()) {
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        ctx->it_t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        ctx->it_attempts = (double)n_sweeps * ctx->V * ctx->p;
    }
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_H, 0, sizeof(uint64_t) * ctx->n_bins, ctx->stream));
    if ((rc = launch_sweeps(ctx, kPhaseIterate, n_sweeps, 0u, ctx->iteration, true, nullptr, nullptr, false)))
        return rc;
    ctx->iteration += 1;
    ctx->have_hist = 1;
    return copy_out(ctx, H_out, ctx->d_H, sizeof(uint64_t) * ctx->n_bins);
}

int muca_update_weights(muca_ctx *ctx, muca_iter_stats *out)
{
    MUCA_RANGE("muca_update_weights");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!ctx->have_hist) return fail(MUCA_ERR_STATE, "no histogram since the last update");
    if ((rc = launch_update(ctx))) return rc;
    ctx->have_hist = 0;
    ctx->lnw_version += 1;
    FILE *log = metrics_log();
    if (out || log) {
        MUCA_CUDA_TRY(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(muca_iter_stats), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (out) *out = *ctx->h_stats;
    }
    if (log) {
        const muca_iter_stats &st = *ctx->h_stats;
        const double t1 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        const double rate = ctx->it_t0 > 0 && t1 > ctx->it_t0 ? ctx->it_attempts / ((t1 - ctx->it_t0) * 1e9) : 0.0;
        std::fprintf(log,
                     "{\"ctx\": \"%p\", \"iteration\": %u, \"lo\": %d, \"hi\": %d, \"n_sampled\": %lld, "
                     "\"covered\": %d, \"flat\": %d, \"min_over_mean\": %.6g, \"max_over_mean\": %.6g, "
                     "\"total\": %llu, \"attempts_per_ns\": %.6g}\n",
                     (void *)ctx, ctx->iteration, st.lo, st.hi, (long long)st.n_sampled, st.covered, st.flat,
                     st.min_over_mean, st.max_over_mean, (unsigned long long)st.total, rate);
        std::fflush(log);
        ctx->it_t0 = 0.0;
    }
    return MUCA_OK;
}

int muca_converge(muca_ctx *ctx, int n_sweeps, int therm_sweeps, int max_iterations, int *n_iter_out,
                  muca_iter_stats *last)
{
    MUCA_RANGE("muca_converge");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (n_sweeps < 1 || max_iterations < 1 || therm_sweeps < 0)
        return fail(MUCA_ERR_ARG, "need n_sweeps >= 1, therm_sweeps >= 0 and max_iterations >= 1");
    muca_iter_stats st{};
    int conv = -1;
    for (int it = 1; it <= max_iterations; ++it) {
        if ((rc = muca_iterate(ctx, n_sweeps, nullptr))) return rc;
        if ((rc = muca_update_weights(ctx, &st))) return rc;
        if (st.flat) {
            conv = it;
            break;
        }
        // intermediate thermalisation with the new weights before the next iteration
        if (it < max_iterations && (rc = muca_thermalize(ctx, therm_sweeps))) return rc;
    }
    if (n_iter_out) *n_iter_out = conv;
    if (last) *last = st;
    return MUCA_OK;
}

int muca_thermalize(muca_ctx *ctx, int n_sweeps)
{
    MUCA_RANGE("muca_thermalize");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (n_sweeps < 0) return fail(MUCA_ERR_ARG, "n_sweeps must be >= 0");
    if (n_sweeps == 0) return MUCA_OK;
    if ((rc = launch_sweeps(ctx, kPhaseThermalize, n_sweeps, ctx->sweeps_therm, 0u, false, nullptr, nullptr, false)))
        return rc;
    ctx->sweeps_therm += (uint32_t)n_sweeps;
    return MUCA_OK;
}

int muca_reset_samples(muca_ctx *ctx)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    MUCA_CUDA_TRY(cudaMemsetAsync(ctx->d_samples, 0, sizeof(uint64_t) * 3 * ctx->n_bins, ctx->stream));
    ctx->samples_active = 0;
    return MUCA_OK;
}

int muca_set_samples(muca_ctx *ctx, const uint64_t *n, const uint64_t *sum_abs_m, const uint64_t *sum_m2)
{
    MUCA_RANGE("muca_set_samples");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (ctx->cfg.ensemble != MUCA_ENSEMBLE_ENERGY)
        return fail(MUCA_ERR_STATE, "no energy production sums in the multimagnetic ensemble");
    if (!n || !sum_abs_m || !sum_m2) return fail(MUCA_ERR_ARG, "null buffer");
    const size_t bytes = sizeof(uint64_t) * ctx->n_bins;
    if ((rc = copy_in(ctx, ctx->d_samples, n, bytes))) return rc;
    if ((rc = copy_in(ctx, ctx->d_samples + ctx->n_bins, sum_abs_m, bytes))) return rc;
    if ((rc = copy_in(ctx, ctx->d_samples + 2 * (size_t)ctx->n_bins, sum_m2, bytes))) return rc;
    MUCA_CUDA_TRY(cudaMemcpyAsync(ctx->d_lnw_prod, ctx->d_lnw, sizeof(double) * ctx->n_bins,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->samples_active = 1;
    ctx->samples_lnw_version = ctx->lnw_version;
    return MUCA_OK;
}

int muca_produce(muca_ctx *ctx, int n_sweeps, int32_t *E_out, int32_t *M_out)
{
    MUCA_RANGE("muca_produce");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (n_sweeps < 1) return fail(MUCA_ERR_ARG, "n_sweeps must be >= 1");
    if (ctx->samples_active && ctx->samples_lnw_version != ctx->lnw_version)
        return fail(MUCA_ERR_STATE, "weights changed since the production records started; reset samples");
    if (!ctx->samples_active) {
        MUCA_CUDA_TRY(cudaMemcpyAsync(ctx->d_lnw_prod, ctx->d_lnw, sizeof(double) * ctx->n_bins,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
        ctx->samples_active = 1;
        ctx->samples_lnw_version = ctx->lnw_version;
    }
    const bool dE = is_device_ptr(E_out), dM = is_device_ptr(M_out);
    const bool host_out = (E_out && !dE) || (M_out && !dM);
    if (!host_out) {
        rc = launch_sweeps(ctx, kPhaseProduce, n_sweeps, ctx->sweeps_prod, 0u, false, E_out, M_out, true);
        if (rc) return rc;
        ctx->sweeps_prod += (uint32_t)n_sweeps;
        return MUCA_OK;
    }
    // host buffers: produce in chunks through the device series buffer
    const size_t chunk_sweeps = std::max<size_t>(1, std::min<size_t>(n_sweeps, (size_t)(64u << 20) / ctx->p));
    if ((rc = ensure_series(ctx, chunk_sweeps * ctx->p))) return rc;
    for (int done = 0; done < n_sweeps;) {
        const int n = (int)std::min<size_t>(chunk_sweeps, (size_t)(n_sweeps - done));
        int32_t *sE = ctx->d_series, *sM = ctx->d_series + ctx->series_cap;
        rc = launch_sweeps(ctx, kPhaseProduce, n, ctx->sweeps_prod, 0u, false, sE, sM, true);
        if (rc) return rc;
        ctx->sweeps_prod += (uint32_t)n;
        const size_t bytes = sizeof(int32_t) * (size_t)n * ctx->p;
        const size_t off = (size_t)done * ctx->p;
        if (E_out) {
            if ((rc = copy_out(ctx, E_out + off, sE, bytes))) return rc;
        }
        if (M_out) {
            if ((rc = copy_out(ctx, M_out + off, sM, bytes))) return rc;
        }
        done += n;
    }
    return MUCA_OK;
}

int muca_reweight(muca_ctx *ctx, const double *betas, int n_beta, int precision, double *e, double *C,
                  double *absm, double *chi)
{
    MUCA_RANGE("muca_reweight");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (ctx->cfg.ensemble != MUCA_ENSEMBLE_ENERGY)
        return fail(MUCA_ERR_STATE, "no energy production sums in the multimagnetic ensemble");
    if (!betas || n_beta < 1) return fail(MUCA_ERR_ARG, "need at least one beta");
    if (precision != MUCA_FP64 && precision != MUCA_FP32 && precision != MUCA_BF16)
        return fail(MUCA_ERR_ARG, "unknown precision");
    if (!ctx->samples_active) return fail(MUCA_ERR_STATE, "no production records");
    // context scratch: the four output arrays and (for host input) the betas
    const size_t need = (size_t)5 * n_beta;
    if (ctx->rwout_cap < need) {
        MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (ctx->d_rwout) cudaFree(ctx->d_rwout);
        ctx->d_rwout = nullptr;
        ctx->rwout_cap = 0;
        if ((rc = dalloc(&ctx->d_rwout, need, "reweight outputs"))) return rc;
        ctx->rwout_cap = need;
    }
    double *d_tmp = ctx->d_rwout;
    const double *d_betas = betas;
    if (!is_device_ptr(betas)) {
        MUCA_CUDA_TRY(cudaMemcpyAsync(d_tmp + 4 * (size_t)n_beta, betas, sizeof(double) * n_beta,
                                      cudaMemcpyHostToDevice, ctx->stream));
        d_betas = d_tmp + 4 * (size_t)n_beta;
    }
    // device outputs are written in place; host (or null) outputs go through the scratch
    double *outs[4] = {e, C, absm, chi};
    double *dev[4];
    bool staged[4];
    for (int k = 0; k < 4; ++k) {
        staged[k] = !(outs[k] && is_device_ptr(outs[k]));
        dev[k] = staged[k] ? d_tmp + (size_t)k * n_beta : outs[k];
    }
    if ((rc = launch_reweight(ctx, d_betas, n_beta, precision, dev))) return rc;
    for (int k = 0; k < 4; ++k)
        if (staged[k] && (rc = copy_out(ctx, outs[k], dev[k], sizeof(double) * n_beta))) return rc;
    return MUCA_OK;
}

int muca_get_lnw(muca_ctx *ctx, double *lnw)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!lnw) return fail(MUCA_ERR_ARG, "null buffer");
    return copy_out(ctx, lnw, ctx->d_lnw, sizeof(double) * ctx->n_bins);
}

int muca_set_lnw(muca_ctx *ctx, const double *lnw)
{
    MUCA_RANGE("muca_set_lnw");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!lnw) return fail(MUCA_ERR_ARG, "null buffer");
    if ((rc = copy_in(ctx, ctx->d_lnw, lnw, sizeof(double) * ctx->n_bins))) return rc;
    ctx->lnw_version += 1;
    return launch_thresholds(ctx);
}

int muca_get_thresholds(muca_ctx *ctx, uint32_t *thr)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!thr) return fail(MUCA_ERR_ARG, "null buffer");
    return copy_out(ctx, thr, ctx->d_thr, sizeof(uint32_t) * ctx->n_bins * ctx->n_de);
}

int muca_set_thresholds(muca_ctx *ctx, const uint32_t *thr)
{
    MUCA_RANGE("muca_set_thresholds");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!thr) return fail(MUCA_ERR_ARG, "null buffer");
    ctx->ktab_dirty = 1;
    return copy_in(ctx, ctx->d_thr, thr, sizeof(uint32_t) * ctx->n_bins * ctx->n_de);
}

int muca_get_spins(muca_ctx *ctx, int8_t *spins)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!spins) return fail(MUCA_ERR_ARG, "null buffer");
    const size_t bytes = (size_t)ctx->V * ctx->p;
    if (is_device_ptr(spins)) return launch_unpack_spins(ctx, spins);
    int8_t *tmp = nullptr;
    if ((rc = dalloc(&tmp, bytes, "spin export"))) return rc;
    rc = launch_unpack_spins(ctx, tmp);
    if (rc == MUCA_OK) rc = copy_out(ctx, spins, tmp, bytes);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    return rc;
}

int muca_get_energies(muca_ctx *ctx, int64_t *E, int64_t *M)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    std::vector<int32_t> e(ctx->p), m(ctx->p);
    MUCA_CUDA_TRY(cudaMemcpyAsync(e.data(), ctx->d_E, sizeof(int32_t) * ctx->p, cudaMemcpyDeviceToHost, ctx->stream));
    MUCA_CUDA_TRY(cudaMemcpyAsync(m.data(), ctx->d_M, sizeof(int32_t) * ctx->p, cudaMemcpyDeviceToHost, ctx->stream));
    MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < ctx->p; ++c) {
        if (E) E[c] = e[c];
        if (M) M[c] = m[c];
    }
    return MUCA_OK;
}

int muca_get_histogram(muca_ctx *ctx, uint64_t *H)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!H) return fail(MUCA_ERR_ARG, "null buffer");
    return copy_out(ctx, H, ctx->d_H, sizeof(uint64_t) * ctx->n_bins);
}

int muca_get_samples(muca_ctx *ctx, uint64_t *n, uint64_t *sum_abs_m, uint64_t *sum_m2)
{
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    const size_t bytes = sizeof(uint64_t) * ctx->n_bins;
    if ((rc = copy_out(ctx, n, ctx->d_samples, bytes))) return rc;
    if ((rc = copy_out(ctx, sum_abs_m, ctx->d_samples + ctx->n_bins, bytes))) return rc;
    return copy_out(ctx, sum_m2, ctx->d_samples + 2 * (size_t)ctx->n_bins, bytes);
}

// ---------------------------------------------------------------------------
// checkpoint: fixed header followed by the device arrays in a fixed order
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, model, L, q, p, pad0;
    uint64_t seed;
    muca_config cfg;
    uint32_t iteration, sweeps_therm, sweeps_prod;
    int32_t have_hist, samples_active, pad1;
    uint64_t lnw_version, samples_lnw_version;
};

// A device array in the file.  Per-chain arrays (rows x p_pad on the device: the
// chain-interleaved layout, whose padding depends on the device's SM count) are
// written as rows x p, so that a checkpoint loads on any device.
struct Blob {
    void *dev;
    size_t elem, rows;  // element bytes; rows of p_pad (per chain) or one row of `n`
    size_t n;           // elements of a non-chain array (0: per chain)
    size_t file_bytes(const muca_ctx *c) const { return elem * (n ? n : rows * (size_t)c->p); }
};

std::vector<Blob> blobs(muca_ctx *c)
{
    const size_t nb = c->n_bins;
    return {{c->d_lat, 4, (size_t)c->lat_words, 0},
            {c->d_E, 4, 1, 0},
            {c->d_M, 4, 1, 0},
            {c->d_cnt, 8, 2, 0},
            {c->d_lnw, 8, 1, nb},
            {c->d_P, 8, 1, nb},
            {c->d_lnw_prod, 8, 1, nb},
            {c->d_thr, 4, 1, nb * c->n_de},
            {c->d_H, 8, 1, nb},
            {c->d_samples, 8, 1, 3 * nb}};
}

constexpr int32_t kCkptVersion = 3;

// Spins of a checkpoint's lattice (rows x p words) are values of the model: Potts
// bytes below q, and the bits / bytes past site L - 1 of a row's last word zero.
bool lattice_valid(const muca_ctx *c, const uint32_t *lat)
{
    const int per = c->model == MUCA_ISING ? 32 : 4;
    const int last = c->L - per * (c->row_words - 1);  // sites in a row's last word
    for (int k = 0; k < c->lat_words; ++k) {
        const bool lastw = (k % c->row_words) == c->row_words - 1;
        const uint32_t *row = lat + (size_t)k * c->p;
        for (int i = 0; i < c->p; ++i) {
            const uint32_t w = row[i];
            if (c->model == MUCA_ISING) {
                if (lastw && last < 32 && (w >> last) != 0u) return false;
            } else {
                for (int b = 0; b < 4; ++b) {
                    const uint32_t v = (w >> (8 * b)) & 0xFFu;
                    if ((lastw && b >= last) ? v != 0u : v >= (uint32_t)c->q) return false;
                }
            }
        }
    }
    return true;
}
}  // namespace

int muca_save(muca_ctx *ctx, const char *path)
{
    MUCA_RANGE("muca_save");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!path) return fail(MUCA_ERR_ARG, "null path");
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "MUCACKP1", 8);
    h.version = kCkptVersion;
    h.model = ctx->model;
    h.L = ctx->L;
    h.q = ctx->q;
    h.p = ctx->p;
    h.seed = ctx->seed;
    h.cfg = ctx->cfg;
    h.iteration = ctx->iteration;
    h.sweeps_therm = ctx->sweeps_therm;
    h.sweeps_prod = ctx->sweeps_prod;
    h.have_hist = ctx->have_hist;
    h.samples_active = ctx->samples_active;
    h.lnw_version = ctx->lnw_version;
    h.samples_lnw_version = ctx->samples_lnw_version;
    MUCA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MUCA_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    std::vector<uint8_t> buf;
    for (const Blob &b : blobs(ctx)) {
        if (!ok) break;
        const size_t dev_bytes = b.elem * (b.n ? b.n : b.rows * (size_t)ctx->p_pad);
        buf.resize(dev_bytes);
        if (cudaMemcpy(buf.data(), b.dev, dev_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(cudaGetLastError(), "checkpoint read-back");
        }
        if (b.n) {
            ok = std::fwrite(buf.data(), 1, dev_bytes, f) == dev_bytes;
        } else {
            // the p chains of every row, without the padding columns
            const size_t row = b.elem * (size_t)ctx->p;
            for (size_t r = 0; r < b.rows && ok; ++r)
                ok = std::fwrite(buf.data() + r * b.elem * (size_t)ctx->p_pad, 1, row, f) == row;
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MUCA_OK : fail(MUCA_ERR_IO, std::string("write failed: ") + path);
}

int muca_load(muca_ctx **out, const char *path, void *cuda_stream)
{
    MUCA_RANGE("muca_load");
    if (!out || !path) return fail(MUCA_ERR_ARG, "null argument");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MUCA_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "MUCACKP1", 8) != 0) {
        std::fclose(f);
        return fail(MUCA_ERR_IO, "not a checkpoint file (bad header)");
    }
    if (h.version != kCkptVersion) {
        std::fclose(f);
        return fail(MUCA_ERR_IO, "checkpoint format version " + std::to_string(h.version) + " (this library reads " +
                                     std::to_string(kCkptVersion) + ")");
    }
    muca_ctx *ctx = nullptr;
    int rc = muca_init(&ctx, h.model, h.L, h.q, h.p, h.seed, &h.cfg, cuda_stream);
    if (rc) {
        std::fclose(f);
        return rc;
    }
    auto bail = [&](int code, const std::string &msg) {
        std::fclose(f);
        muca_destroy(ctx);
        return code == MUCA_ERR_CUDA ? cuda_fail(cudaGetLastError(), msg.c_str()) : fail(code, msg);
    };
    std::vector<uint8_t> buf, dev;
    std::vector<uint8_t> chain_state[4];  // lattice, E, M, counts as read (rows x p)
    int bi = 0;
    for (const Blob &b : blobs(ctx)) {
        const size_t fb = b.file_bytes(ctx);
        buf.resize(fb);
        if (std::fread(buf.data(), 1, fb, f) != fb) return bail(MUCA_ERR_IO, "checkpoint truncated");
        if (b.n) {
            if (cudaMemcpy(b.dev, buf.data(), fb, cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(MUCA_ERR_CUDA, "checkpoint upload");
        } else {
            if (bi == 0 && !lattice_valid(ctx, reinterpret_cast<const uint32_t *>(buf.data())))
                return bail(MUCA_ERR_IO, "checkpoint holds spins outside the model");
            // scatter the p chains of every row into the padded layout (padding zero)
            const size_t row = b.elem * (size_t)ctx->p, drow = b.elem * (size_t)ctx->p_pad;
            dev.assign(drow * b.rows, 0);
            for (size_t r = 0; r < b.rows; ++r) std::memcpy(dev.data() + r * drow, buf.data() + r * row, row);
            if (cudaMemcpy(b.dev, dev.data(), dev.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(MUCA_ERR_CUDA, "checkpoint upload");
            chain_state[bi] = buf;
        }
        ++bi;
    }
    std::fclose(f);
    // E, M and the state counts must be those of the spins: recount them on the device
    // and compare (a chain whose E does not match its spins would walk its bin off the
    // weight table).  The uploads ran on the legacy stream, the recount runs on the
    // context's stream: wait for both.
    if (cudaDeviceSynchronize() != cudaSuccess || (rc = launch_recount(ctx)) ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        if (!rc) rc = cuda_fail(cudaGetLastError(), "checkpoint check");
        muca_destroy(ctx);
        return rc;
    }
    const int32_t *E_f = reinterpret_cast<const int32_t *>(chain_state[1].data());
    const int32_t *M_f = reinterpret_cast<const int32_t *>(chain_state[2].data());
    const uint64_t *C_f = reinterpret_cast<const uint64_t *>(chain_state[3].data());
    std::vector<int32_t> E(ctx->p), M(ctx->p);
    std::vector<uint64_t> C(2 * (size_t)ctx->p);
    bool same = cudaMemcpy(E.data(), ctx->d_E, 4 * (size_t)ctx->p, cudaMemcpyDeviceToHost) == cudaSuccess &&
                cudaMemcpy(M.data(), ctx->d_M, 4 * (size_t)ctx->p, cudaMemcpyDeviceToHost) == cudaSuccess &&
                cudaMemcpy(C.data(), ctx->d_cnt, 8 * (size_t)ctx->p, cudaMemcpyDeviceToHost) == cudaSuccess &&
                cudaMemcpy(C.data() + ctx->p, ctx->d_cnt + ctx->p_pad, 8 * (size_t)ctx->p, cudaMemcpyDeviceToHost) ==
                    cudaSuccess;
    if (!same) {
        rc = cuda_fail(cudaGetLastError(), "checkpoint check");
        muca_destroy(ctx);
        return rc;
    }
    same = std::memcmp(E.data(), E_f, 4 * (size_t)ctx->p) == 0 && std::memcmp(M.data(), M_f, 4 * (size_t)ctx->p) == 0 &&
           (ctx->model != MUCA_POTTS || std::memcmp(C.data(), C_f, 16 * (size_t)ctx->p) == 0);
    if (!same) {
        muca_destroy(ctx);
        return fail(MUCA_ERR_IO, "checkpoint energies do not match its spins");
    }
    ctx->ktab_dirty = 1;
    ctx->iteration = h.iteration;
    ctx->sweeps_therm = h.sweeps_therm;
    ctx->sweeps_prod = h.sweeps_prod;
    ctx->have_hist = h.have_hist;
    ctx->samples_active = h.samples_active;
    ctx->lnw_version = h.lnw_version;
    ctx->samples_lnw_version = h.samples_lnw_version;
    *out = ctx;
    return MUCA_OK;
}

}  // extern "C"
