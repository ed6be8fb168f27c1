// Batched form: many independent lattices (uneven L, both models) in one persistent
// sweep kernel per weight iteration, a batched weight update, and CUDA-graph capture
// of the whole iteration loop; plus a small timing-based autotuner.
//
// Every lattice is an ordinary context and follows exactly the trajectory it would
// follow alone: the work units run the same warp-specialised bodies with the same
// arguments (seed, chain ids, iteration and sweep counters); only which SM runs a
// unit, and when, differs.  The work queue is a monotone atomic counter, so no block
// ever waits on another.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "ws_bodies.cuh"

namespace muca {
namespace {
using namespace ws;

struct BatchUnit {
    int job, cblk;
};

__device__ __forceinline__ SweepArgs batch_args(const BatchJob &j, int n_sweeps, uint32_t sweep0, bool therm)
{
    SweepArgs a;
    a.lat = j.lat;
    a.E = j.E;
    a.M = j.M;
    a.cnt = j.cnt;
    a.thr = j.thr;
    a.ktab = j.ktab;
    a.H = j.H;
    a.E_rec = nullptr;
    a.M_rec = nullptr;
    a.samples = nullptr;
    a.L = j.L;
    a.q = j.q;
    a.p = j.p;
    a.p_pad = j.p_pad;
    a.cpg = 32;
    a.row_words = j.row_words;
    a.lat_words = j.lat_words;
    a.n_bins = j.n_bins;
    a.n_sweeps = n_sweeps;
    // weight iterations: counter words (sweep in the iteration, iteration, phase 1);
    // thermalisation: (running sweep count, 0, phase 2), as the standalone calls
    a.sweep0 = therm ? *j.therm + sweep0 : sweep0;
    a.iteration = therm ? 0u : *j.iteration;
    a.ctr3 = therm ? j.ctr3_therm : j.ctr3_iter;
    a.key0 = j.key0;
    a.rec_stride = j.p;
    return a;
}

// H: histogram mode (0 global, 1 shared per attempt, 2 shared per pair of attempts;
// the Potts body without a bookkeeper warp counts per attempt)
template <int MODEL, bool HIST, bool T, int H, bool Lt>
__device__ __forceinline__ void body(const SweepArgs &a, int cblk, uint32_t *smem)
{
    if (MODEL == MUCA_ISING)
        ising_ws_body<HIST, false, T, HIST ? H : 0, Lt>(a, cblk, smem);
    else
        potts_ws_body<HIST, false, T, (HIST && H) ? 1 : 0, Lt>(a, cblk, smem);
}

template <int MODEL, bool HIST>
__device__ __forceinline__ void run_unit(const SweepArgs &a, int flags, int cblk, uint32_t *smem)
{
    if constexpr (MODEL == MUCA_ISING) {
        if (flags & 8) {  // histogram of attempt pairs (table and lattices staged)
            body<MODEL, HIST, true, 2, true>(a, cblk, smem);
            return;
        }
    }
    switch (flags & 7) {
    case 0: body<MODEL, HIST, false, 0, false>(a, cblk, smem); break;
    case 1: body<MODEL, HIST, false, 0, true>(a, cblk, smem); break;
    case 2: body<MODEL, HIST, false, 1, false>(a, cblk, smem); break;
    case 3: body<MODEL, HIST, false, 1, true>(a, cblk, smem); break;
    case 4: body<MODEL, HIST, true, 0, false>(a, cblk, smem); break;
    case 5: body<MODEL, HIST, true, 0, true>(a, cblk, smem); break;
    case 6: body<MODEL, HIST, true, 1, false>(a, cblk, smem); break;
    default: body<MODEL, HIST, true, 1, true>(a, cblk, smem); break;
    }
}

// Persistent sweep kernel of one weight iteration (or part of it); THERM: sweeps of
// an intermediate thermalisation (no histogram).
template <bool THERM>
__global__ void __launch_bounds__(128, 1) batch_sweep_kernel(const BatchJob *jobs, const BatchUnit *units, int n_units,
                                                          unsigned *queue, int n_sweeps, uint32_t sweep0)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_unit, s_model, s_flags, s_cblk;
    // The unit's arguments live in shared memory and the bodies read them where they
    // need them (the standalone kernels read theirs from the parameter bank); built in
    // registers they raised the register pressure of the bodies into spills.
    __shared__ SweepArgs s_args;
    for (;;) {
        __syncthreads();  // every warp is done with the previous unit's arguments
        if (threadIdx.x == 0) {
            const int u = (int)atomicAdd(queue, 1u);
            s_unit = u;
            if (u < n_units) {
                const BatchUnit un = units[u];
                const BatchJob &j = jobs[un.job];
                s_model = *j.active ? j.model : -1;  // -1: converged, frozen
                s_flags = j.flags;
                s_cblk = un.cblk;
                s_args = batch_args(j, n_sweeps, sweep0, THERM);
            }
        }
        __syncthreads();
        if (s_unit >= n_units) break;
        const int model = s_model;
        if (model == MUCA_ISING)
            run_unit<MUCA_ISING, !THERM>(s_args, s_flags, s_cblk, smem);
        else if (model == MUCA_POTTS)
            run_unit<MUCA_POTTS, !THERM>(s_args, s_flags, s_cblk, smem);
    }
}

// zero every lattice's histogram and the work counter
__global__ void batch_prepare_kernel(const BatchJob *jobs, unsigned *queue)
{
    const BatchJob &j = jobs[blockIdx.y];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *queue = 0u;
    if (!*j.active) return;  // a frozen lattice keeps its last histogram
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < j.n_bins; t += gridDim.x * blockDim.x) j.H[t] = 0ull;
}

// kernel tables from the thresholds of every lattice; then advance the iteration
// counters (counter word 2 of the random streams)
__global__ void batch_ktab_kernel(const BatchJob *jobs)
{
    const BatchJob &j = jobs[blockIdx.y];
    if (!*j.active) return;
    const int width = j.model == MUCA_ISING ? 5 : 9;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < j.n_bins * width; t += gridDim.x * blockDim.x) {
        const int b = t / width, k = t % width;
        uint32_t v;
        if (j.model == MUCA_ISING) {
            v = k == 2 ? kAlways : j.thr[b * 4 + (k >= 3 ? 4 - k : 3 - k)];
        } else {
            const int dE = k - 4;
            v = dE == 0 ? kAlways : j.thr[b * 8 + (dE < 0 ? dE + 4 : dE + 3)];
        }
        j.ktab[t] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *j.iteration += 1u;
}

// Convergence test of Sec. 3 after the update of iteration `it` (1-based): a lattice
// whose merged histogram was covered and flat is frozen and records `it`.
__global__ void batch_converge_kernel(const BatchJob *jobs, int n_jobs, int it)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_jobs) return;
    const BatchJob &j = jobs[i];
    if (*j.active && j.stats->flat) {
        *j.active = 0;
        *j.conv = it;
    }
}

// after a thermalisation pass: advance the sweep counters of the running lattices
__global__ void batch_therm_advance_kernel(const BatchJob *jobs, int n_jobs, int n_sweeps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_jobs && *jobs[i].active) *jobs[i].therm += (uint32_t)n_sweeps;
}

__global__ void batch_fill_kernel(int *x, int n, int v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

struct TuneChoice {
    int grid, staging, split;
};

}  // namespace
}  // namespace muca

using namespace muca;

struct muca_batch {
    int n_jobs = 0;
    std::vector<muca_ctx *> ctx;
    std::vector<muca_job> jobs;
    muca_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<BatchJob> h_jobs;
    std::vector<int> plan_flags;  // MUCA_PLAN_* of every job
    BatchJob *d_jobs = nullptr;
    BatchUnit *d_units = nullptr;
    int n_units = 0;
    unsigned *d_queue = nullptr;
    uint32_t *d_iter = nullptr;
    int *d_active = nullptr;  // [n_jobs]: 1 running, 0 frozen (converged)
    int *d_conv = nullptr;    // [n_jobs]: iteration of convergence, -1 before
    uint32_t *d_therm = nullptr;  // [n_jobs]: thermalisation sweep counters
    size_t smem = 0;
    int grid = 0, staging = MUCA_STAGING_AUTO, split = 1;
    int max_bins = 0, max_thr = 0, max_ktab = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int g_iters = -1, g_sweeps = -1;
};

namespace {

void drop_graph(muca_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->g_iters = b->g_sweeps = -1;
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// (Re)build the job table for the batch's staging choice and upload it.
int configure(muca_batch *b)
{
    b->h_jobs.assign(b->n_jobs, BatchJob{});
    b->plan_flags.assign(b->n_jobs, 0);
    b->smem = 0;
    b->max_bins = b->max_thr = b->max_ktab = 0;
    std::vector<std::pair<long long, BatchUnit>> units;
    // Every block gets the shared memory of the largest job, so the histogram of
    // attempt pairs is used only where it does not raise that maximum (more shared
    // memory leaves less L1 to the jobs that read their tables from global memory).
    size_t smem_plain = 0;
    for (int i = 0; i < b->n_jobs; ++i) {
        b->ctx[i]->cfg.staging = b->staging;
        const SweepPlan pl = plan_sweeps(b->ctx[i], false, false);
        smem_plain = std::max(smem_plain, pl.smem_bytes + ws_extra_smem(b->ctx[i]->model));
    }
    for (int i = 0; i < b->n_jobs; ++i) {
        muca_ctx *c = b->ctx[i];
        c->cfg.staging = b->staging;
        if (c->cfg.ensemble != MUCA_ENSEMBLE_ENERGY)
            return fail(MUCA_ERR_ARG, "batched lattices need the energy ensemble (job " + std::to_string(i) + ")");
        // pairs of attempts for Ising (its body has a bookkeeper warp here) within the
        // shared memory of the largest job; the batched Potts body counts per attempt
        SweepPlan pl = plan_sweeps(c, c->model == MUCA_ISING, false);
        if (pl.hist_pairs && pl.smem_bytes + ws_extra_smem(c->model) > smem_plain) pl = plan_sweeps(c, false, false);
        if (!pl.warp_specialized)
            return fail(MUCA_ERR_ARG, "batched lattices need L % 4 == 0 (job " + std::to_string(i) + ")");
        BatchJob &j = b->h_jobs[i];
        j.model = c->model;
        j.L = c->L;
        j.q = c->q;
        j.p = c->p;
        j.p_pad = c->p_pad;
        j.row_words = c->row_words;
        j.lat_words = c->lat_words;
        j.n_bins = c->n_bins;
        j.n_de = c->n_de;
        j.V = c->V;
        j.accumulated = c->cfg.recursion == MUCA_RECURSION_ACCUMULATED;
        j.width = c->cfg.correction_width > 0 ? c->cfg.correction_width : c->L;
        j.key0 = (uint32_t)c->seed;
        j.ctr3_iter = ((uint32_t)(c->seed >> 32) << 2) | kPhaseIterate;
        j.lat = c->d_lat;
        j.E = c->d_E;
        j.M = c->d_M;
        j.cnt = c->d_cnt;
        j.lnw = c->d_lnw;
        j.P = c->d_P;
        j.wscratch = c->d_wscratch;
        j.acc = c->d_acc;
        j.thr = c->d_thr;
        j.ktab = c->d_ktab;
        j.H = c->d_H;
        j.stats = c->d_stats;
        j.iteration = b->d_iter + i;
        j.active = b->d_active + i;
        j.conv = b->d_conv + i;
        j.ctr3_therm = ((uint32_t)(c->seed >> 32) << 2) | kPhaseThermalize;
        j.therm = b->d_therm + i;
        j.flags = (pl.hist_pairs ? 8 : 0) | (pl.table_smem ? 4 : 0) | (pl.hist_smem ? 2 : 0) | (pl.lattice_smem ? 1 : 0);
        b->plan_flags[i] = plan_flags(pl);
        b->smem = std::max(b->smem, pl.smem_bytes + ws_extra_smem(c->model));
        b->max_bins = std::max(b->max_bins, c->n_bins);
        b->max_thr = std::max(b->max_thr, c->n_bins * c->n_de);
        b->max_ktab = std::max(b->max_ktab, c->n_bins * (c->model == MUCA_ISING ? 5 : 9));
        // cost of a unit ~ sites per sweep x time per site (Potts sites cost about 3 Ising sites)
        const long long cost = (long long)c->V * (c->model == MUCA_ISING ? 1 : 3);
        for (int cb = 0; cb < c->p_pad / 32; ++cb) units.push_back({cost, BatchUnit{i, cb}});
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const std::pair<long long, BatchUnit> &x, const std::pair<long long, BatchUnit> &y) {
                         return x.first > y.first;
                     });
    std::vector<BatchUnit> hu;
    for (auto &u : units) hu.push_back(u.second);
    b->n_units = (int)hu.size();
    if (!b->d_units) {
        if (cudaMalloc(reinterpret_cast<void **>(&b->d_units), sizeof(BatchUnit) * hu.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(MUCA_ERR_OOM, "batch unit table");
        }
    }
    MUCA_CUDA_TRY(cudaMemcpyAsync(b->d_units, hu.data(), sizeof(BatchUnit) * hu.size(), cudaMemcpyHostToDevice,
                                  b->stream));
    MUCA_CUDA_TRY(cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), sizeof(BatchJob) * b->n_jobs, cudaMemcpyHostToDevice,
                                  b->stream));
    MUCA_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (b->smem > 227 * 1024) return fail(MUCA_ERR_ARG, "batched staging exceeds shared memory");
    MUCA_CUDA_TRY(
        cudaFuncSetAttribute(batch_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    MUCA_CUDA_TRY(
        cudaFuncSetAttribute(batch_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    if (b->grid <= 0) b->grid = std::min(b->n_units, sm_count());
    drop_graph(b);
    return MUCA_OK;
}

// Queue one weight iteration of every lattice on the batch stream.
int enqueue_iteration(muca_batch *b, int n_sweeps)
{
    const int split = std::max(1, std::min(b->split, n_sweeps));
    for (int s = 0; s < split; ++s) {
        const int s0 = (int)((long long)n_sweeps * s / split), s1 = (int)((long long)n_sweeps * (s + 1) / split);
        if (s == 0) {
            dim3 g((b->max_bins + 255) / 256, b->n_jobs);
            batch_prepare_kernel<<<g, 256, 0, b->stream>>>(b->d_jobs, b->d_queue);
            MUCA_CUDA_TRY(cudaGetLastError());
            note_launches(1);
        } else {
            MUCA_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), b->stream));
        }
        batch_sweep_kernel<false><<<b->grid, 128, b->smem, b->stream>>>(b->d_jobs, b->d_units, b->n_units, b->d_queue,
                                                                         s1 - s0, (uint32_t)s0);
        MUCA_CUDA_TRY(cudaGetLastError());
        note_launches(1);
    }
    cudaError_t e = launch_batch_update(b->d_jobs, b->n_jobs, b->max_thr, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched weight update");
    dim3 g((b->max_ktab + 255) / 256, b->n_jobs);
    batch_ktab_kernel<<<g, 256, 0, b->stream>>>(b->d_jobs);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}

void free_batch(muca_batch *b)
{
    if (!b) return;
    drop_graph(b);
    for (muca_ctx *c : b->ctx)
        if (c) muca_destroy(c);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_units) cudaFree(b->d_units);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->d_iter) cudaFree(b->d_iter);
    if (b->d_active) cudaFree(b->d_active);
    if (b->d_conv) cudaFree(b->d_conv);
    if (b->d_therm) cudaFree(b->d_therm);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

std::string device_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    return pr.name;
}

std::string tune_key(const muca_batch *b, int n_sweeps)
{
    std::ostringstream k;
    k << device_name() << "|sweeps=" << n_sweeps;
    for (const muca_job &j : b->jobs) k << "|" << j.model << ":" << j.L << ":" << j.p;
    return k.str();
}

// cache file: {"<key>": [grid, staging, split], ...}
std::map<std::string, TuneChoice> read_cache(const std::string &path)
{
    std::map<std::string, TuneChoice> m;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return m;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    std::fclose(f);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
        const size_t end = text.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = text.substr(pos + 1, end - pos - 1);
        const size_t lb = text.find('[', end), rb = text.find(']', end);
        if (lb == std::string::npos || rb == std::string::npos) break;
        TuneChoice c{0, 0, 1};
        if (std::sscanf(text.c_str() + lb + 1, "%d , %d , %d", &c.grid, &c.staging, &c.split) == 3) m[key] = c;
        pos = rb + 1;
    }
    return m;
}

void write_cache(const std::string &path, const std::map<std::string, TuneChoice> &m)
{
    const std::string tmp = path + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : m) {
        std::fprintf(f, "  \"%s\": [%d, %d, %d]%s\n", kv.first.c_str(), kv.second.grid, kv.second.staging,
                     kv.second.split, ++i < m.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

extern "C" {

int muca_batch_create(muca_batch **out, const muca_job *jobs, int n_jobs, const muca_config *cfg, void *cuda_stream)
{
    MUCA_RANGE("muca_batch_create");
    if (!out) return fail(MUCA_ERR_ARG, "out is null");
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > 4096) return fail(MUCA_ERR_ARG, "need 1..4096 jobs");
    muca_batch *b = new muca_batch();
    b->n_jobs = n_jobs;
    b->jobs.assign(jobs, jobs + n_jobs);
    if (cfg) b->cfg = *cfg;
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return fail(MUCA_ERR_CUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    b->staging = cfg ? cfg->staging : MUCA_STAGING_AUTO;
    b->ctx.assign(n_jobs, nullptr);
    // the persistent kernel's work units are groups of 32 chains
    muca_config jc{MUCA_RECURSION_ACCUMULATED, 0, 0, MUCA_STAGING_AUTO, MUCA_ENSEMBLE_ENERGY, 0.0};
    if (cfg) jc = *cfg;
    if (jc.chains_per_block == 0) jc.chains_per_block = 32;
    b->cfg = jc;
    for (int i = 0; i < n_jobs; ++i) {
        int rc = muca_init(&b->ctx[i], jobs[i].model, jobs[i].L, jobs[i].q, jobs[i].p, jobs[i].seed, &jc, b->stream);
        if (rc) {
            free_batch(b);
            return rc;
        }
    }
    if (alloc_should_fail() ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_jobs), sizeof(BatchJob) * n_jobs) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_queue), sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_iter), sizeof(uint32_t) * n_jobs) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_active), sizeof(int) * n_jobs) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_conv), sizeof(int) * n_jobs) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_therm), sizeof(uint32_t) * n_jobs) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return fail(MUCA_ERR_OOM, "batch tables");
    }
    batch_fill_kernel<<<(n_jobs + 255) / 256, 256, 0, b->stream>>>(b->d_active, n_jobs, 1);
    batch_fill_kernel<<<(n_jobs + 255) / 256, 256, 0, b->stream>>>(b->d_conv, n_jobs, -1);
    if (cudaGetLastError() != cudaSuccess) {
        free_batch(b);
        return fail(MUCA_ERR_CUDA, "batch flags");
    }
    note_launches(2);
    int rc = configure(b);
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return MUCA_OK;
}

int muca_batch_destroy(muca_batch *b)
{
    if (!b) return MUCA_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return MUCA_OK;
}

muca_ctx *muca_batch_job(muca_batch *b, int j)
{
    if (!b || j < 0 || j >= b->n_jobs) return nullptr;
    return b->ctx[j];
}

int muca_batch_plan(const muca_batch *b, int j)
{
    if (!b || j < 0 || j >= b->n_jobs) return fail(MUCA_ERR_ARG, "no such job");
    return b->plan_flags[j];
}

namespace {
// Before a call that queues iterations: sweep launches per iteration, pending tables
// of individual contexts, and the iteration counters of the random streams.
int begin_iterations(muca_batch *b, int n_sweeps)
{
    // uint32 block histograms: 32 chains x sweeps x sites per launch below 2^31
    long long vmax = 0;
    for (muca_ctx *c : b->ctx) vmax = std::max<long long>(vmax, c->V);
    while (32LL * ((n_sweeps + b->split - 1) / b->split) * vmax >= (1LL << 31)) {
        b->split *= 2;
        drop_graph(b);
    }
    // pending threshold tables of individual contexts, iteration and thermalisation
    // counters
    std::vector<uint32_t> it(b->n_jobs), th(b->n_jobs);
    for (int i = 0; i < b->n_jobs; ++i) {
        muca_ctx *c = b->ctx[i];
        if (c->ktab_dirty) {
            int rc = launch_ktab(c);
            if (rc) return rc;
        }
        it[i] = c->iteration;
        th[i] = c->sweeps_therm;
    }
    MUCA_CUDA_TRY(cudaMemcpyAsync(b->d_iter, it.data(), sizeof(uint32_t) * b->n_jobs, cudaMemcpyHostToDevice,
                                  b->stream));
    MUCA_CUDA_TRY(cudaMemcpyAsync(b->d_therm, th.data(), sizeof(uint32_t) * b->n_jobs, cudaMemcpyHostToDevice,
                                  b->stream));
    MUCA_CUDA_TRY(cudaStreamSynchronize(b->stream));
    return MUCA_OK;
}
}  // namespace

int muca_batch_iterate(muca_batch *b, int n_iterations, int n_sweeps, int use_graph)
{
    MUCA_RANGE("muca_batch_iterate");
    if (!b) return fail(MUCA_ERR_ARG, "null batch");
    if (n_iterations < 1 || n_sweeps < 1) return fail(MUCA_ERR_ARG, "need n_iterations >= 1 and n_sweeps >= 1");
    int rc0 = begin_iterations(b, n_sweeps);
    if (rc0) return rc0;
    if (use_graph) {
        if (!b->gexec || b->g_iters != n_iterations || b->g_sweeps != n_sweeps) {
            drop_graph(b);
            MUCA_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            const unsigned long long before = muca_kernel_launches();
            for (int i = 0; i < n_iterations; ++i) {
                int rc = enqueue_iteration(b, n_sweeps);
                if (rc) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(b->stream, &g);
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
            }
            // capture records kernels without running them
            note_launches((uint64_t)0 - (muca_kernel_launches() - before));
            MUCA_CUDA_TRY(cudaStreamEndCapture(b->stream, &b->graph));
            MUCA_CUDA_TRY(cudaGraphInstantiate(&b->gexec, b->graph, 0));
            b->g_iters = n_iterations;
            b->g_sweeps = n_sweeps;
        }
        MUCA_CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
        note_launches((uint64_t)n_iterations * (4 + b->split));
    } else {
        for (int i = 0; i < n_iterations; ++i) {
            int rc = enqueue_iteration(b, n_sweeps);
            if (rc) return rc;
        }
    }
    for (muca_ctx *c : b->ctx) {
        c->iteration += (uint32_t)n_iterations;
        c->have_hist = 0;
        c->lnw_version += (uint64_t)n_iterations;
        c->ktab_dirty = 0;
    }
    return MUCA_OK;
}

namespace {
// Thermalisation sweeps of every running lattice (no histogram), in launches that
// keep the uint32 block histogram bound of the iteration launches.
int enqueue_thermalization(muca_batch *b, int n_sweeps)
{
    const int split = std::max(1, std::min(b->split, n_sweeps));
    for (int s = 0; s < split; ++s) {
        const int s0 = (int)((long long)n_sweeps * s / split), s1 = (int)((long long)n_sweeps * (s + 1) / split);
        MUCA_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), b->stream));
        batch_sweep_kernel<true><<<b->grid, 128, b->smem, b->stream>>>(b->d_jobs, b->d_units, b->n_units, b->d_queue,
                                                                        s1 - s0, (uint32_t)s0);
        MUCA_CUDA_TRY(cudaGetLastError());
        note_launches(1);
    }
    batch_therm_advance_kernel<<<(b->n_jobs + 255) / 256, 256, 0, b->stream>>>(b->d_jobs, b->n_jobs, n_sweeps);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    return MUCA_OK;
}
}  // namespace

int muca_batch_converge(muca_batch *b, int n_sweeps, int therm_sweeps, int max_iterations, int *n_iter_out)
{
    MUCA_RANGE("muca_batch_converge");
    if (!b) return fail(MUCA_ERR_ARG, "null batch");
    if (n_sweeps < 1 || max_iterations < 1 || therm_sweeps < 0)
        return fail(MUCA_ERR_ARG, "need n_sweeps >= 1, therm_sweeps >= 0 and max_iterations >= 1");
    int rc = begin_iterations(b, n_sweeps);
    if (rc) return rc;
    const int nb = (b->n_jobs + 255) / 256;
    batch_fill_kernel<<<nb, 256, 0, b->stream>>>(b->d_active, b->n_jobs, 1);
    batch_fill_kernel<<<nb, 256, 0, b->stream>>>(b->d_conv, b->n_jobs, -1);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(2);
    std::vector<int> conv(b->n_jobs, -1);
    // Iterations are queued in chunks and the host looks at the flags between chunks; a
    // lattice freezes on the device in the iteration it converges, so the chunk size
    // changes nothing but how soon the call returns.
    int done = 0, chunk = 1;
    while (done < max_iterations) {
        const int n = std::min(chunk, max_iterations - done);
        for (int i = 0; i < n; ++i) {
            if ((rc = enqueue_iteration(b, n_sweeps))) return rc;
            batch_converge_kernel<<<nb, 256, 0, b->stream>>>(b->d_jobs, b->n_jobs, done + i + 1);
            MUCA_CUDA_TRY(cudaGetLastError());
            note_launches(1);
            // intermediate thermalisation before the next iteration of the running lattices
            if (therm_sweeps > 0 && done + i + 1 < max_iterations && (rc = enqueue_thermalization(b, therm_sweeps)))
                return rc;
        }
        done += n;
        MUCA_CUDA_TRY(cudaMemcpyAsync(conv.data(), b->d_conv, sizeof(int) * b->n_jobs, cudaMemcpyDeviceToHost,
                                      b->stream));
        MUCA_CUDA_TRY(cudaStreamSynchronize(b->stream));
        if (std::all_of(conv.begin(), conv.end(), [](int v) { return v >= 0; })) break;
        chunk = std::min(chunk * 2, 8);
    }
    // host-side state of every context: the iterations it actually ran
    for (int i = 0; i < b->n_jobs; ++i) {
        muca_ctx *c = b->ctx[i];
        const int ran = conv[i] >= 0 ? conv[i] : done;
        c->iteration += (uint32_t)ran;
        c->sweeps_therm += (uint32_t)therm_sweeps * (uint32_t)(conv[i] >= 0 ? ran - 1 : std::min(done, max_iterations - 1));
        c->have_hist = 0;
        c->lnw_version += (uint64_t)ran;
        c->ktab_dirty = 0;
        if (n_iter_out) n_iter_out[i] = conv[i];
    }
    batch_fill_kernel<<<nb, 256, 0, b->stream>>>(b->d_active, b->n_jobs, 1);
    MUCA_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    MUCA_CUDA_TRY(cudaStreamSynchronize(b->stream));
    return MUCA_OK;
}

int muca_batch_autotune(muca_batch *b, int n_sweeps, const char *cache_path, int chosen[3])
{
    MUCA_RANGE("muca_batch_autotune");
    if (!b) return fail(MUCA_ERR_ARG, "null batch");
    if (n_sweeps < 1) return fail(MUCA_ERR_ARG, "n_sweeps must be >= 1");
    std::string path = cache_path ? cache_path : "";
    if (path.empty() && std::getenv("MUCA_AUTOTUNE_CACHE")) path = std::getenv("MUCA_AUTOTUNE_CACHE");
    const std::string key = tune_key(b, n_sweeps);
    std::map<std::string, TuneChoice> cache;
    if (!path.empty()) cache = read_cache(path);
    TuneChoice best{0, 0, 1};
    auto hit = cache.find(key);
    if (hit != cache.end()) {
        best = hit->second;
    } else {
        // trials on a scratch copy of the batch (other seeds), so that the batch's own
        // chains and weights are untouched
        std::vector<muca_job> jobs = b->jobs;
        for (muca_job &j : jobs) j.seed ^= 0x5A5A5A5Aull;
        muca_batch *t = nullptr;
        int rc = muca_batch_create(&t, jobs.data(), (int)jobs.size(), &b->cfg, nullptr);
        if (rc) return rc;
        const int sms = sm_count();
        std::vector<int> grids = {std::min(t->n_units, sms), std::min(t->n_units, 2 * sms)};
        grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int staging : {MUCA_STAGING_AUTO, MUCA_STAGING_GLOBAL}) {
            for (int grid : grids) {
                for (int split : {1, 2}) {
                    t->staging = staging;
                    t->grid = grid;
                    t->split = split;
                    if ((rc = configure(t))) break;
                    if ((rc = muca_batch_iterate(t, 1, n_sweeps, 0))) break;  // warm-up
                    cudaEventRecord(e0, t->stream);
                    if ((rc = muca_batch_iterate(t, 1, n_sweeps, 0))) break;
                    cudaEventRecord(e1, t->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = TuneChoice{grid, staging, split};
                    }
                }
                if (rc) break;
            }
            if (rc) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        muca_batch_destroy(t);
        if (rc) return rc;
        if (!path.empty()) {
            cache[key] = best;
            write_cache(path, cache);
        }
    }
    b->grid = best.grid;
    b->staging = best.staging;
    b->split = best.split;
    int rc = configure(b);
    if (rc) return rc;
    if (chosen) {
        chosen[0] = best.grid;
        chosen[1] = best.staging;
        chosen[2] = best.split;
    }
    return MUCA_OK;
}

}  // extern "C"
