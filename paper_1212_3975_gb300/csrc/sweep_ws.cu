// Standalone launches of the warp-specialised sweep bodies (ws_bodies.cuh).
#include "ws_bodies.cuh"

namespace muca {
namespace {
using namespace ws;

template <bool HIST, bool RECORD, bool TSMEM, int HMODE, bool LSMEM, int RU, bool T16>
__global__ void __launch_bounds__(128, T16 ? 3 : 1) ising_ws_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    ising_ws_body<HIST, RECORD, TSMEM, HMODE, LSMEM, RU, T16>(a, blockIdx.x, smem);
}

// iteration and production launches: five warps (decider, 3 producers, bookkeeper).
// One block per SM at least: without it the compiler holds the kernel to 64 registers
// and the unrolled slot decider loses 14% (32x32 iterations, 118 -> 137 attempts/ns).
template <bool HIST, bool RECORD, bool TSMEM, int HMODE, bool LSMEM>
__global__ void __launch_bounds__(160, 1) potts_ws_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    potts_ws_body<HIST, RECORD, TSMEM, HMODE, LSMEM, true>(a, blockIdx.x, smem);
}

// HMODE: histogram in global memory (0), shared per attempt (1), shared per pair of
// attempts (2)
template <int MODEL, bool HIST, bool RECORD, bool TSMEM, int HMODE, bool LSMEM, int RU = kRingU, bool T16 = false>
cudaError_t launch_ws(const SweepArgs &a, int blocks, size_t smem, cudaStream_t st)
{
    auto kern = MODEL == MUCA_ISING ? ising_ws_kernel<HIST, RECORD, TSMEM, HMODE, LSMEM, RU, T16>
                                    : potts_ws_kernel<HIST, RECORD, TSMEM, HMODE, LSMEM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (RU != kRingU) {
        // compact staging: the whole carve-out as shared memory, so two (three) blocks fit
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, (MODEL == MUCA_POTTS && (HIST || RECORD)) ? 160 : 128, smem, st>>>(a);
    return cudaGetLastError();
}

template <int MODEL, bool HIST, bool RECORD>
cudaError_t ws_staging(const SweepArgs &a, const SweepPlan &pl, int blocks, size_t smem, cudaStream_t st)
{
    // pair histogram: planned only with the table and the lattices in shared memory
    if (HIST && pl.hist_smem && pl.hist_pairs)
        return launch_ws<MODEL, HIST, RECORD, true, 2, true>(a, blocks, smem, st);
    // compact Ising staging (two blocks per SM): table and histogram in shared memory,
    // lattices in global memory, three draw-ring slots; with the table of 16-bit
    // threshold halves three blocks per SM
    if (MODEL == MUCA_ISING && pl.compact && pl.t16)
        return launch_ws<MODEL, HIST, RECORD, true, HIST ? 1 : 0, false, kCompactRing, true>(a, blocks, smem, st);
    if (MODEL == MUCA_ISING && pl.compact)
        return launch_ws<MODEL, HIST, RECORD, true, HIST ? 1 : 0, false, kCompactRing>(a, blocks, smem, st);
    // 16-bit counts (Ising histograms too large for 32-bit counts; the table and the
    // lattices are then in global memory too)
    if (MODEL == MUCA_ISING && pl.hist16) {
        if (pl.table_smem || pl.lattice_smem) return cudaErrorInvalidConfiguration;  // not planned
        return launch_ws<MODEL, HIST, RECORD, false, HIST ? 3 : 0, false>(a, blocks, smem, st);
    }
    const int key = (pl.table_smem ? 4 : 0) | ((HIST && pl.hist_smem) ? 2 : 0) | (pl.lattice_smem ? 1 : 0);
    switch (key) {
    case 0: return launch_ws<MODEL, HIST, RECORD, false, 0, false>(a, blocks, smem, st);
    case 1: return launch_ws<MODEL, HIST, RECORD, false, 0, true>(a, blocks, smem, st);
    case 2: return launch_ws<MODEL, HIST, RECORD, false, 1, false>(a, blocks, smem, st);
    case 3: return launch_ws<MODEL, HIST, RECORD, false, 1, true>(a, blocks, smem, st);
    case 4: return launch_ws<MODEL, HIST, RECORD, true, 0, false>(a, blocks, smem, st);
    case 5: return launch_ws<MODEL, HIST, RECORD, true, 0, true>(a, blocks, smem, st);
    case 6: return launch_ws<MODEL, HIST, RECORD, true, 1, false>(a, blocks, smem, st);
    default: return launch_ws<MODEL, HIST, RECORD, true, 1, true>(a, blocks, smem, st);
    }
}

}  // namespace

// shared memory of the warp-specialised kernels beyond the staging of the plan
size_t ws_extra_smem(int model, bool compact, bool hist, bool record)
{
    const int ring = compact ? kCompactRing : kRingU;
    return model == MUCA_ISING
               ? (size_t)ring * 8 * 32 * sizeof(uint4) + ((hist || record) ? (size_t)kRingS * kSnapWords * 32 * sizeof(Snap) : 0)
               : potts_ws_extra_smem(hist, record);
}

cudaError_t launch_ws_sweep(const SweepArgs &a, const SweepPlan &pl, int model, int blocks, bool hist, bool record,
                            cudaStream_t st)
{
    // what this launch uses: no histogram (and no snapshots) in thermalisation, no
    // histogram in production; the rest of the SM's shared memory stays L1 cache,
    // which holds the hot rows of a table in global memory
    const size_t smem = pl.table_bytes + (hist ? pl.hist_bytes : 0) + pl.lat_bytes +
                        ws_extra_smem(model, pl.compact, hist, record);
    if (model == MUCA_ISING) {
        if (hist && record) return ws_staging<MUCA_ISING, true, true>(a, pl, blocks, smem, st);
        if (hist) return ws_staging<MUCA_ISING, true, false>(a, pl, blocks, smem, st);
        if (record) return ws_staging<MUCA_ISING, false, true>(a, pl, blocks, smem, st);
        return ws_staging<MUCA_ISING, false, false>(a, pl, blocks, smem, st);
    }
    if (hist && record) return ws_staging<MUCA_POTTS, true, true>(a, pl, blocks, smem, st);
    if (hist) return ws_staging<MUCA_POTTS, true, false>(a, pl, blocks, smem, st);
    if (record) return ws_staging<MUCA_POTTS, false, true>(a, pl, blocks, smem, st);
    return ws_staging<MUCA_POTTS, false, false>(a, pl, blocks, smem, st);
}

}  // namespace muca
