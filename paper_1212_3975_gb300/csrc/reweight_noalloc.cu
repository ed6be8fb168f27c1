// Reweighting entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they want observables:
// an application whose framework allocator already owns the free device memory
// (a new cudaMalloc would fail or fragment it), or a latency-critical loop where
// cudaMalloc/cudaFree would stall it (cudaFree synchronises the whole device).
// muca_reweight_noalloc serves them: the caller passes its own device buffers for
// every input and output, and the per-bin scratch of the reweighting kernels lives
// in one fixed file-scope device array instead of memory owned by a context.
//
// The array is part of this library's device image: once the image is loaded on a
// GPU (with CUDA's default lazy loading, at the first call on that device, which
// therefore needs kNoallocScratchBytes = 1,806,336 bytes of free device memory once;
// make that first call at start-up, before any stream capture), the GPU holds it until
// the process exits.  Host code may not use the array's name as a device address;
// every call looks the address up with cudaGetSymbolAddress for the current device, so
// a device reset or a newly created primary context (which may place the array
// elsewhere) never leaves a stale address behind.
#include <string>

#include "muca_internal.cuh"

namespace {

using muca::kNoallocMaxBins;

// Scratch of the tiled reweighting kernels for at most kNoallocMaxBins bins and
// kNoallocBetasPerPass betas per pass: per-bin arrays (ln n - ln W, E, mean |M|, mean
// M^2, within-bin variance of |M|, a float copy of the first, the sampled range of
// each block of bins, the setup kernel's completion counter) and per-pass tile
// parameters, shifts, completion counters and partial sums.  Every entry a call reads
// is written or cleared by the same call first, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[muca::kNoallocScratchBytes / sizeof(double)];
static_assert(muca::kNoallocScratchBytes % sizeof(double) == 0, "scratch size");
static_assert(muca::kNoallocScratchBytes == 1806336, "the documented size of the scratch");

// device (or managed) memory that the current device `dev` can use
bool device_pointer_on(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int muca_reweight_noalloc(int model, int L, int q, const uint64_t *samples, const double *lnw,
                                     const double *betas, int n_beta, int precision, double *out,
                                     void *cuda_stream)
{
    using muca::fail;
    if (model == MUCA_ISING) {
        if (q != 2 || L < 4 || (L & 1)) return fail(MUCA_ERR_ARG, "Ising requires q = 2 and even L >= 4");
    } else if (model == MUCA_POTTS) {
        if (q != 8 || L < 3) return fail(MUCA_ERR_ARG, "Potts requires q = 8 and L >= 3");
    } else {
        return fail(MUCA_ERR_ARG, "unknown model");
    }
    const long long nb = model == MUCA_ISING ? (long long)L * L + 1 : 2LL * L * L + 1;
    if (nb > kNoallocMaxBins)
        return fail(MUCA_ERR_ARG, "muca_reweight_noalloc supports at most " + std::to_string(kNoallocMaxBins) +
                                      " energy bins (Ising L <= 128, 8-Potts L <= 90); this lattice has " +
                                      std::to_string(nb));
    if (n_beta < 1) return fail(MUCA_ERR_ARG, "need at least one beta");
    if (precision != MUCA_FP64 && precision != MUCA_FP32)
        return fail(MUCA_ERR_ARG, "muca_reweight_noalloc supports MUCA_FP64 and MUCA_FP32");
    if (!samples || !lnw || !betas || !out) return fail(MUCA_ERR_ARG, "null buffer");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return muca::cuda_fail(e, "cudaGetDevice");
    if (!device_pointer_on(samples, dev) || !device_pointer_on(lnw, dev) || !device_pointer_on(betas, dev) ||
        !device_pointer_on(out, dev))
        return fail(MUCA_ERR_ARG,
                    "muca_reweight_noalloc needs device buffers of the current device for all inputs and outputs");
    // the array's address on the current device and context (the first call on a
    // device loads the library's device image there)
    double *scratch = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&scratch), g_noalloc_scratch);
    if (e != cudaSuccess) return muca::cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return muca::cuda_fail(e, "cudaDeviceGetAttribute");
    e = muca::launch_reweight_buffers(scratch, samples, lnw, model, L, q, betas, n_beta, precision, out, n_sm,
                                      static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return muca::cuda_fail(e, "muca_reweight_noalloc launch");
    return MUCA_OK;
}
