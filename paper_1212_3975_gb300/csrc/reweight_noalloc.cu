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
// The array is part of this library's device image, so every GPU that loads the
// library holds it (kNoallocMaxBins * 5 doubles, 655,400 bytes) until the process
// exits.  Host code may not use the array's name as a device address; the address
// is looked up once per device with cudaGetSymbolAddress.
#include <atomic>
#include <string>

#include "muca_internal.cuh"

namespace muca {
cudaError_t launch_reweight_buffers(double *scratch, const uint64_t *samples, const double *lnw, int model, int L,
                                    int q, const double *d_betas, int n_beta, int precision, double *d_out,
                                    cudaStream_t st);
}

namespace {

constexpr int kNoallocMaxBins = 16385;  // Ising L <= 128, 8-Potts L <= 90
constexpr int kMaxDevices = 64;

// Per-bin scratch: 5 arrays of kNoallocMaxBins doubles (ln n - ln W, E, mean |M|,
// mean M^2, within-bin variance of |M|).  Every entry a call reads is written by the
// same call first, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[5 * kNoallocMaxBins];

std::atomic<double *> g_scratch_addr[kMaxDevices];

bool device_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
    if (!device_pointer(samples) || !device_pointer(lnw) || !device_pointer(betas) || !device_pointer(out))
        return fail(MUCA_ERR_ARG, "muca_reweight_noalloc needs device buffers for all inputs and outputs");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return muca::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(MUCA_ERR_ARG, "device index beyond the supported range");
    double *scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        // one-time set-up on this device (the device must be current)
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&scratch), g_noalloc_scratch);
        if (e != cudaSuccess) return muca::cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_addr[dev].store(scratch, std::memory_order_release);
    }
    e = muca::launch_reweight_buffers(scratch, samples, lnw, model, L, q, betas, n_beta, precision, out,
                                      static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return muca::cuda_fail(e, "muca_reweight_noalloc launch");
    return MUCA_OK;
}
