// lat_static.cu -- lat_correlation_static: the correlation sums of a packed
// lattice the caller already holds on the device, computed without any
// device allocation.
//
// Some callers cannot allocate device memory when they need a measurement:
// a library loaded into another framework whose caching allocator owns the
// GPU's memory (a raw cudaMalloc there can fail, or take memory the framework
// has reserved), and latency-bound serving loops in which cudaMalloc/cudaFree
// would synchronise the device and stall every other stream.  The existing
// path keeps its accumulators in the workspace of a lat_create handle; this
// entry point keeps them in a fixed file-scope device array instead, so it
// needs neither a handle nor an allocation.
//
// The array holds 2 * (LAT_STATIC_RMAX + 1) int64 accumulators (64 KiB) and
// exists on every GPU that loads the library until the process exits.  Host
// code cannot pass the array's name to a kernel (on the host it is only a
// stand-in symbol); its device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device, and kept for the life of the process (a
// cudaDeviceReset, which ends the context the address belongs to, is not
// followed: call no entry point of this file after one).  Every call reuses
// the same array: the
// accumulators are cleared on the caller's stream before each use, and two
// calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/lat.h"
#include "lat_internal.cuh"

namespace {

__device__ __align__(256) long long g_static_corr[2 * (LAT_STATIC_RMAX + 1)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
long long* g_addr[kMaxDevices] = {};

// Device address of g_static_corr on the current device (looked up once).
long long* static_scratch(int* err)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *err = LAT_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_corr) != cudaSuccess || !p) {
            *err = LAT_ECUDA;
            return nullptr;
        }
        g_addr[dev] = static_cast<long long*>(p);
    }
    *err = LAT_OK;
    return g_addr[dev];
}

}  // namespace

extern "C" int lat_correlation_static(int32_t model, uint32_t L, const void* dev_spins, uint32_t rmax, int64_t* cx,
                                      int64_t* cy, void* stream)
{
    if (model != LAT_ISING && model != LAT_BLUME_CAPEL) return LAT_EINVAL;
    if (L < 64 || L % 64 != 0 || L > LAT_MAX_L || (model == LAT_BLUME_CAPEL && L > LAT_MAX_L / 2)) return LAT_EINVAL;
    if (!dev_spins || !cx || !cy || rmax > L / 2 || rmax > LAT_STATIC_RMAX) return LAT_EINVAL;
    // The correlation kernels read rows as 8-byte (Ising) or 16-byte
    // (Blume-Capel) words: refuse a pointer that would make those loads
    // misaligned, before anything is launched.
    if (reinterpret_cast<uintptr_t>(dev_spins) % 16 != 0) return LAT_EINVAL;
    int err = LAT_OK;
    long long* scratch = static_scratch(&err);
    if (!scratch) return err;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long* dcx = scratch;
    long long* dcy = scratch + (rmax + 1);
    // launch_correlation clears both accumulator ranges on `st` before its kernels run.
    cudaError_t e = latk::launch_correlation(model, dev_spins, L, L / 64, rmax, dcx, dcy, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cx, dcx, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cy, dcy, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LAT_OK : LAT_ECUDA;
}
