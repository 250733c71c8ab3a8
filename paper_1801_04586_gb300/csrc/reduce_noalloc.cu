// reduce_noalloc.cu -- clbm_reduce_pair_noalloc: the FP64 pair reduction of
// clbm_reduce_pair for callers that cannot allocate device memory.
//
// clbm_reduce_pair keeps its per-block partial sums in scratch that
// clbm_create allocated. Some callers can make neither that allocation nor a
// context: cudaMalloc and cudaFree can synchronise the device and can fail
// with out-of-memory, which code such as a monitoring hook inside a running
// simulation, or a component living beside a framework's caching allocator
// that has reserved nearly all device memory, must not risk. This variant
// needs no context and allocates nothing: its partial sums live in a
// file-scope __device__ array of fixed size, loaded with the library.
//
// Limits and sharing:
//   - one partial per 8192 input elements, at most kMaxPartials partials, so
//     n <= 8192 * 16384 = 134,217,728 elements (larger n: CLBM_ERR_ARG);
//   - the array (3 * 16384 doubles = 384 KiB) is held on every GPU that loads
//     the library until the process exits;
//   - every call on a device shares it: each call's blocks overwrite exactly
//     the slots its final pass reads, so nothing needs clearing between
//     calls, but calls that overlap on the GPU (different streams, or another
//     host thread) race on it and must be serialised by the caller;
//   - the array's device address is looked up once per device and cached for
//     the process: it belongs to the device's primary context, so a
//     cudaDeviceReset leaves it stale (callers must not call after a reset);
//   - under lazy module loading the first call on a device may load the
//     module (allocating the array and the code): it is the set-up call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/clbm.h"
#include "kernels.cuh"

namespace {

constexpr int64_t kChunk = 8192;          // input elements per partial (256 threads x 32)
constexpr int kMaxPartials = 16384;       // partials the static array holds
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_pair_partials[3 * kMaxPartials];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};  // device address of g_pair_partials, per device

// Set-up, once per device, with that device current: the host-side name of a
// __device__ array is not a device address, so ask the runtime for it.
cudaError_t partials_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pair_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int clbm_reduce_pair_noalloc(const float *a, const float *b, int64_t n, double *out, void *stream) {
    if (!out || n < 0 || (!a && n > 0))
        return clbm::set_error(CLBM_ERR_ARG, "clbm_reduce_pair_noalloc: bad argument");
    if (n > kChunk * kMaxPartials)
        return clbm::set_error(CLBM_ERR_ARG,
                               "clbm_reduce_pair_noalloc: n exceeds the 134217728-element limit of its static scratch");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return clbm::set_error(CLBM_ERR_CUDA, "clbm_reduce_pair_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices)
        return clbm::set_error(CLBM_ERR_ARG, "clbm_reduce_pair_noalloc: device index beyond 63");
    double *partials = nullptr;
    if ((e = partials_address(dev, &partials)) != cudaSuccess)
        return clbm::set_error(CLBM_ERR_CUDA, "clbm_reduce_pair_noalloc: cudaGetSymbolAddress failed");
    const int nblocks = n == 0 ? 1 : (int)((n + kChunk - 1) / kChunk);
    e = clbm::launch_reduce_pair(a, b, n, partials, nblocks, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return clbm::set_error(CLBM_ERR_CUDA, "clbm_reduce_pair_noalloc: launch failed");
    return CLBM_OK;
}
