// leiden_modularity_noalloc: modularity (Eq. 1) of a membership without any
// device allocation.
//
// leiden_modularity takes its scratch (the total weight Sigma_c of every
// community, plus four running sums) from the stream-ordered allocator. Some
// callers cannot allocate device memory at the moment they need the score:
// a host framework may own the whole device memory through its own pool and
// forbid allocation calls from plug-in code, a process may run at its memory
// cap, or a latency-critical path may not accept an allocator call. This
// entry point serves them: the scratch is a file-scope device array of fixed
// size that every GPU loading the library holds until the process exits.
//
// Limits and rules:
//   - n <= kNoAllocMaxVertices (1,048,576); larger n is rejected with
//     LEIDEN_ERR_INVALID before any device work.
//   - The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current and caches it; make
//     that first call before any stream capture on the device. A reset of
//     the device (cudaDeviceReset) reloads the module at another address and
//     leaves the cached one stale: after a reset this entry point must not be
//     called again in the same process.
//   - All calls on a device share the one array. Calls whose work overlaps
//     on the GPU (different streams, or threads racing on one stream) race
//     on it and give wrong results; serialise them.
//   - The array keeps the previous call's contents, so every call clears
//     the part it uses before accumulating into it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "engine.h"
#include "kernels.h"

namespace {

constexpr int64_t kNoAllocMaxVertices = 1 << 20;
constexpr int kMaxDevices = 256;

// Sigma_c of every community label, then 4 sums (intra weight, 2m, sum of
// Sigma_c^2, labels out of range)
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxVertices + 4];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" leiden_status leiden_modularity_noalloc(int64_t n, const int64_t *offsets, const int32_t *indices,
                                                   const float *weights, const int32_t *membership, double gamma,
                                                   void *stream, double *q_out) {
    if (n < 0 || !q_out || (n > 0 && (!offsets || !indices || !membership))) {
        lgb::set_last_error("invalid arguments to leiden_modularity_noalloc");
        return LEIDEN_ERR_INVALID;
    }
    if (n > kNoAllocMaxVertices) {
        lgb::set_last_error("leiden_modularity_noalloc: n = " + std::to_string(n) + " exceeds its scratch limit of " +
                            std::to_string(kNoAllocMaxVertices) + " vertices");
        return LEIDEN_ERR_INVALID;
    }
    if (n == 0) {
        *q_out = 0.0;
        return LEIDEN_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        lgb::set_last_error("leiden_modularity_noalloc: no usable current device");
        return LEIDEN_ERR_CUDA;
    }
    double *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // the host-side symbol is only a stand-in: ask the runtime for the
            // array's address on the current device
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                lgb::set_last_error(std::string("leiden_modularity_noalloc: cudaGetSymbolAddress failed: ") +
                                    cudaGetErrorString(e));
                return LEIDEN_ERR_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *sigtot = base;
    double *sums = base + kNoAllocMaxVertices;
    double h[4] = {0, 0, 0, 0};
    if ((e = cudaMemsetAsync(sigtot, 0, sizeof(double) * n, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sums, 0, sizeof(double) * 4, s)) != cudaSuccess ||
        (e = lgb::launch_modularity_parts(n, offsets, indices, weights, membership, sigtot, sums, s)) != cudaSuccess ||
        (e = lgb::launch_sum_squares(sigtot, n, &sums[2], s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        lgb::set_last_error(std::string("leiden_modularity_noalloc: ") + cudaGetErrorString(e));
        return LEIDEN_ERR_CUDA;
    }
    if (h[3] != 0.0) {
        lgb::set_last_error("leiden_modularity_noalloc: membership labels must lie in [0, n)");
        return LEIDEN_ERR_INVALID;
    }
    *q_out = h[1] > 0 ? h[0] / h[1] - gamma * h[2] / (h[1] * h[1]) : 0.0;
    return LEIDEN_OK;
}
