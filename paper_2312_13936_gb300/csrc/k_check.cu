// Disconnected communities (Appendix A.1, Algorithm 5): the number of
// communities whose vertices do not form one connected subgraph.
//
// Algorithm 5 runs a BFS inside each community. Here the connected
// components of the subgraph of intra-community edges are found for all
// communities at once by hooking and pointer jumping: every vertex starts
// as its own root; each pass hooks, for every intra-community edge whose
// ends have different roots, the larger root under the smaller one
// (atomicMin, so a parent is always smaller than its child and no cycle can
// form), then every vertex jumps to its root. When a pass hooks nothing,
// each component has one root; a community with more than one root is
// disconnected.
#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}

__global__ void k_cc_labels(int64_t n, const int32_t *C, int *bad) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (C[v] < 0 || C[v] >= n) atomicExch(bad, 1);
}

__global__ void k_cc_init(int64_t n, int32_t *parent, int32_t *roots) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        parent[v] = (int32_t)v;
        roots[v] = 0;
    }
}

// the root of x (parents only ever decrease, so the walk ends)
__device__ __forceinline__ int32_t root_of(const int32_t *parent, int32_t x) {
    int32_t p = __ldcg(&parent[x]);
    while (p != x) {
        x = p;
        p = __ldcg(&parent[x]);
    }
    return x;
}

// hook the roots of the intra-community edges (u, v), u < v, of row u taken
// from entry `from` with stride `step`
__device__ __forceinline__ bool hook_row(const int32_t *idx, const int32_t *C, int32_t *parent, int32_t u,
                                         int32_t cu, int64_t e0, int64_t from, int64_t to, int step) {
    bool hooked = false;
    for (int64_t e = e0 + from; e < e0 + to; e += step) {
        const int32_t v = idx[e];
        if (v <= u || C[v] != cu) continue;
        const int32_t ru = root_of(parent, u), rv = root_of(parent, v);
        if (ru != rv) {
            atomicMin(&parent[ru > rv ? ru : rv], ru < rv ? ru : rv);
            hooked = true;
        }
    }
    return hooked;
}

// one hooking pass (rows longer than 64 entries by the whole warp)
__global__ void k_cc_hook(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *C, int32_t *parent,
                          int *changed) {
    const int lane = threadIdx.x & 31;
    bool hooked = false;
    for (int64_t u0 = (int64_t)blockIdx.x * blockDim.x; u0 < n; u0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = u0 + threadIdx.x;
        int64_t e0 = 0, d = 0;
        int32_t cu = -1;
        if (u < n) {
            e0 = off[u];
            d = off[u + 1] - e0;
            cu = C[u];
            if (d <= 64) hooked |= hook_row(idx, C, parent, (int32_t)u, cu, e0, 0, d, 1);
        }
        unsigned longs = __ballot_sync(kFull, u < n && d > 64);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            hooked |= hook_row(idx, C, parent, (int32_t)__shfl_sync(kFull, u, src), __shfl_sync(kFull, cu, src),
                               __shfl_sync(kFull, e0, src), lane, __shfl_sync(kFull, d, src), 32);
        }
    }
    if (__any_sync(kFull, hooked) && lane == 0) atomicExch(changed, 1);
}

__global__ void k_cc_jump(int64_t n, int32_t *parent) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = root_of(parent, (int32_t)v);
}

// roots per community, then the communities with more than one
__global__ void k_cc_roots(int64_t n, const int32_t *C, const int32_t *parent, int32_t *roots) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (parent[v] == (int32_t)v) atomicAdd(&roots[C[v]], 1);
}
__global__ void k_cc_count(int64_t n, const int32_t *roots, unsigned long long *count) {
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += roots[v] > 1 ? 1 : 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

cudaError_t launch_cc_labels(int64_t n, const int32_t *C, int *bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_labels<<<grid_for(n, 256), 256, 0, s>>>(n, C, bad);
    return cudaGetLastError();
}
cudaError_t launch_cc_init(int64_t n, int32_t *parent, int32_t *roots, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_init<<<grid_for(n, 256), 256, 0, s>>>(n, parent, roots);
    return cudaGetLastError();
}
cudaError_t launch_cc_pass(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *C, int32_t *parent,
                           int *changed, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_hook<<<grid_for(n, 256), 256, 0, s>>>(n, off, idx, C, parent, changed);
    k_cc_jump<<<grid_for(n, 256), 256, 0, s>>>(n, parent);
    return cudaGetLastError();
}
cudaError_t launch_cc_count(int64_t n, const int32_t *C, const int32_t *parent, int32_t *roots,
                            unsigned long long *count, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cc_roots<<<grid_for(n, 256), 256, 0, s>>>(n, C, parent, roots);
    k_cc_count<<<grid_for(n, 256), 256, 0, s>>>(n, roots, count);
    return cudaGetLastError();
}

}  // namespace lgb
