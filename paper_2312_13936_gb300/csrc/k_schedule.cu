// Sweep schedule of a pass (reading S0). Vertex priorities come from
// SplitMix64; u precedes v when prio(u) > prio(v) (ties: smaller id).
// layer(v) = 1 + max layer of v's preceding neighbours (0 if none): the
// rounds of Jones & Plassmann's parallel colouring. They are found level by
// level: cnt[v] counts v's preceding neighbours; a vertex enters layer r+1
// when the last of them is released in round r. Rounds stop at layer L-2;
// every vertex not placed by then takes step L-1 + ((prio >> 32) mod B).
// In a batch of graphs a vertex's priority is drawn at its index inside its
// own graph (and, when graphs are at different passes, from the state of its
// own graph's pass), so every graph gets the schedule it would get alone.
#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

// first vertex of v's graph (0 for a single graph)
__device__ __forceinline__ int64_t graph_base(const int32_t *gid, const int64_t *vseg, int64_t v) {
    return gid ? __ldg(&vseg[__ldg(&gid[v])]) : 0;
}
// generator state of v's graph: the pass state, advanced by the graph's own
// pass index when graphs are at different passes
__device__ __forceinline__ uint64_t graph_state(uint64_t state, const int32_t *gid, const int32_t *gpass, int64_t v) {
    return gpass ? state + (uint64_t)__ldg(&gpass[__ldg(&gid[v])]) : state;
}

// preceding neighbours of v among row entries [from, to) taken with stride step
__device__ __forceinline__ int32_t count_preceding(const int32_t *idx, int64_t e0, int32_t from, int32_t to,
                                                   int32_t step, uint64_t state, int64_t base, int64_t v,
                                                   uint64_t pv) {
    int32_t c = 0;
    for (int32_t e = from; e < to; e += step) {
        const int32_t u = idx[e0 + e];
        if (u != (int32_t)v && precedes(splitmix64_at(state, (uint64_t)(u - base)), u, pv, (int32_t)v)) c++;
    }
    return c;
}

// cnt[v] = number of v's preceding neighbours; layer[v] = 0 if none.
// settled[0] counts the layer-0 vertices. LONG: rows longer than kLongRow
// are counted by the whole warp (hubs of heavy-tailed graphs); otherwise one
// thread per vertex.
template <bool LONG>
__global__ void __launch_bounds__(256) k_sched_init(int64_t n, const int64_t *off, const int32_t *deg,
                                                    const int32_t *idx, uint64_t state0, const int32_t *gid,
                                                    const int64_t *vseg, const int32_t *gpass, int32_t *cnt,
                                                    int32_t *layer, int32_t *settled) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const int32_t dv = v < n ? deg[v] : 0;
        int64_t base = 0;
        uint64_t state = 0, pv = 0;
        int64_t e0 = 0;
        if (v < n) {
            base = graph_base(gid, vseg, v);
            state = graph_state(state0, gid, gpass, v);
            pv = splitmix64_at(state, (uint64_t)(v - base));
            e0 = off[v];
        }
        int32_t c = (v < n && (!LONG || dv <= kLongRow)) ? count_preceding(idx, e0, 0, dv, 1, state, base, v, pv) : 0;
        unsigned longs = LONG ? __ballot_sync(kFull, v < n && dv > kLongRow) : 0u;
        while (longs) {  // long rows: the warp counts together
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int32_t cl = warp_sum(count_preceding(
                idx, __shfl_sync(kFull, e0, src), lane, __shfl_sync(kFull, dv, src), 32,
                __shfl_sync(kFull, state, src), __shfl_sync(kFull, base, src), __shfl_sync(kFull, v, src),
                __shfl_sync(kFull, pv, src)));
            if (lane == src) c = cl;
        }
        if (v < n) {
            cnt[v] = c;
            layer[v] = c == 0 ? 0 : -1;
            if (c == 0) atomicAdd(&s_cnt, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&settled[0], s_cnt);
}

// release the succeeding neighbours of v (layer r) among row entries
// [from, to) taken with stride step; returns how many joined layer r+1
__device__ __forceinline__ int release_succeeding(const int32_t *idx, int64_t e0, int32_t from, int32_t to,
                                                  int32_t step, uint64_t state, int64_t base, int64_t v,
                                                  uint64_t pv, int32_t r, int32_t *cnt, int32_t *layer) {
    int placed = 0;
    for (int32_t e = from; e < to; e += step) {
        const int32_t u = idx[e0 + e];
        if (u == (int32_t)v || !precedes(pv, (int32_t)v, splitmix64_at(state, (uint64_t)(u - base)), u)) continue;
        if (atomicSub(&cnt[u], 1) == 1) {
            layer[u] = r + 1;
            placed++;
        }
    }
    return placed;
}

// round r: every vertex of layer r releases its succeeding neighbours; a
// neighbour whose last preceding neighbour is released joins layer r+1. The
// round scans the layer array, so layer-r vertices are visited in id order;
// it returns at once when layer r is empty (settled[r] == 0).
template <bool LONG>
__global__ void __launch_bounds__(256) k_sched_round(int64_t n, const int64_t *off, const int32_t *deg,
                                                     const int32_t *idx, uint64_t state0, const int32_t *gid,
                                                     const int64_t *vseg, const int32_t *gpass, int32_t r,
                                                     int32_t *cnt, int32_t *layer, int32_t *settled) {
    if (__ldcg(&settled[r]) == 0) return;
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int placed = 0;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const bool act = v < n && __ldcg(&layer[v]) == r;
        const int32_t dv = act ? deg[v] : 0;
        int64_t base = 0, e0 = 0;
        uint64_t state = 0, pv = 0;
        if (act) {
            base = graph_base(gid, vseg, v);
            state = graph_state(state0, gid, gpass, v);
            pv = splitmix64_at(state, (uint64_t)(v - base));
            e0 = off[v];
            if (!LONG || dv <= kLongRow)
                placed += release_succeeding(idx, e0, 0, dv, 1, state, base, v, pv, r, cnt, layer);
        }
        unsigned longs = LONG ? __ballot_sync(kFull, act && dv > kLongRow) : 0u;
        while (longs) {  // long rows: the warp releases together
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            placed += release_succeeding(idx, __shfl_sync(kFull, e0, src), lane, __shfl_sync(kFull, dv, src), 32,
                                         __shfl_sync(kFull, state, src), __shfl_sync(kFull, base, src),
                                         __shfl_sync(kFull, v, src), __shfl_sync(kFull, pv, src), r, cnt, layer);
        }
    }
    if (placed) atomicAdd(&s_cnt, placed);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&settled[r + 1], s_cnt);
}

__global__ void k_sched_finish(int64_t n, uint64_t state0, int32_t L, int32_t B, const int32_t *gid,
                               const int64_t *vseg, const int32_t *gpass, const int32_t *layer, int32_t *step) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = layer[v];
        if (l >= 0 && l < L - 1) {
            step[v] = l;
        } else {
            const uint64_t p = splitmix64_at(graph_state(state0, gid, gpass, v), (uint64_t)(v - graph_base(gid, vseg, v)));
            step[v] = L - 1 + (int32_t)((p >> 32) % (uint64_t)B);
        }
    }
}

__global__ void k_step_bin_keys(const int32_t *step, const int32_t *deg, int64_t n, int32_t nsteps, bool bin_major,
                                int32_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int b = degree_bin(deg[v]);
        // vertices without edges go to a trailing bucket (never swept)
        key[v] = b == 0 ? nsteps * kNumBins : (bin_major ? b * nsteps + step[v] : step[v] * kNumBins + b);
    }
}

inline int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

cudaError_t launch_schedule(const GraphView &g, uint64_t state, int32_t L, int32_t B, const SchedWork &w,
                            int32_t *step, cudaStream_t s, const int32_t *gid, const int64_t *vseg,
                            const int32_t *gpass, bool long_rows) {
    if (g.n <= 0) return cudaSuccess;
    const int grid = grid_for(g.n, 256);
    cudaError_t e = cudaMemsetAsync(w.settled, 0, sizeof(int32_t) * (L + 1), s);
    if (e != cudaSuccess) return e;
    auto init = long_rows ? k_sched_init<true> : k_sched_init<false>;
    auto round = long_rows ? k_sched_round<true> : k_sched_round<false>;
    init<<<grid, 256, 0, s>>>(g.n, g.off, g.deg, g.idx, state, gid, vseg, gpass, w.cnt, w.layer, w.settled);
    for (int32_t r = 0; r + 2 <= L - 1; ++r)  // produce layers 1 .. L-2
        round<<<grid, 256, 0, s>>>(g.n, g.off, g.deg, g.idx, state, gid, vseg, gpass, r, w.cnt, w.layer, w.settled);
    k_sched_finish<<<grid, 256, 0, s>>>(g.n, state, L, B, gid, vseg, gpass, w.layer, step);
    return cudaGetLastError();
}
cudaError_t launch_step_bin_keys(const int32_t *step, const int32_t *deg, int64_t n, int32_t nsteps, bool bin_major,
                                 int32_t *key, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_bin_keys<<<grid_for(n, 256), 256, 0, s>>>(step, deg, n, nsteps, bin_major, key);
    return cudaGetLastError();
}

}  // namespace lgb
