// Sweep schedule of a pass (reading S0). h(v) is SplitMix64 output number
// v+1 (v's index inside its graph) and prio(v) = deg(v) * 2^32 + (h(v) >> 32):
// longer rows first, the hash breaking ties; u precedes v when
// prio(u) > prio(v) (ties: smaller id). layer(v) = 1 + max layer of v's
// preceding neighbours (0 if none): the rounds of Jones & Plassmann's
// parallel colouring. One persistent cooperative launch finds them: cnt[v]
// counts v's preceding neighbours, the vertices of layer 0 are appended to
// an order array, and round r walks the vertices of layer r in that array,
// releasing their succeeding neighbours; a neighbour whose last preceding
// neighbour is released joins layer r+1 and is appended. Rounds stop at
// layer L-2 or when a layer is empty; every vertex not placed by then takes
// step L-1 + ((h >> 32) mod B). Each round touches only its own layer, so
// heavy-tailed graphs (thousands of thin layers) cost a grid barrier per
// round, not a pass over all vertices.
// In a batch of graphs a vertex's priority is drawn at its index inside its
// own graph (and, when graphs are at different passes, from the state of its
// own graph's pass), so every graph gets the schedule it would get alone.
#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

constexpr int kSchedThreads = 256;

// first vertex of v's graph (0 for a single graph)
__device__ __forceinline__ int64_t graph_base(const int32_t *gid, const int64_t *vseg, int64_t v) {
    return gid ? __ldg(&vseg[__ldg(&gid[v])]) : 0;
}
// generator state of v's graph: the pass state, advanced by the graph's own
// pass index when graphs are at different passes
__device__ __forceinline__ uint64_t graph_state(uint64_t state, const int32_t *gid, const int32_t *gpass, int64_t v) {
    return gpass ? state + (uint64_t)__ldg(&gpass[__ldg(&gid[v])]) : state;
}
__device__ __forceinline__ uint64_t vprio(uint64_t state, int64_t local, int32_t d) {
    return ((uint64_t)(uint32_t)d << 32) | (splitmix64_at(state, (uint64_t)local) >> 32);
}

struct SA {
    int64_t n;
    const int64_t *off;
    const int32_t *deg, *idx;
    uint64_t state0;
    const int32_t *gid;
    const int64_t *vseg;
    const int32_t *gpass;
    int32_t L, B;        // L: the largest of the graphs' layer caps
    const int32_t *gL;   // layer cap of every graph (null: L for all)
    int32_t *cnt, *layer, *ord, *lord, *step;
    // counters: [0..2] appends to ord, [3..5] appends to lord (round r
    // appends layer r+1 on [(r+1) % 3] and [3 + (r+1) % 3], layer 0 on [0]
    // and [3]; a counter is cleared two rounds before its next use, after
    // every block has read it), [6] long rows listed at the start
    unsigned *size;
    unsigned *bar;   // grid barrier (2 words)
    int32_t *info;   // [0] layers produced, [1] vertices in bucket steps
    int *err;
};

// Appends to a layer of the order array, staged per warp in shared memory:
// one global atomic reserves room for up to kStage vertices at a time (a
// single counter per layer would otherwise take an atomic from every warp
// step). Every lane of the warp calls push and flush together.
constexpr int kStage = 256;
struct Stage {
    int32_t *buf;  // kStage entries of this warp's shared memory
    int count;     // the same in every lane
    __device__ __forceinline__ void flush(int32_t *ord, unsigned *size) {
        if (count == 0) return;
        const int lane = threadIdx.x & 31;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(size, (unsigned)count);
        base = __shfl_sync(kFull, base, 0);
        __syncwarp();
        for (int i = lane; i < count; i += 32) ord[base + i] = buf[i];
        __syncwarp();
        count = 0;
    }
    __device__ __forceinline__ void push(bool take, int32_t v, int32_t *ord, unsigned *size) {
        const unsigned m = __ballot_sync(kFull, take);
        if (!m) return;
        const int lane = threadIdx.x & 31;
        if (take) buf[count + __popc(m & ((1u << lane) - 1u))] = v;
        count += __popc(m);
        if (count > kStage - 32) flush(ord, size);
    }
};

// The long rows [0, R) of a list are shared by all warps: with fewer rows
// than warps, row gw mod R goes to the group of warps congruent to it, which
// split its entries; otherwise every warp takes whole rows gw, gw + warps, ...
// f(i, first entry, entry stride) is called by every lane of the warp.
template <class F>
__device__ __forceinline__ void share_long_rows(int64_t R, int64_t warps, int64_t gw, F &&f) {
    const int lane = threadIdx.x & 31;
    if (R <= 0) return;
    if (R <= warps) {
        const int64_t i = gw % R, k = gw / R;
        const int64_t group = (warps - 1 - i) / R + 1;  // warps congruent to i
        f(i, k * 32 + lane, group * 32);
    } else {
        for (int64_t i = gw; i < R; i += warps) f(i, (int64_t)lane, (int64_t)32);
    }
}

// preceding neighbours of v among row entries [from, to) taken with stride step
__device__ __forceinline__ int32_t count_preceding(const SA &a, int64_t e0, int64_t from, int64_t to, int64_t step,
                                                   uint64_t state, int64_t base, int64_t v, uint64_t pv) {
    int32_t c = 0;
    for (int64_t e = from; e < to; e += step) {
        const int32_t u = a.idx[e0 + e];
        if (u != (int32_t)v && precedes(vprio(state, u - base, __ldg(&a.deg[u])), u, pv, (int32_t)v)) c++;
    }
    return c;
}

// entry e of v's row: true when its vertex u is released by v (v precedes
// u) and v was the last of u's preceding neighbours; u then joins layer r+1
// (Lv: the layer cap of v's graph; layers stop at Lv-2, vertices past it
// stay unplaced)
__device__ __forceinline__ bool release(const SA &a, int64_t e, uint64_t state, int64_t base, int64_t v, uint64_t pv,
                                        int32_t r, int32_t Lv, int32_t &u) {
    u = a.idx[e];
    if (u == (int32_t)v || !precedes(pv, (int32_t)v, vprio(state, u - base, __ldg(&a.deg[u])), u)) return false;
    if (atomicSub(&a.cnt[u], 1) != 1 || r + 2 > Lv - 1) return false;
    a.layer[u] = r + 1;
    return true;
}
__device__ __forceinline__ int32_t layer_cap(const SA &a, int64_t v) {
    return a.gL ? __ldg(&a.gL[__ldg(&a.gid[v])]) : a.L;
}

struct VHead {
    int64_t base, e0;
    uint64_t state, pv;
    int32_t dv, Lv;
};
__device__ __forceinline__ VHead vhead(const SA &a, int64_t v) {
    VHead h;
    h.Lv = layer_cap(a, v);
    h.dv = a.deg[v];
    h.base = graph_base(a.gid, a.vseg, v);
    h.state = graph_state(a.state0, a.gid, a.gpass, v);
    h.pv = vprio(h.state, v - h.base, h.dv);
    h.e0 = a.off[v];
    return h;
}

template <bool LONG>
__global__ void __launch_bounds__(kSchedThreads) k_sched_coop(SA a) {
    __shared__ int32_t s_stage[kSchedThreads / 32][kStage];
    __shared__ int32_t s_lstage[LONG ? kSchedThreads / 32 : 1][kStage];
    const int lane = threadIdx.x & 31;
    Stage st{s_stage[threadIdx.x >> 5], 0};
    Stage lst{s_lstage[LONG ? (threadIdx.x >> 5) : 0], 0};
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // cnt[v] = number of v's preceding neighbours; short rows are counted
    // here (layer 0 if none), long rows are listed (in step[], free until
    // the end) and counted by the whole grid next
    for (int64_t v0 = gw * 32; v0 < a.n; v0 += warps * 32) {
        const int64_t v = v0 + lane;
        const bool in = v < a.n;
        VHead h{};
        if (in) h = vhead(a, v);
        const bool lng = LONG && in && h.dv > kLongRow;
        const int32_t c = (in && !lng) ? count_preceding(a, h.e0, 0, h.dv, 1, h.state, h.base, v, h.pv) : 0;
        if (in) {
            a.cnt[v] = c;
            a.layer[v] = (!lng && c == 0) ? 0 : -1;
        }
        st.push(in && !lng && c == 0, (int32_t)v, a.ord, &a.size[0]);
        if (LONG) lst.push(lng, (int32_t)v, a.step, &a.size[6]);
    }
    st.flush(a.ord, &a.size[0]);
    bool ok = true;
    if (LONG) {
        lst.flush(a.step, &a.size[6]);
        ok = grid_barrier(a.bar, a.err);
        const int64_t nl = ok ? (int64_t)__ldcg(&a.size[6]) : 0;
        share_long_rows(nl, warps, gw, [&](int64_t i, int64_t from, int64_t stride) {
            const int32_t v = __ldcg(&a.step[i]);
            const VHead h = vhead(a, v);
            const int32_t c = warp_sum(count_preceding(a, h.e0, from, h.dv, stride, h.state, h.base, v, h.pv));
            if (lane == 0 && c) atomicAdd(&a.cnt[v], c);
        });
        ok = ok && grid_barrier(a.bar, a.err);
        for (int64_t i0 = gw * 32; i0 < nl; i0 += warps * 32) {
            const int64_t i = i0 + lane;
            int32_t v = 0;
            bool take = false;
            if (i < nl) {
                v = __ldcg(&a.step[i]);
                take = __ldcg(&a.cnt[v]) == 0;
                if (take) a.layer[v] = 0;
            }
            st.push(take, v, a.ord, &a.size[0]);
            lst.push(take, v, a.lord, &a.size[3]);
        }
        st.flush(a.ord, &a.size[0]);
        lst.flush(a.lord, &a.size[3]);
    }
    ok = ok && grid_barrier(a.bar, a.err);
    // round r: layer r is ord[lo, hi) (its long rows also lord[llo, lhi));
    // it appends layer r+1 (up to L-2) from ord[hi] and lord[lhi]
    int64_t lo = 0, hi = ok ? (int64_t)__ldcg(&a.size[0]) : 0;
    int64_t llo = 0, lhi = (ok && LONG) ? (int64_t)__ldcg(&a.size[3]) : 0;
    int32_t r = 0;
    while (ok && hi > lo && r + 2 <= a.L - 1) {
        unsigned *nsz = &a.size[(r + 1) % 3], *nlsz = &a.size[3 + (r + 1) % 3];
        int32_t *nord = a.ord + hi, *nlord = a.lord + lhi;
        if (blockIdx.x == 0 && threadIdx.x == 0) {  // for round r+1
            a.size[(r + 2) % 3] = 0u;
            a.size[3 + (r + 2) % 3] = 0u;
        }
        auto placed = [&](bool take, int32_t u) {
            st.push(take, u, nord, nsz);
            if (LONG) lst.push(take && __ldg(&a.deg[u]) > kLongRow, u, nlord, nlsz);
        };
        // short rows: one lane each, stepping together to the warp's
        // longest short row so that every lane reaches the append
        for (int64_t i0 = lo + gw * 32; i0 < hi; i0 += warps * 32) {
            const int64_t i = i0 + lane;
            int64_t v = 0;
            VHead h{};
            if (i < hi) {
                v = __ldcg(&a.ord[i]);
                h = vhead(a, v);
            }
            const int32_t ds = (i < hi && (!LONG || h.dv <= kLongRow)) ? h.dv : 0;
            int32_t dmax = ds;
            for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(kFull, dmax, o));
            for (int32_t j = 0; j < dmax; ++j) {
                int32_t u = 0;
                const bool take = j < ds && release(a, h.e0 + j, h.state, h.base, v, h.pv, r, h.Lv, u);
                placed(take, u);
            }
        }
        // long rows: shared by the whole grid
        if (LONG)
            share_long_rows(lhi - llo, warps, gw, [&](int64_t i, int64_t from, int64_t stride) {
                const int32_t v = __ldcg(&a.lord[llo + i]);
                const VHead h = vhead(a, v);
                for (int64_t j0 = from - lane; j0 < h.dv; j0 += stride) {
                    int32_t u = 0;
                    const int64_t j = j0 + lane;
                    const bool take = j < h.dv && release(a, h.e0 + j, h.state, h.base, v, h.pv, r, h.Lv, u);
                    placed(take, u);
                }
            });
        st.flush(nord, nsz);
        if (LONG) lst.flush(nlord, nlsz);
        ok = grid_barrier(a.bar, a.err);
        lo = hi;
        hi = ok ? hi + (int64_t)__ldcg(nsz) : lo;
        llo = lhi;
        lhi = (ok && LONG) ? lhi + (int64_t)__ldcg(nlsz) : llo;
        ++r;
    }
    const int32_t layers = r + (hi > lo ? 1 : 0);
    // steps: the layer below the graph's cap Lv-1, else a bucket after L-1
    // (the largest cap: every graph keeps its own order of layers, then
    // buckets); step[] held the long-row list until the last barrier
    unsigned capped = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = a.layer[v];
        if (l >= 0 && l < layer_cap(a, v) - 1) {
            a.step[v] = l;
        } else {
            const uint64_t h = splitmix64_at(graph_state(a.state0, a.gid, a.gpass, v), (uint64_t)(v - graph_base(a.gid, a.vseg, v)));
            a.step[v] = a.L - 1 + (int32_t)((h >> 32) % (uint64_t)a.B);
            capped++;
        }
    }
    capped = warp_sum(capped);
    if (lane == 0 && capped) atomicAdd(reinterpret_cast<unsigned *>(&a.info[1]), capped);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.info[0] = layers;
}

template <bool LONG> int sched_blocks_per_sm() {
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sched_coop<LONG>, kSchedThreads, 0) != cudaSuccess) b = 0;
        per_sm = b;
    }
    return per_sm;
}

__global__ void k_step_bin_keys(const int32_t *step, const int32_t *deg, int64_t n, int32_t nsteps, bool bin_major,
                                BinBounds bb, int32_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int b = degree_bin(deg[v], bb);
        // vertices without edges go to a trailing bucket (never swept)
        key[v] = b == 0 ? nsteps * kNumBins : (bin_major ? b * nsteps + step[v] : step[v] * kNumBins + b);
    }
}

// block k: the hubs of step k go to hubs[base ..) in list order (base: the
// hubs of the steps before); max_span = the largest sum of one step's table
// sizes (2^max(6, ceil log2 2 deg))
__global__ void k_hub_gather(const int64_t *key_off, int32_t nsteps, const int32_t *list, const int32_t *deg,
                             int32_t *hubs, unsigned long long *max_span) {
    __shared__ long long s_part[8];
    const int k = blockIdx.x;
    long long part = 0;  // hubs of the steps before k
    for (int q = threadIdx.x; q < k; q += blockDim.x)
        part += key_off[(int64_t)q * kNumBins + 7] - key_off[(int64_t)q * kNumBins + 6];
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    long long base = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) base += s_part[w];
    __syncthreads();
    const int64_t lo = key_off[(int64_t)k * kNumBins + 6], hi = key_off[(int64_t)k * kNumBins + 7];
    long long span = 0;
    for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
        const int32_t v = list[t];
        hubs[base + (t - lo)] = v;
        int bits = ceil_log2(2 * (int64_t)deg[v]);
        if (bits < 6) bits = 6;
        span += 1LL << bits;
    }
    span = warp_sum(span);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = span;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sp = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sp += s_part[w];
        if (sp) atomicMax(max_span, (unsigned long long)sp);
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
                            const int32_t *gpass, bool long_rows, const int32_t *gL) {
    if (g.n <= 0) return cudaMemsetAsync(w.scratch, 0, sizeof(int32_t) * 11, s);
    if (g.n > INT32_MAX || L < 1 || B < 1) return cudaErrorInvalidValue;
    // scratch: [0..6] counters, [7..8] barrier, [9..10] info
    cudaError_t e = cudaMemsetAsync(w.scratch, 0, sizeof(int32_t) * 11, s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int per_sm = long_rows ? sched_blocks_per_sm<true>() : sched_blocks_per_sm<false>();
    if (per_sm <= 0) return cudaErrorLaunchOutOfResources;
    int64_t grid = (g.n + 4 * kSchedThreads - 1) / (4 * kSchedThreads);  // a few vertices per thread
    if (grid > (int64_t)per_sm * sms) grid = (int64_t)per_sm * sms;
    if (grid < 1) grid = 1;
    SA a;
    a.n = g.n;
    a.off = g.off;
    a.deg = g.deg;
    a.idx = g.idx;
    a.state0 = state;
    a.gid = gid;
    a.vseg = vseg;
    a.gpass = gpass;
    a.L = L;
    a.B = B;
    a.gL = gid ? gL : nullptr;
    a.cnt = w.cnt;
    a.layer = w.layer;
    a.ord = w.ord;
    a.lord = w.lord;
    a.step = step;
    a.size = reinterpret_cast<unsigned *>(w.scratch);
    a.bar = reinterpret_cast<unsigned *>(w.scratch + 7);
    a.info = w.scratch + 9;
    a.err = w.err;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel(long_rows ? (const void *)k_sched_coop<true> : (const void *)k_sched_coop<false>,
                                       dim3((unsigned)grid), dim3(kSchedThreads), args, 0, s);
}
cudaError_t launch_hub_prep(const int64_t *key_off, int32_t nsteps, const int32_t *list, const int32_t *deg,
                            int32_t *hubs, unsigned long long *max_span, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(max_span, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || nsteps <= 0) return e;
    k_hub_gather<<<nsteps, 256, 0, s>>>(key_off, nsteps, list, deg, hubs, max_span);
    return cudaGetLastError();
}
cudaError_t launch_step_bin_keys(const int32_t *step, const int32_t *deg, int64_t n, int32_t nsteps, bool bin_major,
                                 const BinBounds &bb, int32_t *key, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_bin_keys<<<grid_for(n, 256), 256, 0, s>>>(step, deg, n, nsteps, bin_major, bb, key);
    return cudaGetLastError();
}

}  // namespace lgb
