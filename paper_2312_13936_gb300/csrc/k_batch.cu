// Batches of independent graphs (a disjoint union swept as one graph).
//
// Graph g of a batch owns the vertex range [vseg[g], vseg[g+1]) of every
// pass's graph; gid maps a vertex to its graph. Nothing of Algorithm 1
// couples two graphs except the shared launches: each graph keeps its own
// 2m (Eq. 1, Eq. 2), its own convergence tests and its own pass count, and a
// graph that stops (Algorithm 1's two break conditions) leaves the union at
// the next renumbering, its vertices' final labels fixed in the dendrogram.
// These kernels hold the per-graph bookkeeping of that scheme.
#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_graph_ids(const int64_t *vseg, int32_t G, int64_t n, int32_t *gid) {
    GRID_STRIDE(v, n) {
        // the last g with vseg[g] <= v (empty graphs share their start with the next one)
        int32_t lo = 0, hi = G;
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if (__ldg(&vseg[mid]) <= v) lo = mid;
            else hi = mid;
        }
        gid[v] = lo;
    }
}

__global__ void k_globalize(const int64_t *vseg, const int32_t *gid, int64_t n, const int64_t *off, int64_t m,
                            int32_t *idx, int *err) {
    GRID_STRIDE(v, n) {
        const int32_t g = gid[v];
        const int64_t base = vseg[g], ng = vseg[g + 1] - base;
        const int64_t e0 = off[v], e1 = off[v + 1];
        if (e0 < 0 || e1 > m || e1 < e0) {  // malformed offsets: nothing is written
            set_error(err, 1);
            continue;
        }
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t j = idx[e];
            if (j < 0 || j >= ng) {
                set_error(err, 1);  // malformed: a local index outside the graph
                idx[e] = (int32_t)base;
            } else {
                idx[e] = (int32_t)(base + j);
            }
        }
    }
}

// per-graph sums of K: every thread takes a run of consecutive vertices and
// flushes its running sum when the graph changes
constexpr int kRun = 16;
template <class A, class T> __global__ void k_graph_sums(const A *K, const int32_t *gid, int64_t n, T *out) {
    GAcc<T> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kRun;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRun; r < n; r += stride) {
        const int64_t end = r + kRun < n ? r + kRun : n;
        for (int64_t i = r; i < end; ++i) gacc_add(acc, true, gid[i], (T)K[i], out);
    }
    gacc_flush(acc, out);
}

__global__ void k_graph_scales_det(const long long *sums, int32_t G, long long *gks, double *g2m) {
    GRID_STRIDE(g, G) {
        gks[g] = sums[g];
        g2m[g] = (double)sums[g];
    }
}
__global__ void k_graph_scales_async(const double *sums, int32_t G, float *gks, double *g2m) {
    GRID_STRIDE(g, G) {
        const double t = sums[g];
        gks[g] = t > 0 ? (float)(1.0 / t) : 0.0f;  // a graph without edges sweeps no vertex
        g2m[g] = t;
    }
}

__global__ void k_phase_init(const int32_t *state, int32_t G, int32_t *gdone, int32_t *giters) {
    GRID_STRIDE(g, G) {
        gdone[g] = state[g] != kGraphActive ? 1 : 0;
        giters[g] = 0;
    }
}

// gz[g] += vertices of graph g without edges (one atomic per graph per warp)
__global__ void k_graph_zero_deg(const int32_t *deg, const int32_t *gid, int64_t n, unsigned long long *gz) {
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n;
         v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + lane;
        const bool z = v < n && deg[v] == 0;
        if (!__ballot_sync(kFull, z)) continue;
        const int32_t g = (z && gid) ? gid[v] : 0;
        const unsigned peers = __match_any_sync(kFull, z ? g : -1);
        if (z && lane == __ffs(peers) - 1) atomicAdd(&gz[g], (unsigned long long)__popc(peers));
    }
}

__global__ void k_graph_stop(const int64_t *vseg, const int64_t *pos, const int64_t *pos2, const int32_t *li,
                             const double *g2m, double agg_tol, int32_t G, int32_t *state, int64_t *keep,
                             int32_t *passes, const int32_t *gpass, int32_t max_passes,
                             const unsigned long long *gz, int32_t *fresh, bool refine_labels) {
    GRID_STRIDE(g, G) {
        if (state[g] != kGraphActive) {
            keep[g] = 0;
            continue;
        }
        passes[g]++;
        const int64_t a = vseg[g], b = vseg[g + 1];
        const int64_t ncomm = pos[b] - pos[a], nbound = pos2[b] - pos2[a];
        // R4 leaves out the z vertices without edges (each is its own community)
        const int64_t z = (int64_t)gz[g], live = (b - a) - z;
        const bool stop = !(g2m[g] > 0)                              // reading R12: no edges
                          || (li[g] <= 1 && nbound == ncomm && fresh[g])  // globally converged (R5')
                          || (live > 0 && (double)(ncomm - z) / (double)live > agg_tol)  // low shrink (R4)
                          || (gpass && gpass[g] + 1 >= max_passes);   // its MAX_PASSES
        if (stop) {
            state[g] = kGraphFinishing;
            keep[g] = 0;
        } else {
            keep[g] = ncomm;
            // R5': the next pass begins from singletons when every
            // local-moving community is one refined community (move-based
            // labels), or always under refine-based labels
            fresh[g] = (refine_labels || nbound == ncomm) ? 1 : 0;
        }
    }
}

__global__ void k_renumber_batch(const int32_t *C, const int64_t *pos, const int32_t *gid, const int64_t *vseg,
                                 const int64_t *vseg2, const int32_t *state, int32_t *Cd, int64_t n) {
    GRID_STRIDE(i, n) {
        const int32_t g = gid ? gid[i] : 0;
        Cd[i] = state[g] == kGraphActive ? (int32_t)(vseg2[g] + pos[C[i]] - pos[vseg[g]]) : -1;
    }
}

__global__ void k_lookup_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                               const int32_t *state, const int32_t *Cd, const int32_t *Cp, int64_t n0) {
    GRID_STRIDE(v, n0) {
        const int32_t g = gid0 ? gid0[v] : 0;
        const int32_t st = state[g];
        if (st == kGraphActive) C0[v] = Cd[C0[v]];
        else if (st == kGraphFinishing) C0[v] = (int32_t)(vseg0[g] + Cp[C0[v]] - vseg[g]);
    }
}

__global__ void k_finalize_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                                 const int32_t *state, int64_t n0) {
    GRID_STRIDE(v, n0) {
        const int32_t g = gid0[v];
        if (state[g] == kGraphActive) C0[v] = (int32_t)(vseg0[g] + C0[v] - vseg[g]);
    }
}

__global__ void k_commit_states(int32_t *state, int32_t G) {
    GRID_STRIDE(g, G) if (state[g] == kGraphFinishing) state[g] = kGraphFinished;
}

__global__ void k_init_labels(const int32_t *label, int64_t n_cont, int64_t n, int32_t *Cp) {
    GRID_STRIDE(v, n) Cp[v] = v < n_cont ? label[v] : (int32_t)v;
}

// one thread per row of the appended graph
__global__ void k_append_graph(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int64_t v0,
                               int64_t e0, bool w_int, int32_t g, int64_t *out_off, int32_t *out_deg,
                               int32_t *out_idx, float *out_wf, WInt *out_wi, int32_t *gid, int32_t *C0,
                               int64_t a0) {
    GRID_STRIDE(i, n) {
        const int64_t a = off[i], b = off[i + 1];
        out_off[v0 + i] = e0 + a;
        out_deg[v0 + i] = (int32_t)(b - a);
        for (int64_t e = a; e < b; ++e) {
            out_idx[e0 + e] = (int32_t)(v0 + idx[e]);
            if (w_int) out_wi[e0 + e] = (WInt)w[e];
            else out_wf[e0 + e] = w[e];
        }
        gid[v0 + i] = g;
        C0[a0 + i] = (int32_t)(v0 + i);
    }
}

__global__ void k_shift_labels(const int32_t *src, int64_t n, int64_t off, int32_t *dst) {
    GRID_STRIDE(v, n) dst[v] = (int32_t)(src[v] - off);
}

__global__ void k_graph_counts(const int64_t *pos, const int64_t *vseg, int32_t G, int64_t *out) {
    GRID_STRIDE(g, G) out[g] = pos[vseg[g + 1]] - pos[vseg[g]];
}

__global__ void k_next_gid(const int32_t *Cd, const int32_t *gid, int64_t n, int32_t *gid2) {
    GRID_STRIDE(i, n) {
        const int32_t c = Cd[i];
        if (c >= 0) gid2[c] = gid[i];
    }
}

__global__ void k_canonical_batch(const int32_t *C0, const int32_t *minv, const int64_t *rank, const int32_t *gid0,
                                  const int64_t *vseg0, int64_t n0, int32_t *out) {
    GRID_STRIDE(v, n0) out[v] = (int32_t)(rank[minv[C0[v]]] - rank[vseg0[gid0[v]]]);
}

// add x to slot 3g+k of every lane's graph: one atomic per warp when the
// whole warp is in one graph (the common case), else one per lane
__device__ __forceinline__ void graph_add(double *gsum, int32_t g, int k, double x) {
    const int32_t g0 = __shfl_sync(kFull, g, 0);
    if (__all_sync(kFull, g == g0)) {
        x = warp_sum(x);
        if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(&gsum[3 * (int64_t)g0 + k], x);
    } else if (x != 0.0) {
        atomicAdd(&gsum[3 * (int64_t)g + k], x);
    }
}

template <bool LONG>
__global__ void k_modularity_batch(int64_t n0, const int64_t *off, const int32_t *idx, const float *w,
                                   const int32_t *C, const int32_t *gid0, const int64_t *vseg0, double *sigtot,
                                   double *gsum, double *bad) {
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n0; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = v0 + threadIdx.x;
        // lanes past the end count nothing in the graph of the warp's first vertex
        const int32_t g = i < n0 ? gid0[i] : gid0[v0];
        double k = 0, in = 0;
        int64_t key = -1;  // slot of Sigma_c
        int32_t ci = -1;
        if (i < n0) {
            const int64_t ng = vseg0[g + 1] - vseg0[g];
            ci = C[i];
            if (ci < 0 || ci >= ng) {
                atomicAdd(bad, 1.0);
                ci = -1;
            }
        }
        warp_rows<LONG>(off, idx, w, C, ci >= 0, i, ci, k, in);
        if (ci >= 0 && k != 0.0) key = vseg0[g] + ci;
        warp_add_by_key(sigtot, key, k);
        graph_add(gsum, g, 0, in);
        graph_add(gsum, g, 1, k);
    }
}
__global__ void k_square_sums_batch(const double *sigtot, const int32_t *gid0, int64_t n0, double *gsum) {
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < n0; c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        const int32_t g = c < n0 ? gid0[c] : gid0[c0];
        const double x = c < n0 ? sigtot[c] : 0.0;
        graph_add(gsum, g, 2, x * x);
    }
}
__global__ void k_graph_q(const double *gsum, int32_t G, double gamma, double *q) {
    GRID_STRIDE(g, G) {
        const double in = gsum[3 * g], tm = gsum[3 * g + 1], sq = gsum[3 * g + 2];
        q[g] = tm > 0 ? in / tm - gamma * sq / (tm * tm) : 0.0;
    }
}

__global__ void k_graph_max_deg(const int32_t *deg, const int32_t *gid, int64_t n, int32_t *out) {
    GRID_STRIDE(v, n) atomicMax(&out[gid[v]], deg[v]);
}

}  // namespace

cudaError_t launch_graph_ids(const int64_t *vseg, int32_t G, int64_t n, int32_t *gid, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_graph_ids<<<grid_for(n, 256), 256, 0, s>>>(vseg, G, n, gid);
    return cudaGetLastError();
}
cudaError_t launch_globalize_indices(const int64_t *vseg, const int32_t *gid, int64_t n, const int64_t *off,
                                     int64_t m, int32_t *idx, int *err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_globalize<<<grid_for(n, 256), 256, 0, s>>>(vseg, gid, n, off, m, idx, err);
    return cudaGetLastError();
}
cudaError_t launch_graph_max_deg(const int32_t *deg, const int32_t *gid, int64_t n, int32_t *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_graph_max_deg<<<grid_for(n, 256), 256, 0, s>>>(deg, gid, n, out);
    return cudaGetLastError();
}
cudaError_t launch_graph_sums(const void *K, bool det, const int32_t *gid, int64_t n, void *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for((n + kRun - 1) / kRun, 256);
    if (det) k_graph_sums<long long, long long><<<grid, 256, 0, s>>>((const long long *)K, gid, n, (long long *)out);
    else k_graph_sums<float, double><<<grid, 256, 0, s>>>((const float *)K, gid, n, (double *)out);
    return cudaGetLastError();
}
cudaError_t launch_graph_scales(const void *sums, bool det, int32_t G, void *gks, double *g2m, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    if (det) k_graph_scales_det<<<grid_for(G, 256), 256, 0, s>>>((const long long *)sums, G, (long long *)gks, g2m);
    else k_graph_scales_async<<<grid_for(G, 256), 256, 0, s>>>((const double *)sums, G, (float *)gks, g2m);
    return cudaGetLastError();
}
cudaError_t launch_phase_init(const int32_t *state, int32_t G, int32_t *gdone, int32_t *giters, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    k_phase_init<<<grid_for(G, 256), 256, 0, s>>>(state, G, gdone, giters);
    return cudaGetLastError();
}
cudaError_t launch_graph_stop(const int64_t *vseg, const int64_t *pos, const int64_t *pos2, const int32_t *li,
                              const double *g2m, double agg_tol, int32_t G, int32_t *state, int64_t *keep,
                              int32_t *passes, cudaStream_t s, const int32_t *gpass, int32_t max_passes,
                              const int32_t *deg, const int32_t *gid, int64_t n, unsigned long long *gz,
                              int32_t *fresh, bool refine_labels) {
    if (G <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(gz, 0, sizeof(unsigned long long) * G, s);
    if (e != cudaSuccess) return e;
    if (n > 0) k_graph_zero_deg<<<grid_for(n, 256), 256, 0, s>>>(deg, gid, n, gz);
    k_graph_stop<<<grid_for(G, 256), 256, 0, s>>>(vseg, pos, pos2, li, g2m, agg_tol, G, state, keep, passes, gpass,
                                                  max_passes, gz, fresh, refine_labels);
    return cudaGetLastError();
}
cudaError_t launch_renumber_batch(const int32_t *C, const int64_t *pos, const int32_t *gid, const int64_t *vseg,
                                  const int64_t *vseg2, const int32_t *state, int32_t *Cd, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_renumber_batch<<<grid_for(n, 256), 256, 0, s>>>(C, pos, gid, vseg, vseg2, state, Cd, n);
    return cudaGetLastError();
}
cudaError_t launch_lookup_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                                const int32_t *state, const int32_t *Cd, const int32_t *Cp, int64_t n0,
                                cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_lookup_batch<<<grid_for(n0, 256), 256, 0, s>>>(C0, gid0, vseg0, vseg, state, Cd, Cp, n0);
    return cudaGetLastError();
}
cudaError_t launch_finalize_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                                  const int32_t *state, int64_t n0, cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_finalize_batch<<<grid_for(n0, 256), 256, 0, s>>>(C0, gid0, vseg0, vseg, state, n0);
    return cudaGetLastError();
}
cudaError_t launch_commit_states(int32_t *state, int32_t G, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    k_commit_states<<<grid_for(G, 256), 256, 0, s>>>(state, G);
    return cudaGetLastError();
}
cudaError_t launch_init_labels(const int32_t *label, int64_t n_cont, int64_t n, int32_t *Cp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_init_labels<<<grid_for(n, 256), 256, 0, s>>>(label, n_cont, n, Cp);
    return cudaGetLastError();
}
cudaError_t launch_append_graph(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int64_t v0,
                                int64_t e0, bool w_int, int32_t g, int64_t *out_off, int32_t *out_deg,
                                int32_t *out_idx, void *out_w, int32_t *gid, int32_t *C0, int64_t a0,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_append_graph<<<grid_for(n, 256), 256, 0, s>>>(n, off, idx, w, v0, e0, w_int, g, out_off, out_deg, out_idx,
                                                    static_cast<float *>(out_w), static_cast<WInt *>(out_w),
                                                    gid, C0, a0);
    return cudaGetLastError();
}
cudaError_t launch_shift_labels(const int32_t *src, int64_t n, int64_t off, int32_t *dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_shift_labels<<<grid_for(n, 256), 256, 0, s>>>(src, n, off, dst);
    return cudaGetLastError();
}
cudaError_t launch_graph_counts(const int64_t *pos, const int64_t *vseg, int32_t G, int64_t *out, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    k_graph_counts<<<grid_for(G, 256), 256, 0, s>>>(pos, vseg, G, out);
    return cudaGetLastError();
}
cudaError_t launch_next_gid(const int32_t *Cd, const int32_t *gid, int64_t n, int32_t *gid2, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_next_gid<<<grid_for(n, 256), 256, 0, s>>>(Cd, gid, n, gid2);
    return cudaGetLastError();
}
cudaError_t launch_canonical_batch(const int32_t *C0, const int32_t *minv, const int64_t *rank, const int32_t *gid0,
                                   const int64_t *vseg0, int64_t n0, int32_t *out, cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_canonical_batch<<<grid_for(n0, 256), 256, 0, s>>>(C0, minv, rank, gid0, vseg0, n0, out);
    return cudaGetLastError();
}
cudaError_t launch_modularity_batch(int64_t n0, const int64_t *off, const int32_t *idx, const float *w,
                                    const int32_t *C, const int32_t *gid0, const int64_t *vseg0, int32_t G,
                                    double gamma, double *sigtot, double *gsum, double *bad, double *q,
                                    cudaStream_t s, bool long_rows) {
    if (G <= 0) return cudaSuccess;
    if (n0 > 0) {
        auto kern = long_rows ? k_modularity_batch<true> : k_modularity_batch<false>;
        kern<<<grid_for(n0, 256), 256, 0, s>>>(n0, off, idx, w, C, gid0, vseg0, sigtot, gsum, bad);
        k_square_sums_batch<<<grid_for(n0, 256), 256, 0, s>>>(sigtot, gid0, n0, gsum);
    }
    k_graph_q<<<grid_for(G, 256), 256, 0, s>>>(gsum, G, gamma, q);
    return cudaGetLastError();
}

}  // namespace lgb
