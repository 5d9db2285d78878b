// Pass bookkeeping of Algorithm 1: community totals, counting and
// renumbering communities, dendrogram lookup, the community-vertex CSR of
// Algorithm 4, move-based labels of the super-vertices, canonical output
// labels and modularity (Eq. 1).
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

template <class A, class T>
__global__ void k_community_totals(const int32_t *C, const A *K, int64_t n, T *Sig, int32_t *size) {
    GRID_STRIDE(i, n) {
        const int32_t c = C[i];
        atomic_add_acc(&Sig[c], (T)K[i]);
        atomicAdd(&size[c], 1);
    }
}
__global__ void k_nonempty(const int32_t *size, int64_t n, int32_t *flag) {
    GRID_STRIDE(i, n) flag[i] = size[i] > 0 ? 1 : 0;
}
__global__ void k_mark(const int32_t *lab, int64_t n, int32_t *flag) {
    GRID_STRIDE(i, n) flag[lab[i]] = 1;
}
__global__ void k_gather_map(const int32_t *map, const int32_t *in, int32_t *out, int64_t n) {
    GRID_STRIDE(i, n) out[i] = map[in[i]];
}
__global__ void k_renumber(const int32_t *C, const int64_t *pos, int32_t *Cd, int64_t n) {
    GRID_STRIDE(i, n) Cd[i] = (int32_t)pos[C[i]];
}
__global__ void k_lookup(int32_t *C0, const int32_t *map, int64_t n0) {
    GRID_STRIDE(v, n0) C0[v] = map[C0[v]];
}
__global__ void k_comm_counts(const int32_t *Cd, const int32_t *deg, int64_t n, int64_t *cnt, int64_t *tdeg) {
    GRID_STRIDE(i, n) {
        const int32_t c = Cd[i];
        if (c < 0) continue;  // a graph of a batch that stopped
        atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[c]), 1ULL);
        atomicAdd(reinterpret_cast<unsigned long long *>(&tdeg[c]), (unsigned long long)deg[i]);
    }
}
__global__ void k_comm_fill(const int32_t *Cd, int64_t n, const int64_t *coff, int32_t *cursor, int32_t *members) {
    GRID_STRIDE(i, n) {
        const int32_t c = Cd[i];
        if (c < 0) continue;
        members[coff[c] + atomicAdd(&cursor[c], 1)] = (int32_t)i;
    }
}
__global__ void k_comm_bin_keys(const int64_t *tdeg, int64_t ncomm, BinBounds bb, int32_t *key) {
    GRID_STRIDE(c, ncomm) {
        const int b = degree_bin(tdeg[c], bb);
        key[c] = b == 0 ? -1 : b;
    }
}
__global__ void k_bound_of(const int32_t *Cd, const int32_t *CB, int64_t n, int32_t *bnd) {
    GRID_STRIDE(i, n) {
        const int32_t c = Cd[i];
        if (c >= 0) bnd[c] = CB[i];  // all members of a refined community share one bound
    }
}
__global__ void k_rep_min(const int32_t *bnd, int64_t ncomm, int32_t *rep) {
    GRID_STRIDE(s, ncomm) atomicMin(&rep[bnd[s]], (int32_t)s);
}
__global__ void k_labels(const int32_t *bnd, const int32_t *rep, int64_t ncomm, int32_t *label) {
    GRID_STRIDE(s, ncomm) label[s] = rep[bnd[s]];
}
// smallest vertex of each community: lanes of a warp that share a label
// reduce among themselves first (few large communities would otherwise
// serialise on one address)
__global__ void k_min_vertex(const int32_t *C0, int64_t n0, int32_t *minv) {
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n0; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const int32_t c = v < n0 ? C0[v] : -1;
        const unsigned peers = __match_any_sync(kFull, c);
        const unsigned m = __reduce_min_sync(peers, (unsigned)(v < n0 ? v : 0x7fffffff));
        if (c >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(&minv[c], (int32_t)m);
    }
}
__global__ void k_first(const int32_t *C0, const int32_t *minv, int64_t n0, int32_t *first) {
    GRID_STRIDE(v, n0) first[v] = (minv[C0[v]] == (int32_t)v) ? 1 : 0;
}
__global__ void k_canonical(const int32_t *C0, const int32_t *minv, const int64_t *rank, int64_t n0, int32_t *out) {
    GRID_STRIDE(v, n0) out[v] = (int32_t)rank[minv[C0[v]]];
}

// Eq. 1: intra-community weight, 2m and Sigma_c of each community, in two
// kernels. Rows of up to kLongRow entries: each by its own lane, whole warps
// stepping through the vertices so that Sigma_c is summed per label in the
// warp before its atomic; every label is range-checked here. Longer rows
// (LONG): by k_modularity_long below, so that no warp walks a hub alone.
template <bool LONG>
__global__ void k_modularity_parts(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                   const int32_t *C, double *sigtot, double *sums) {
    double intra = 0, tot = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        int32_t ci = -1;
        double k = 0, in = 0;
        if (i < n) {
            ci = C[i];
            if (ci < 0 || ci >= n) {  // label out of range: counted in sums[3], not used
                atomicAdd(&sums[3], 1.0);
                ci = -1;
            }
            if (ci >= 0) {
                const int64_t e0 = off[i], d = off[i + 1] - e0;
                if (!LONG || d <= kLongRow) row_part(idx, w, C, e0, 0, d, 1, ci, k, in);
            }
        }
        warp_add_by_key(sigtot, k != 0.0 ? ci : -1, k);
        intra += in;
        tot += k;
    }
    intra = warp_sum(intra);
    tot = warp_sum(tot);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], intra);
        atomicAdd(&sums[1], tot);
    }
}

// Rows longer than kLongRow, balanced over rows and entries together: row r
// and its entry e take positions r + off[r] and r + 1 + e of one merged
// sequence of n + m items; warp k of W takes positions [T k / W,
// T (k+1) / W) (W at most T / 4096), finds the row at its first position by
// binary search over r + off[r], walks its rows 32 at a time and sums the
// long rows' entries in its range with all lanes, four entries per lane in
// flight. A hub's row is thus shared by the warps its entries span, and no
// warp walks more than its share of rows.
constexpr int kModUnroll = 4;
constexpr int64_t kModMinRange = 4096;
__global__ void k_modularity_long(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                  const int32_t *C, double *sigtot, double *sums) {
    const int lane = threadIdx.x & 31;
    const int64_t m = off[n], Tn = n + m;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t Wg = ((int64_t)gridDim.x * blockDim.x) >> 5, Wm = (Tn + kModMinRange - 1) / kModMinRange;
    const int64_t W = Wg < Wm ? Wg : Wm;
    if (wid >= W) return;
    const int64_t P0 = (int64_t)((__int128)Tn * wid / W), P1 = (int64_t)((__int128)Tn * (wid + 1) / W);
    if (P0 >= P1) return;
    int64_t lo = 0, hi = n;  // the last row r with r + off[r] <= P0
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (mid + off[mid] <= P0) lo = mid;
        else hi = mid;
    }
    double intra = 0, tot = 0;
    for (int64_t r = lo; r < n; r += 32) {
        const int64_t row = r + lane;
        const bool valid = row < n;
        const int64_t a = valid ? off[row] : m, b = valid ? off[row + 1] : m;
        const int64_t s0 = a > P0 - row - 1 ? a : P0 - row - 1;  // its entries in the range
        const int64_t t0 = b < P1 - row - 1 ? b : P1 - row - 1;
        const bool mine = valid && b - a > kLongRow && s0 < t0;
        int32_t ci = mine ? C[row] : -1;
        if (ci >= n) ci = -1;  // out of range: counted by k_modularity_parts
        unsigned todo = __ballot_sync(kFull, mine && ci >= 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t s = __shfl_sync(kFull, s0, src), t = __shfl_sync(kFull, t0, src);
            const int32_t c = __shfl_sync(kFull, ci, src);
            double kl = 0, il = 0;
            for (int64_t x0 = s + lane; x0 < t; x0 += 32 * kModUnroll) {
                int32_t j[kModUnroll];
                float wv[kModUnroll];
#pragma unroll
                for (int u = 0; u < kModUnroll; ++u) {
                    const int64_t x = x0 + 32 * u;
                    j[u] = x < t ? idx[x] : -1;
                    wv[u] = x < t ? (w ? w[x] : 1.0f) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < kModUnroll; ++u)
                    if (j[u] >= 0) {
                        kl += (double)wv[u];
                        if (C[j[u]] == c) il += (double)wv[u];
                    }
            }
            kl = warp_sum(kl);
            il = warp_sum(il);
            if (lane == 0 && kl != 0.0) atomicAdd(&sigtot[c], kl);
            intra += il;
            tot += kl;
        }
        const int64_t next = row + 1 < n ? row + 1 + off[row + 1] : Tn;  // the next row's position
        if (__ballot_sync(kFull, !valid || next >= P1)) break;  // the range ends in this batch of rows
    }
    if (lane == 0) {
        atomicAdd(&sums[0], intra);
        atomicAdd(&sums[1], tot);
    }
}

__global__ void k_max_i64(const int64_t *a, int64_t n, unsigned long long *out) {
    unsigned long long m = 0;
    GRID_STRIDE(i, n) m = max(m, (unsigned long long)a[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
// weights: flag non-integer values, sum in fp64 (deterministic-mode checks)
__global__ void k_weight_props(const float *w, int64_t m, int *nonint, double *sum) {
    double s = 0;
    GRID_STRIDE(e, m) {
        const float x = w[e];
        if (x != truncf(x)) atomicExch(nonint, 1);
        s += (double)x;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(sum, s);
}
__global__ void k_sum_squares(const double *x, int64_t n, double *out) {
    double s = 0;
    GRID_STRIDE(i, n) s += x[i] * x[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

}  // namespace

cudaError_t launch_community_totals(const int32_t *C, const void *K, bool det, int64_t n, void *Sig, int32_t *size,
                                    cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (det)
        k_community_totals<long long, long long><<<grid_for(n, 256), 256, 0, s>>>(C, (const long long *)K, n,
                                                                                  (long long *)Sig, size);
    else
        k_community_totals<float, double><<<grid_for(n, 256), 256, 0, s>>>(C, (const float *)K, n, (double *)Sig, size);
    return cudaGetLastError();
}
cudaError_t launch_nonempty_flags(const int32_t *size, int64_t n, int32_t *flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_nonempty<<<grid_for(n, 256), 256, 0, s>>>(size, n, flag);
    return cudaGetLastError();
}
cudaError_t launch_mark_labels(const int32_t *lab, int64_t n, int32_t *flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_mark<<<grid_for(n, 256), 256, 0, s>>>(lab, n, flag);
    return cudaGetLastError();
}
cudaError_t launch_gather_map(const int32_t *map, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gather_map<<<grid_for(n, 256), 256, 0, s>>>(map, in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_renumber(const int32_t *C, const int64_t *pos, int32_t *Cd, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_renumber<<<grid_for(n, 256), 256, 0, s>>>(C, pos, Cd, n);
    return cudaGetLastError();
}
cudaError_t launch_lookup(int32_t *C0, const int32_t *map, int64_t n0, cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_lookup<<<grid_for(n0, 256), 256, 0, s>>>(C0, map, n0);
    return cudaGetLastError();
}
cudaError_t launch_comm_counts(const int32_t *Cd, const int32_t *deg, int64_t n, int64_t *cnt, int64_t *tdeg,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_comm_counts<<<grid_for(n, 256), 256, 0, s>>>(Cd, deg, n, cnt, tdeg);
    return cudaGetLastError();
}
cudaError_t launch_comm_fill(const int32_t *Cd, int64_t n, const int64_t *coff, int32_t *cursor, int32_t *members,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_comm_fill<<<grid_for(n, 256), 256, 0, s>>>(Cd, n, coff, cursor, members);
    return cudaGetLastError();
}
cudaError_t launch_comm_bin_keys(const int64_t *tdeg, int64_t ncomm, const BinBounds &bb, int32_t *key,
                                 cudaStream_t s) {
    if (ncomm <= 0) return cudaSuccess;
    k_comm_bin_keys<<<grid_for(ncomm, 256), 256, 0, s>>>(tdeg, ncomm, bb, key);
    return cudaGetLastError();
}
cudaError_t launch_bound_labels(const int32_t *Cd, const int32_t *CB, int64_t n, int64_t ncomm, int32_t *bnd,
                                int32_t *rep, int32_t *label, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bound_of<<<grid_for(n, 256), 256, 0, s>>>(Cd, CB, n, bnd);
    cudaError_t e = launch_fill_i32(rep, 0x7fffffff, n, s);
    if (e != cudaSuccess) return e;
    k_rep_min<<<grid_for(ncomm, 256), 256, 0, s>>>(bnd, ncomm, rep);
    k_labels<<<grid_for(ncomm, 256), 256, 0, s>>>(bnd, rep, ncomm, label);
    return cudaGetLastError();
}
cudaError_t launch_min_vertex(const int32_t *C0, int64_t n0, int32_t *minv, cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    cudaError_t e = launch_fill_i32(minv, 0x7fffffff, n0, s);
    if (e != cudaSuccess) return e;
    k_min_vertex<<<grid_for(n0, 256), 256, 0, s>>>(C0, n0, minv);
    return cudaGetLastError();
}
cudaError_t launch_first_flags(const int32_t *C0, const int32_t *minv, int64_t n0, int32_t *first, cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_first<<<grid_for(n0, 256), 256, 0, s>>>(C0, minv, n0, first);
    return cudaGetLastError();
}
cudaError_t launch_canonical(const int32_t *C0, const int32_t *minv, const int64_t *rank, int64_t n0, int32_t *out,
                             cudaStream_t s) {
    if (n0 <= 0) return cudaSuccess;
    k_canonical<<<grid_for(n0, 256), 256, 0, s>>>(C0, minv, rank, n0, out);
    return cudaGetLastError();
}
cudaError_t launch_modularity_parts(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                    const int32_t *C, double *sigtot, double *sums, cudaStream_t s,
                                    bool long_rows) {
    if (n <= 0) return cudaSuccess;
    auto kern = long_rows ? k_modularity_parts<true> : k_modularity_parts<false>;
    kern<<<grid_for(n, 256), 256, 0, s>>>(n, off, idx, w, C, sigtot, sums);
    if (!long_rows) return cudaGetLastError();
    k_modularity_long<<<152 * 8, 256, 0, s>>>(n, off, idx, w, C, sigtot, sums);
    return cudaGetLastError();
}
cudaError_t launch_max_i64(const int64_t *a, int64_t n, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    k_max_i64<<<grid_for(n, 256), 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}
cudaError_t launch_weight_props(const float *w, int64_t m, int *nonint, double *sum, cudaStream_t s) {
    if (m <= 0 || !w) return cudaSuccess;
    k_weight_props<<<grid_for(m, 256), 256, 0, s>>>(w, m, nonint, sum);
    return cudaGetLastError();
}
cudaError_t launch_sum_squares(const double *x, int64_t n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_sum_squares<<<grid_for(n, 256), 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

}  // namespace lgb
