// Utility kernels: fills, degrees, vertex weights (Algorithm 1,
// vertexWeights), exclusive scans (Algorithm 4's exclusiveScan and the
// renumbering), bucket partition by (schedule step, degree bin), CSR
// validation.
#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

__global__ void k_iota(int32_t *a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}
__global__ void k_fill_i32(int32_t *a, int32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}
__global__ void k_fill_u64(unsigned long long *a, unsigned long long v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}
__global__ void k_degrees(const int64_t *off, int32_t *deg, int64_t n, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = off[i + 1] - off[i];
        if (d < 0 || d > 0x7fffffff) set_error(err, 1);  // malformed offsets
        deg[i] = (int32_t)(d < 0 ? 0 : d);
    }
}

// K_i = sum of row i. One thread per row; rows longer than 64 entries are
// left to k_vertex_weights_long (their K_i starts at 0 here).
template <class A, class T, class W>
__global__ void k_vertex_weights(int64_t n, const int64_t *off, const int32_t *deg, const W *w, A *K, T *two_m) {
    const int lane = threadIdx.x & 31;
    T local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[i];
        A s = 0;
        if (d <= 64) {
            const int64_t e0 = off[i];
            for (int32_t e = 0; e < d; ++e) s += wconv<A>(w[e0 + e]);
            local += s;
        }
        K[i] = s;
    }
    local = warp_sum(local);
    if (lane == 0 && local != (T)0) atomic_add_acc(two_m, local);
}

// K_i of the rows longer than 64 entries, balanced over rows and entries
// together (holey CSR: row r holds entries [off[r], off[r] + deg[r]) of
// [off[r], off[r+1])). Row r and entry e of it take positions r + off[r]
// and r + 1 + e of one merged sequence of T = n + M items (M = off[n-1] +
// deg[n-1]); warp k of W takes positions [T k / W, T (k+1) / W) (W at most
// T / 4096), finds the row at its first position by binary search over
// r + off[r], walks its rows 32 at a time and sums the long ones' entries
// that fall in its range with all lanes, adding them to K_i and 2m. A hub's
// row is thus shared by the warps its entries span, and no warp walks more
// than its share of rows (a graph of millions of empty rows and few entries,
// as late aggregated graphs are, would leave a range of entries a walk over
// millions of rows).
template <class A, class T, class W>
__global__ void k_vertex_weights_long(int64_t n, const int64_t *off, const int32_t *deg, const W *w, A *K,
                                      T *two_m) {
    constexpr int64_t kMinRange = 4096;
    const int lane = threadIdx.x & 31;
    const int64_t M = off[n - 1] + deg[n - 1], Tn = n + M;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t Wg = ((int64_t)gridDim.x * blockDim.x) >> 5, Wm = (Tn + kMinRange - 1) / kMinRange;
    const int64_t Wn = Wg < Wm ? Wg : Wm;
    if (wid >= Wn) return;
    const int64_t P0 = (int64_t)((__int128)Tn * wid / Wn), P1 = (int64_t)((__int128)Tn * (wid + 1) / Wn);
    if (P0 >= P1) return;
    int64_t lo = 0, hi = n;  // the last row r with r + off[r] <= P0
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (mid + off[mid] <= P0) lo = mid;
        else hi = mid;
    }
    T local = 0;
    for (int64_t r = lo; r < n; r += 32) {
        const int64_t row = r + lane;
        const bool valid = row < n;
        const int64_t a = valid ? off[row] : M;
        const int32_t d = valid ? deg[row] : 0;
        const int64_t s0 = a > P0 - row - 1 ? a : P0 - row - 1;  // its entries in the range
        const int64_t t0 = a + d < P1 - row - 1 ? a + d : P1 - row - 1;
        const int64_t next = row + 1 < n ? row + 1 + off[row + 1] : Tn;  // the next row's position
        unsigned todo = __ballot_sync(kFull, valid && d > 64 && s0 < t0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t x0 = __shfl_sync(kFull, s0, src), x1 = __shfl_sync(kFull, t0, src);
            A sum = 0;
            for (int64_t x = x0 + lane; x < x1; x += 32) sum += wconv<A>(w[x]);
            sum = warp_sum(sum);
            if (lane == 0 && sum != (A)0) {
                atomic_add_acc(&K[r + src], sum);
                local += (T)sum;
            }
        }
        if (__ballot_sync(kFull, !valid || next >= P1)) break;  // the range ends in this batch of rows
    }
    if (lane == 0 && local != (T)0) atomic_add_acc(two_m, local);
}

// ---- exclusive scan: tile reduce, scan of tile sums, tile rescan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *s_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wib] = x;
    __syncthreads();
    if (wib == 0) {
        const int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    const int64_t before = wib > 0 ? s_warp[wib - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

template <class T> __global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T *in, int64_t n, int64_t *part) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    int64_t total;
    block_excl_scan(s, s_warp, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}
__global__ void __launch_bounds__(1024) k_scan_parts(int64_t *part, int64_t nb) {
    __shared__ int64_t s_warp[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? part[i] : 0;
        int64_t total;
        const int64_t ex = block_excl_scan(v, s_warp, &total);
        if (i < nb) part[i] = carry + ex;
        carry += total;
    }
}
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const T *in, int64_t *out, int64_t n, const int64_t *part,
                                                            int64_t nb) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_excl_scan(s, s_warp, &total) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = part[blockIdx.x] + total;
}

template <class T> cudaError_t scan_impl(const T *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *part = static_cast<int64_t *>(tmp);
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part);
    k_scan_parts<<<1, 1024, 0, s>>>(part, nb);
    k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part, nb);
    return cudaGetLastError();
}

// ---- stable partition by key (a counting sort): every block owns a tile of
// kPartTile consecutive items; counts per (key, block) are scanned key-major,
// so the items of one key keep their input order.
constexpr int kPartThreads = 256;
constexpr int kPartRounds = 8;
constexpr int kPartTile = kPartThreads * kPartRounds;

__global__ void __launch_bounds__(kPartThreads) k_spart_count(const int32_t *key, int64_t n, int32_t nkeys,
                                                              int64_t nblocks, int64_t *counts) {
    extern __shared__ int32_t s_cnt[];
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) s_cnt[k] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    for (int r = 0; r < kPartRounds; ++r) {
        const int64_t i = base + (int64_t)r * kPartThreads + threadIdx.x;
        if (i < n) {
            const int32_t k = key[i];
            if (k >= 0) atomicAdd(&s_cnt[k], 1);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) counts[(int64_t)k * nblocks + blockIdx.x] = s_cnt[k];
}

__global__ void k_spart_key_off(const int64_t *pos, int32_t nkeys, int64_t nblocks, int64_t *key_off) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= nkeys; k += (int64_t)gridDim.x * blockDim.x)
        key_off[k] = pos[k * nblocks];
}

// within a tile, warps take the items of a round in lane order; per key, a
// warp's items land after those of lower warps and earlier rounds
__global__ void __launch_bounds__(kPartThreads) k_spart_scatter(const int32_t *key, int64_t n, int32_t nkeys,
                                                                int64_t nblocks, const int64_t *pos, int32_t *list) {
    extern __shared__ int32_t s_run[];      // nkeys running counts
    __shared__ int32_t s_wcnt[kPartThreads / 32][32];  // per warp: count of the key its lane leads
    __shared__ int32_t s_wkey[kPartThreads / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) s_run[k] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    for (int r = 0; r < kPartRounds; ++r) {
        const int64_t i = base + (int64_t)r * kPartThreads + threadIdx.x;
        const int32_t k = i < n ? key[i] : -1;
        const unsigned peers = __match_any_sync(kFull, k);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        // leaders publish their key and count
        s_wkey[wib][lane] = (lane == leader && k >= 0) ? k : -1;
        s_wcnt[wib][lane] = (lane == leader && k >= 0) ? __popc(peers) : 0;
        __syncthreads();
        if (k >= 0) {
            int before = 0;  // items of key k in lower warps of this iteration (r)
            for (int w2 = 0; w2 < wib; ++w2)
                for (int l2 = 0; l2 < 32; ++l2)
                    if (s_wkey[w2][l2] == k) before += s_wcnt[w2][l2];
            list[pos[(int64_t)k * nblocks + blockIdx.x] + s_run[k] + before + rank] = (int32_t)i;
        }
        __syncthreads();
        if (k >= 0 && lane == leader) atomicAdd(&s_run[k], __popc(peers));
        __syncthreads();
    }
}

__global__ void k_max_i32(const int32_t *a, int64_t n, int32_t *out) {
    int32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// CSR validation: offsets monotone, indices in range, weights finite and
// >= 0, and the multiset of (i, j, w) equal to that of (j, i, w), compared
// through sums of a 64-bit mix of each triple (a mismatch is found with
// probability 1 - 2^-64 per differing entry).
__device__ __forceinline__ uint64_t mix_triple(uint64_t i, uint64_t j, uint32_t wbits) {
    uint64_t z = i * 0x9E3779B97F4A7C15ULL ^ (j + 0x632BE59BD9B4E019ULL) * 0xC2B2AE3D27D4EB4FULL ^ (uint64_t)wbits << 17;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// entries [from, to) of row i with stride step
__device__ __forceinline__ void validate_part(int64_t n, int64_t i, const int32_t *idx, const float *w, int64_t a,
                                              int64_t from, int64_t to, int step, int *err,
                                              unsigned long long &fwd, unsigned long long &bwd) {
    for (int64_t e = a + from; e < a + to; e += step) {
        const int32_t j = idx[e];
        if (j < 0 || j >= n) {
            set_error(err, 1);
            continue;
        }
        const float x = w ? w[e] : 1.0f;
        if (!(x >= 0.0f) || isinf(x)) set_error(err, 1);
        const uint32_t bits = __float_as_uint(x);
        fwd += mix_triple((uint64_t)i, (uint64_t)j, bits);
        bwd += mix_triple((uint64_t)j, (uint64_t)i, bits);
    }
}

__global__ void k_validate(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int *err,
                           unsigned long long *sums) {
    unsigned long long fwd = 0, bwd = 0;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        int64_t a = 0, d = 0;
        if (i < n) {
            a = off[i];
            d = off[i + 1] - a;
            if (d < 0) {
                set_error(err, 1);
                d = 0;
            }
            if (d <= 64) validate_part(n, i, idx, w, a, 0, d, 1, err, fwd, bwd);
        }
        unsigned longs = __ballot_sync(kFull, i < n && d > 64);
        while (longs) {  // long rows: the warp together (sums are order-free)
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            validate_part(n, __shfl_sync(kFull, i, src), idx, w, __shfl_sync(kFull, a, src), lane,
                          __shfl_sync(kFull, d, src), 32, err, fwd, bwd);
        }
    }
    fwd = warp_sum(fwd);
    bwd = warp_sum(bwd);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], fwd);
        atomicAdd(&sums[1], bwd);
    }
}
__global__ void k_validate_finish(const unsigned long long *sums, int *err) {
    if (sums[0] != sums[1]) set_error(err, 2);
}

}  // namespace

cudaError_t launch_iota(int32_t *a, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(a, n);
    return cudaGetLastError();
}
namespace {
__global__ void k_list_lens(const int32_t *list, int64_t nl, const int32_t *deg, int32_t *len) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x)
        len[t] = deg[list[t]];
}
template <class W, class A>
__global__ void k_list_rows(const int32_t *list, int64_t nl, const int64_t *off, const int32_t *idx, const W *w,
                            const A *K, const int64_t *loff, int32_t *lidx, W *lw, A *lK) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[t];
        const int64_t e0 = off[v], o = loff[t], d = loff[t + 1] - o;
        for (int64_t k = 0; k < d; ++k) {
            lidx[o + k] = idx[e0 + k];
            lw[o + k] = w[e0 + k];
        }
        lK[t] = K[v];
    }
}
}  // namespace
cudaError_t launch_list_lens(const int32_t *list, int64_t nl, const int32_t *deg, int32_t *len, cudaStream_t s) {
    if (nl <= 0) return cudaSuccess;
    k_list_lens<<<grid_for(nl, 256), 256, 0, s>>>(list, nl, deg, len);
    return cudaGetLastError();
}
cudaError_t launch_list_rows(const int32_t *list, int64_t nl, const GraphView &g, const void *K, bool det,
                             const int64_t *loff, int32_t *lidx, void *lw, void *lK, cudaStream_t s) {
    if (nl <= 0) return cudaSuccess;
    const int gb = grid_for(nl, 256);
    if (det && g.w_int)
        k_list_rows<WInt, long long><<<gb, 256, 0, s>>>(list, nl, g.off, g.idx, (const WInt *)g.w,
                                                        (const long long *)K, loff, lidx, (WInt *)lw, (long long *)lK);
    else if (det)
        k_list_rows<float, long long><<<gb, 256, 0, s>>>(list, nl, g.off, g.idx, (const float *)g.w,
                                                         (const long long *)K, loff, lidx, (float *)lw, (long long *)lK);
    else
        k_list_rows<float, float><<<gb, 256, 0, s>>>(list, nl, g.off, g.idx, (const float *)g.w, (const float *)K,
                                                     loff, lidx, (float *)lw, (float *)lK);
    return cudaGetLastError();
}
cudaError_t launch_fill_u64(unsigned long long *a, unsigned long long v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill_u64<<<grid_for(n, 256), 256, 0, s>>>(a, v, n);
    return cudaGetLastError();
}
cudaError_t launch_fill_i32(int32_t *a, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(a, v, n);
    return cudaGetLastError();
}
cudaError_t launch_degrees(const int64_t *off, int32_t *deg, int64_t n, int *err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_degrees<<<grid_for(n, 256), 256, 0, s>>>(off, deg, n, err);
    return cudaGetLastError();
}
cudaError_t launch_vertex_weights(const GraphView &g, bool det, void *K, void *two_m, cudaStream_t s) {
    if (g.n <= 0) return cudaSuccess;
    const int gb = grid_for(g.n, 256);
    const int gl = 152 * 8;
    if (det) {
        auto *k = static_cast<long long *>(K);
        auto *t = static_cast<long long *>(two_m);
        if (g.w_int) {
            k_vertex_weights<long long, long long, WInt><<<gb, 256, 0, s>>>(g.n, g.off, g.deg, (const WInt *)g.w, k, t);
            k_vertex_weights_long<long long, long long, WInt>
                <<<gl, 256, 0, s>>>(g.n, g.off, g.deg, (const WInt *)g.w, k, t);
        } else {
            k_vertex_weights<long long, long long, float><<<gb, 256, 0, s>>>(g.n, g.off, g.deg, (const float *)g.w, k, t);
            k_vertex_weights_long<long long, long long, float>
                <<<gl, 256, 0, s>>>(g.n, g.off, g.deg, (const float *)g.w, k, t);
        }
    } else {
        auto *k = static_cast<float *>(K);
        auto *t = static_cast<double *>(two_m);
        k_vertex_weights<float, double, float><<<gb, 256, 0, s>>>(g.n, g.off, g.deg, (const float *)g.w, k, t);
        k_vertex_weights_long<float, double, float><<<gl, 256, 0, s>>>(g.n, g.off, g.deg, (const float *)g.w, k, t);
    }
    return cudaGetLastError();
}
size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile + 1) * sizeof(int64_t); }
cudaError_t launch_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, tmp, s);
}
cudaError_t launch_exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, tmp, s);
}
size_t partition_tmp_bytes(int64_t n, int32_t nkeys) {
    const int64_t nblocks = (n + kPartTile - 1) / kPartTile;
    const int64_t cells = (int64_t)nkeys * (nblocks < 1 ? 1 : nblocks) + 1;
    return (size_t)(2 * cells) * sizeof(int64_t) + scan_tmp_bytes(cells);
}
cudaError_t launch_partition(const int32_t *key, int64_t n, int32_t nkeys, int64_t *key_off, int32_t *list, void *tmp,
                             cudaStream_t s) {
    if (nkeys > 8192) return cudaErrorInvalidValue;
    int64_t nblocks = (n + kPartTile - 1) / kPartTile;
    if (nblocks < 1) nblocks = 1;
    const int64_t cells = (int64_t)nkeys * nblocks;
    int64_t *counts = static_cast<int64_t *>(tmp);
    int64_t *pos = counts + cells + 1;
    void *stmp = pos + cells + 1;
    cudaError_t e;
    if (n > 0) {
        k_spart_count<<<(unsigned)nblocks, kPartThreads, sizeof(int32_t) * nkeys, s>>>(key, n, nkeys, nblocks, counts);
    } else if ((e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * cells, s)) != cudaSuccess) {
        return e;
    }
    if ((e = scan_impl<int64_t>(counts, pos, cells, stmp, s)) != cudaSuccess) return e;
    k_spart_key_off<<<grid_for(nkeys + 1, 256), 256, 0, s>>>(pos, nkeys, nblocks, key_off);
    if (n > 0)
        k_spart_scatter<<<(unsigned)nblocks, kPartThreads, sizeof(int32_t) * nkeys, s>>>(key, n, nkeys, nblocks, pos,
                                                                                       list);
    return cudaGetLastError();
}
cudaError_t launch_max_i32(const int32_t *a, int64_t n, int32_t *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    k_max_i32<<<grid_for(n, 256), 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}
cudaError_t launch_validate(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int *err,
                            cudaStream_t s) {
    // sums live right after the error word (caller provides int[4] aligned to 8)
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(err + 2);
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (n > 0) k_validate<<<grid_for(n, 256), 256, 0, s>>>(n, off, idx, w, err, sums);
    k_validate_finish<<<1, 1, 0, s>>>(sums, err);
    return cudaGetLastError();
}

}  // namespace lgb
