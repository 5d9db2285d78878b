// Edge list to symmetric CSR on the GPU: the input preparation of the
// paper's experiments (edges made undirected, reverse edges added, unit
// weight by default; Section 5.1, Table 2). Every edge (u, v) with u != v
// gives the entries (u, v) and (v, u); a self-loop gives one entry (reading
// R11) unless dropped. Entries are first counted per row and scattered into
// row segments (a counting sort by row, with 64-bit positions, so edge lists
// of billions of edges fit); then the rows are cut into chunks of at most
// 2^30 entries, and each chunk is sorted by (row, target) with an LSD radix
// sort whose passes are the stable counting sort of k_util.cu (8-bit digits,
// so its per-block histograms stay small), and entries with equal (row,
// target) are merged (weights summed in fp64 and rounded once, or the
// largest kept) straight into the output. Row offsets come from a scan of
// the merged row lengths.
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "kernels.h"

namespace lgb {
namespace {

constexpr int kDigitBits = 8;
// entries sorted at once: the counting sort's positions are int32
constexpr int64_t kChunkEntries = (int64_t)1 << 30;

inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// entries per row: row u counts (u, v), row v counts (v, u) for u != v; a
// self-loop counts once unless dropped. err = 1 for an endpoint outside
// [0, n) or a weight that is not finite and >= 0 (such an edge is skipped).
__global__ void k_count_rows(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                             int drop_self, unsigned long long *cnt, int *err) {
    GRID_STRIDE(e, m) {
        const int32_t u = src[e], v = dst[e];
        const float x = w ? w[e] : 1.0f;
        if (!(u >= 0 && u < n && v >= 0 && v < n && isfinite(x) && x >= 0.0f)) {
            set_error(err, 1);
            continue;
        }
        if (u != v) {
            atomicAdd(&cnt[u], 1ULL);
            atomicAdd(&cnt[v], 1ULL);
        } else if (!drop_self) {
            atomicAdd(&cnt[u], 1ULL);
        }
    }
}
// scatter every entry into its row segment: key = (row << 32) | target
// (rows in order, entries of a row in no particular order)
__global__ void k_scatter_rows(int64_t m, const int32_t *src, const int32_t *dst, const float *w, int drop_self,
                               const int64_t *rowstart, unsigned long long *cursor, unsigned long long *key,
                               float *wt) {
    GRID_STRIDE(e, m) {
        const int32_t u = src[e], v = dst[e];
        const float x = w ? w[e] : 1.0f;
        if (u == v && drop_self) continue;
        const int64_t p = rowstart[u] + (int64_t)atomicAdd(&cursor[u], 1ULL);
        key[p] = ((unsigned long long)(uint32_t)u << 32) | (uint32_t)v;
        if (wt) wt[p] = x;
        if (u != v) {
            const int64_t q = rowstart[v] + (int64_t)atomicAdd(&cursor[v], 1ULL);
            key[q] = ((unsigned long long)(uint32_t)v << 32) | (uint32_t)u;
            if (wt) wt[q] = x;
        }
    }
}
// sort digit of entry i of a chunk whose rows start at r0: bits
// [shift, shift + 8) of the relative key ((row - r0) << 32) | target
__global__ void k_digit(const unsigned long long *key, int64_t M, unsigned long long r0, int shift, int32_t *digit) {
    GRID_STRIDE(i, M) digit[i] = (int32_t)(((key[i] - (r0 << 32)) >> shift) & ((1u << kDigitBits) - 1));
}
__global__ void k_gather_kw(const unsigned long long *key, const float *wt, const int32_t *perm, int64_t M,
                            unsigned long long *key2, float *wt2) {
    GRID_STRIDE(i, M) {
        const int32_t p = perm[i];
        key2[i] = key[p];
        if (wt) wt2[i] = wt[p];
    }
}
// first[i] = 1 when sorted entry i starts a run of equal keys
__global__ void k_run_starts(const unsigned long long *key, int64_t M, int32_t *first) {
    GRID_STRIDE(i, M) first[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}
// run r of the chunk (starting at sorted entry i, pos[i] = r) writes its
// target and merged weight (fp64 sum rounded once, or the largest; unit
// weights when wt is null) to out + base + r, while it fits in cap; the
// run's row gains one entry
__global__ void k_merge_runs(const unsigned long long *key, const float *wt, const int32_t *first, const int64_t *pos,
                             int64_t M, int combine, int64_t base, int64_t cap, int32_t *idx, float *wout,
                             unsigned long long *rowlen) {
    GRID_STRIDE(i, M) {
        if (!first[i]) continue;
        const unsigned long long k = key[i];
        double s = wt ? (double)wt[i] : 1.0;
        int64_t j = i + 1;
        for (; j < M && key[j] == k; ++j) {
            const double x = wt ? (double)wt[j] : 1.0;
            s = combine ? fmax(s, x) : s + x;
        }
        const int64_t r = base + pos[i];
        if (r < cap) {
            idx[r] = (int32_t)(uint32_t)k;
            wout[r] = (float)s;
        }
        atomicAdd(&rowlen[k >> 32], 1ULL);
    }
}

}  // namespace

leiden_status csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w, int where,
                             int drop_self, int combine, int64_t *offsets, int32_t *indices, float *weights,
                             int64_t *nnz_io, cudaStream_t s) {
    if (n < 0 || n > INT32_MAX || m < 0 || !nnz_io || !offsets || (m > 0 && (!src || !dst)) ||
        (where != LEIDEN_HOST && where != LEIDEN_DEVICE) || (combine != 0 && combine != 1)) {
        set_last_error("leiden_csr_from_edges: invalid arguments");
        return LEIDEN_ERR_INVALID;
    }
    const int64_t cap = *nnz_io;
    std::vector<void *> mem;
    auto get = [&](void **p, size_t bytes) -> bool {
        if (cudaMallocAsync(p, bytes ? bytes : 1, s) != cudaSuccess) return false;
        mem.push_back(*p);
        return true;
    };
    auto release = [&]() {
        for (void *p : mem) cudaFreeAsync(p, s);
        mem.clear();
    };
    auto fail = [&](leiden_status st, const std::string &msg) {
        release();
        set_last_error(msg);
        return st;
    };
    cudaError_t e = cudaSuccess;
#define IK(x)                                                                                        \
    do {                                                                                             \
        if ((e = (x)) != cudaSuccess) return fail(LEIDEN_ERR_CUDA, std::string("leiden_csr_from_edges: ") + \
                                                  cudaGetErrorString(e));                           \
    } while (0)
    const cudaMemcpyKind in_kind = where == LEIDEN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = where == LEIDEN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int32_t *dsrc = src, *ddst = dst;
    const float *dw = w;
    unsigned long long *cnt = nullptr, *rowlen = nullptr;
    int64_t *rowstart = nullptr, *doff = nullptr;
    int *err = nullptr;
    void *scan_tmp = nullptr;
    if (!get((void **)&cnt, 8 * (size_t)(n + 1)) || !get((void **)&rowstart, 8 * (size_t)(n + 1)) ||
        !get((void **)&rowlen, 8 * (size_t)(n + 1)) || !get((void **)&doff, 8 * (size_t)(n + 1)) ||
        !get((void **)&err, sizeof(int)) || !get(&scan_tmp, scan_tmp_bytes(n + 1)))
        return fail(LEIDEN_ERR_OOM, "leiden_csr_from_edges: device allocation failed");
    if (where == LEIDEN_HOST && m > 0) {  // the edge list on the device
        int32_t *a = nullptr, *b = nullptr;
        float *c = nullptr;
        if (!get((void **)&a, 4 * (size_t)m) || !get((void **)&b, 4 * (size_t)m) || (w && !get((void **)&c, 4 * (size_t)m)))
            return fail(LEIDEN_ERR_OOM, "leiden_csr_from_edges: device allocation failed");
        IK(cudaMemcpyAsync(a, src, 4 * (size_t)m, in_kind, s));
        IK(cudaMemcpyAsync(b, dst, 4 * (size_t)m, in_kind, s));
        if (w) IK(cudaMemcpyAsync(c, w, 4 * (size_t)m, in_kind, s));
        dsrc = a;
        ddst = b;
        dw = c;
    }
    // ---- entries per row, row starts
    IK(cudaMemsetAsync(err, 0, sizeof(int), s));
    IK(cudaMemsetAsync(cnt, 0, 8 * (size_t)(n + 1), s));
    IK(cudaMemsetAsync(rowlen, 0, 8 * (size_t)(n + 1), s));
    if (m > 0) {
        k_count_rows<<<grid_for(m, 256), 256, 0, s>>>(n, m, dsrc, ddst, dw, drop_self, cnt, err);
        IK(cudaGetLastError());
    }
    IK(launch_exclusive_scan(reinterpret_cast<const int64_t *>(cnt), rowstart, n, scan_tmp, s));
    std::vector<int64_t> hstart((size_t)n + 1, 0);
    int herr = 0;
    IK(cudaMemcpyAsync(hstart.data(), rowstart, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, s));
    IK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IK(cudaStreamSynchronize(s));
    if (herr) return fail(LEIDEN_ERR_INVALID, "leiden_csr_from_edges: endpoint outside [0, n) or bad weight");
    const int64_t M = hstart[(size_t)n];  // entries before merging
    // ---- rows into chunks of at most kChunkEntries entries
    std::vector<int64_t> cut = {0};
    for (int64_t r = 0; r < n;) {
        int64_t r1 = r + 1;
        if (hstart[(size_t)r1] - hstart[(size_t)r] > kChunkEntries)
            return fail(LEIDEN_ERR_INVALID, "leiden_csr_from_edges: a row of more than 2^30 entries before merging");
        // the furthest row end within the chunk budget (binary search)
        int64_t lo = r1, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (hstart[(size_t)mid] - hstart[(size_t)r] <= kChunkEntries) lo = mid;
            else hi = mid - 1;
        }
        r = lo;
        cut.push_back(r);
    }
    int64_t chunk_max = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k)
        chunk_max = std::max(chunk_max, hstart[(size_t)cut[k + 1]] - hstart[(size_t)cut[k]]);
    // ---- scatter into row segments
    unsigned long long *key = nullptr, *key2 = nullptr;
    float *wt = nullptr, *wt2 = nullptr, *stw = nullptr;
    int32_t *digit = nullptr, *perm = nullptr, *first = nullptr, *sti = nullptr;
    int64_t *pos = nullptr, *key_off = nullptr;
    void *part_tmp = nullptr, *cscan_tmp = nullptr;
    if (M > 0) {
        if (!get((void **)&key, 8 * (size_t)M) || (dw && !get((void **)&wt, 4 * (size_t)M)) ||
            !get((void **)&key2, 8 * (size_t)chunk_max) || (dw && !get((void **)&wt2, 4 * (size_t)chunk_max)) ||
            !get((void **)&digit, 4 * (size_t)chunk_max) || !get((void **)&perm, 4 * (size_t)chunk_max) ||
            !get((void **)&first, 4 * (size_t)chunk_max) || !get((void **)&pos, 8 * (size_t)(chunk_max + 1)) ||
            !get((void **)&key_off, 8 * ((1 << kDigitBits) + 2)) ||
            !get(&part_tmp, partition_tmp_bytes(chunk_max, 1 << kDigitBits)) ||
            !get(&cscan_tmp, scan_tmp_bytes(chunk_max + 1)))
            return fail(LEIDEN_ERR_OOM, "leiden_csr_from_edges: device allocation failed");
        if (where == LEIDEN_HOST &&
            (!get((void **)&sti, 4 * (size_t)chunk_max) || !get((void **)&stw, 4 * (size_t)chunk_max)))
            return fail(LEIDEN_ERR_OOM, "leiden_csr_from_edges: device allocation failed");
        IK(cudaMemsetAsync(cnt, 0, 8 * (size_t)(n + 1), s));  // the cursors
        k_scatter_rows<<<grid_for(m, 256), 256, 0, s>>>(m, dsrc, ddst, dw, drop_self, rowstart, cnt, key, wt);
        IK(cudaGetLastError());
    }
    int tbits = 1;  // bits of a target
    while ((1LL << tbits) < n) ++tbits;
    // ---- per chunk: sort by (row, target), merge runs into the output
    int64_t nnz = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        const int64_t r0 = cut[k], r1 = cut[k + 1];
        const int64_t a = hstart[(size_t)r0], Mc = hstart[(size_t)r1] - a;
        if (Mc == 0) continue;
        int rbits = 0;  // bits of a row relative to r0
        while ((1LL << rbits) < r1 - r0) ++rbits;
        unsigned long long *ck = key + a, *ck2 = key2;
        float *cw = wt ? wt + a : nullptr, *cw2 = wt2;
        std::vector<int> shifts;
        for (int sh = 0; sh < tbits; sh += kDigitBits) shifts.push_back(sh);
        for (int sh = 0; sh < rbits; sh += kDigitBits) shifts.push_back(32 + sh);
        for (int sh : shifts) {
            k_digit<<<grid_for(Mc, 256), 256, 0, s>>>(ck, Mc, (unsigned long long)r0, sh, digit);
            IK(cudaGetLastError());
            IK(launch_partition(digit, Mc, 1 << kDigitBits, key_off, perm, part_tmp, s));
            k_gather_kw<<<grid_for(Mc, 256), 256, 0, s>>>(ck, cw, perm, Mc, ck2, cw2);
            IK(cudaGetLastError());
            std::swap(ck, ck2);
            std::swap(cw, cw2);
        }
        k_run_starts<<<grid_for(Mc, 256), 256, 0, s>>>(ck, Mc, first);
        IK(cudaGetLastError());
        IK(launch_exclusive_scan_i32(first, pos, Mc, cscan_tmp, s));
        int64_t runs = 0;
        IK(cudaMemcpyAsync(&runs, pos + Mc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        IK(cudaStreamSynchronize(s));
        const bool fits = nnz + runs <= cap && (runs == 0 || (indices && weights));
        if (where == LEIDEN_DEVICE || !fits) {
            k_merge_runs<<<grid_for(Mc, 256), 256, 0, s>>>(ck, cw, first, pos, Mc, combine, nnz, fits ? cap : 0,
                                                           indices, weights, rowlen);
            IK(cudaGetLastError());
        } else {  // staged on the device, then to the host buffers
            k_merge_runs<<<grid_for(Mc, 256), 256, 0, s>>>(ck, cw, first, pos, Mc, combine, 0, runs, sti, stw,
                                                           rowlen);
            IK(cudaGetLastError());
            IK(cudaMemcpyAsync(indices + nnz, sti, 4 * (size_t)runs, out_kind, s));
            IK(cudaMemcpyAsync(weights + nnz, stw, 4 * (size_t)runs, out_kind, s));
            IK(cudaStreamSynchronize(s));
        }
        nnz += runs;
    }
    *nnz_io = nnz;
    if (nnz > cap || (nnz > 0 && (!indices || !weights)))
        return fail(LEIDEN_ERR_INVALID, "leiden_csr_from_edges: output capacity below the entry count");
    // ---- offsets: scan of the merged row lengths
    IK(launch_exclusive_scan(reinterpret_cast<const int64_t *>(rowlen), doff, n, scan_tmp, s));
    IK(cudaMemcpyAsync(offsets, doff, 8 * (size_t)(n + 1), out_kind, s));
    IK(cudaStreamSynchronize(s));
#undef IK
    release();
    return LEIDEN_OK;
}

}  // namespace lgb
