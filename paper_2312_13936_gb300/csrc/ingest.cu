// Edge list to symmetric CSR on the GPU: the input preparation of the
// paper's experiments (edges made undirected, reverse edges added, unit
// weight by default; Section 5.1, Table 2). Every edge (u, v) with u != v
// gives the entries (u, v) and (v, u); a self-loop gives one entry (reading
// R11) unless dropped. The entries are sorted by (row, target) with an LSD
// radix sort whose passes are the stable counting sort of k_util.cu (8-bit
// digits, so its per-block histograms stay small), then entries with equal
// (row, target) are merged (weights summed, or the largest kept), and the
// row offsets are read off the sorted rows.
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

inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}
#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// entries of edge e: position 2e (u, v) and 2e+1 (v, u) with key
// (row << 32) | target; a dropped entry (the second of a self-loop, or both
// when self-loops are dropped) gets the key n << 32 (row n, after every real
// row). err: 1 for an endpoint outside [0, n) or a bad weight.
__global__ void k_expand(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                         int drop_self, unsigned long long *key, float *wt, int *err) {
    const unsigned long long none = (unsigned long long)n << 32;
    GRID_STRIDE(e, m) {
        const int32_t u = src[e], v = dst[e];
        const float x = w ? w[e] : 1.0f;
        const bool ok = u >= 0 && u < n && v >= 0 && v < n && isfinite(x) && x >= 0.0f;
        if (!ok) set_error(err, 1);
        const bool self = u == v;
        const unsigned long long k1 = ((unsigned long long)(uint32_t)u << 32) | (uint32_t)v;
        const unsigned long long k2 = ((unsigned long long)(uint32_t)v << 32) | (uint32_t)u;
        key[2 * e] = (!ok || (self && drop_self)) ? none : k1;
        key[2 * e + 1] = (!ok || self) ? none : k2;
        wt[2 * e] = x;
        wt[2 * e + 1] = x;
    }
}
__global__ void k_digit(const unsigned long long *key, int64_t M, int shift, int32_t *digit) {
    GRID_STRIDE(i, M) digit[i] = (int32_t)((key[i] >> shift) & ((1u << kDigitBits) - 1));
}
__global__ void k_gather_kw(const unsigned long long *key, const float *wt, const int32_t *perm, int64_t M,
                            unsigned long long *key2, float *wt2) {
    GRID_STRIDE(i, M) {
        const int32_t p = perm[i];
        key2[i] = key[p];
        wt2[i] = wt[p];
    }
}
// first[i] = 1 when sorted entry i starts a run of equal keys (dropped
// entries, key n << 32, never count)
__global__ void k_run_starts(const unsigned long long *key, int64_t M, int64_t n, int32_t *first) {
    const unsigned long long none = (unsigned long long)n << 32;
    GRID_STRIDE(i, M) first[i] = key[i] != none && (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}
// run r (starting at sorted i, pos[i] = r) writes its target and its merged
// weight (sum, or largest) to out[r]
__global__ void k_merge_runs(const unsigned long long *key, const float *wt, const int32_t *first, const int64_t *pos,
                             int64_t M, int combine, int32_t *idx, float *wout) {
    GRID_STRIDE(i, M) {
        if (!first[i]) continue;
        const unsigned long long k = key[i];
        float s = wt[i];
        for (int64_t j = i + 1; j < M && key[j] == k; ++j) s = combine ? fmaxf(s, wt[j]) : s + wt[j];
        const int64_t r = pos[i];
        idx[r] = (int32_t)(uint32_t)k;
        wout[r] = s;
    }
}
// offsets: off[u] = first output entry of row u (rows without entries take
// the next row's start); the last run also ends every row after it at nnz
__global__ void k_row_offsets(const unsigned long long *key, const int32_t *first, const int64_t *pos, int64_t M,
                              int64_t n, int64_t nnz, int64_t *off) {
    const unsigned long long none = (unsigned long long)n << 32;
    GRID_STRIDE(i, M) {
        if (!first[i]) continue;
        const int64_t u = (int64_t)(key[i] >> 32);
        // rows (row of the previous run, u] start here: the previous run
        // starts at most one run length before i
        int64_t prev = -1;
        for (int64_t j = i - 1; j >= 0; --j)
            if (first[j]) {
                prev = (int64_t)(key[j] >> 32);
                break;
            }
        for (int64_t r = prev + 1; r <= u; ++r) off[r] = pos[i];
        // the last run (sorted keys: nothing but dropped entries after its
        // run) ends the rows after it
        int64_t j = i + 1;
        while (j < M && key[j] == key[i]) ++j;
        if (j == M || key[j] == none)
            for (int64_t r = u + 1; r <= n; ++r) off[r] = nnz;
    }
}
__global__ void k_fill_i64(int64_t *a, int64_t v, int64_t n) {
    GRID_STRIDE(i, n) a[i] = v;
}

}  // namespace

leiden_status csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w, int where,
                             int drop_self, int combine, int64_t *offsets, int32_t *indices, float *weights,
                             int64_t *nnz_io, cudaStream_t s) {
    if (n < 0 || n > INT32_MAX || m < 0 || !nnz_io || !offsets || (m > 0 && (!src || !dst)) ||
        (where != LEIDEN_HOST && where != LEIDEN_DEVICE) || (combine != 0 && combine != 1) ||
        2 * m > (int64_t)INT32_MAX) {
        set_last_error("leiden_csr_from_edges: invalid arguments (m is limited to 2^30 edges)");
        return LEIDEN_ERR_INVALID;
    }
    const int64_t cap = *nnz_io;
    const int64_t M = 2 * m;
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
    const cudaMemcpyKind in_kind = where == LEIDEN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    int32_t *dsrc = nullptr, *ddst = nullptr, *digit = nullptr, *perm = nullptr, *first = nullptr,
            *didx = nullptr;
    float *dw = nullptr, *wt = nullptr, *wt2 = nullptr, *dwout = nullptr;
    unsigned long long *key = nullptr, *key2 = nullptr;
    int64_t *pos = nullptr, *doff = nullptr, *key_off = nullptr;
    int *err = nullptr;
    void *part_tmp = nullptr, *scan_tmp = nullptr;
    const size_t ptb = partition_tmp_bytes(M, 1 << kDigitBits), stb = scan_tmp_bytes(M + 1);
    if (!get((void **)&dsrc, 4 * (size_t)m) || !get((void **)&ddst, 4 * (size_t)m) ||
        (w && !get((void **)&dw, 4 * (size_t)m)) || !get((void **)&key, 8 * (size_t)M) ||
        !get((void **)&key2, 8 * (size_t)M) || !get((void **)&wt, 4 * (size_t)M) || !get((void **)&wt2, 4 * (size_t)M) ||
        !get((void **)&digit, 4 * (size_t)M) || !get((void **)&perm, 4 * (size_t)M) ||
        !get((void **)&first, 4 * (size_t)M) || !get((void **)&pos, 8 * (size_t)(M + 1)) ||
        !get((void **)&key_off, 8 * ((1 << kDigitBits) + 2)) || !get((void **)&err, sizeof(int)) ||
        !get(&part_tmp, ptb) || !get(&scan_tmp, stb) || !get((void **)&doff, 8 * (size_t)(n + 1)) ||
        !get((void **)&didx, 4 * (size_t)(M ? M : 1)) || !get((void **)&dwout, 4 * (size_t)(M ? M : 1)))
        return fail(LEIDEN_ERR_OOM, "leiden_csr_from_edges: device allocation failed");
    cudaError_t e = cudaSuccess;
#define IK(x)                                                                                        \
    do {                                                                                             \
        if ((e = (x)) != cudaSuccess) return fail(LEIDEN_ERR_CUDA, std::string("leiden_csr_from_edges: ") + \
                                                  cudaGetErrorString(e));                           \
    } while (0)
    IK(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (m > 0) {
        IK(cudaMemcpyAsync(dsrc, src, 4 * (size_t)m, in_kind, s));
        IK(cudaMemcpyAsync(ddst, dst, 4 * (size_t)m, in_kind, s));
        if (w) IK(cudaMemcpyAsync(dw, w, 4 * (size_t)m, in_kind, s));
        k_expand<<<grid_for(m, 256), 256, 0, s>>>(n, m, dsrc, ddst, w ? dw : nullptr, drop_self, key, wt, err);
        IK(cudaGetLastError());
        // LSD radix sort on the bits that (row, target) keys use (rows up to
        // n, the dropped entries' row)
        int bits = 1;
        while ((1LL << bits) <= n) ++bits;
        for (int shift = 0; shift < 32 + bits; shift += kDigitBits) {
            if (shift >= bits && shift < 32) shift = 32;  // the target's unused high bits are 0
            k_digit<<<grid_for(M, 256), 256, 0, s>>>(key, M, shift, digit);
            IK(cudaGetLastError());
            IK(launch_partition(digit, M, 1 << kDigitBits, key_off, perm, part_tmp, s));
            k_gather_kw<<<grid_for(M, 256), 256, 0, s>>>(key, wt, perm, M, key2, wt2);
            IK(cudaGetLastError());
            std::swap(key, key2);
            std::swap(wt, wt2);
        }
        k_run_starts<<<grid_for(M, 256), 256, 0, s>>>(key, M, n, first);
        IK(cudaGetLastError());
        IK(launch_exclusive_scan_i32(first, pos, M, scan_tmp, s));
    } else {
        IK(cudaMemsetAsync(pos, 0, 8, s));
    }
    int64_t nnz = 0;
    int herr = 0;
    IK(cudaMemcpyAsync(&nnz, pos + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    IK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IK(cudaStreamSynchronize(s));
    if (herr) return fail(LEIDEN_ERR_INVALID, "leiden_csr_from_edges: endpoint outside [0, n) or bad weight");
    *nnz_io = nnz;
    if (nnz > cap || (nnz > 0 && (!indices || !weights)))
        return fail(LEIDEN_ERR_INVALID, "leiden_csr_from_edges: output capacity below the entry count");
    if (nnz > 0) {
        k_merge_runs<<<grid_for(M, 256), 256, 0, s>>>(key, wt, first, pos, M, combine, didx, dwout);
        IK(cudaGetLastError());
        k_row_offsets<<<grid_for(M, 256), 256, 0, s>>>(key, first, pos, M, n, nnz, doff);
        IK(cudaGetLastError());
    } else {
        k_fill_i64<<<grid_for(n + 1, 256), 256, 0, s>>>(doff, 0, n + 1);
        IK(cudaGetLastError());
    }
    const cudaMemcpyKind out_kind = where == LEIDEN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    IK(cudaMemcpyAsync(offsets, doff, 8 * (size_t)(n + 1), out_kind, s));
    if (nnz > 0) {
        IK(cudaMemcpyAsync(indices, didx, 4 * (size_t)nnz, out_kind, s));
        IK(cudaMemcpyAsync(weights, dwout, 4 * (size_t)nnz, out_kind, s));
    }
    IK(cudaStreamSynchronize(s));
#undef IK
    release();
    return LEIDEN_OK;
}

}  // namespace lgb
