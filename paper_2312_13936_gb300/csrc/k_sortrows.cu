// Rows of a holey CSR sorted by target: the deterministic mode writes every
// aggregated row in ascending target order (reading R10), so the stored
// super-vertex graph is the same bit for bit whatever order the hash tables
// held. Every entry gets the key (row << tb) | target, and the unused slots
// after a row's fill the key (row << tb) | (2^tb - 1), with tb the fewest
// bits that hold every target below the marker, so a stable LSD radix sort
// of the key's tb + row bits (8-bit digits, the counting sort of k_util.cu)
// leaves every row in place with its entries ascending and its unused slots
// last.
// The sort carries a permutation; targets and weights are gathered by it.
// Rows go in chunks of at most 2^30 entries (the counting sort's positions
// are int32).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

constexpr int kSortDigitBits = 8;
constexpr int64_t kSortChunk = (int64_t)1 << 30;

inline int sgrid(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    return (int)(b > 152 * 16 ? 152 * 16 : b);
}
#define SGRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// keys of the slots [e0, e0 + M) of rows [r0, r1): (row - r0) << tb |
// target, and (row - r0) << tb | (2^tb - 1) for a row's unused slots (the
// targets are below 2^tb - 1); ord = iota. Rows and slots take positions of
// one merged sequence (row rr = r - r0 at rr + off[r] - e0, its slot e at
// rr + 1 + e - e0) and warp k of W takes an equal range of it: a binary
// search over the rows finds where its range starts, then it walks its rows
// 32 at a time and writes the keys of their slots in the range with all
// lanes. No per-slot search, and no warp walks more than its share of rows.
__global__ void k_row_keys(const int64_t *off, const int32_t *deg, const int32_t *idx, int64_t r0, int64_t r1,
                           int64_t e0, int64_t M, int tb, unsigned long long *key, int32_t *ord) {
    const int lane = threadIdx.x & 31;
    const int64_t R = r1 - r0, Tn = R + M;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t P0 = (int64_t)((__int128)Tn * wid / W), P1 = (int64_t)((__int128)Tn * (wid + 1) / W);
    if (P0 >= P1) return;
    const unsigned long long gap = (1ULL << tb) - 1ULL;
    int64_t lo = 0, hi = R;  // the last row rr with rr + off[r0 + rr] - e0 <= P0
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (mid + off[r0 + mid] - e0 <= P0) lo = mid;
        else hi = mid;
    }
    for (int64_t rb = lo; rb < R; rb += 32) {
        const int64_t rr = rb + lane;
        const bool valid = rr < R;
        const int64_t a = valid ? off[r0 + rr] - e0 : M;
        const int64_t b = valid ? (rr + 1 < R ? off[r0 + rr + 1] - e0 : M) : M;
        const int32_t d = valid ? deg[r0 + rr] : 0;
        const int64_t s0 = a > P0 - rr - 1 ? a : P0 - rr - 1;  // its slots in the range
        const int64_t t0 = b < P1 - rr - 1 ? b : P1 - rr - 1;
        unsigned todo = __ballot_sync(0xffffffffu, valid && s0 < t0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t xs = __shfl_sync(0xffffffffu, s0, src), xt = __shfl_sync(0xffffffffu, t0, src);
            const int64_t as = __shfl_sync(0xffffffffu, a, src);
            const int32_t ds = __shfl_sync(0xffffffffu, d, src);
            const unsigned long long hk = (unsigned long long)(rb + src) << tb;
            for (int64_t x = xs + lane; x < xt; x += 32) {
                key[x] = hk | (x < as + ds ? (unsigned long long)(uint32_t)idx[e0 + x] : gap);
                ord[x] = (int32_t)x;
            }
        }
        const int64_t next = rr + 1 < R ? rr + 1 + off[r0 + rr + 1] - e0 : Tn;  // the next row's position
        if (__ballot_sync(0xffffffffu, !valid || next >= P1)) break;
    }
}
__global__ void k_key_digit(const unsigned long long *key, int64_t M, int shift, int32_t *digit) {
    SGRID_STRIDE(i, M) digit[i] = (int32_t)((key[i] >> shift) & ((1u << kSortDigitBits) - 1));
}
__global__ void k_gather_key_ord(const unsigned long long *key, const int32_t *ord, const int32_t *perm, int64_t M,
                                 unsigned long long *key2, int32_t *ord2) {
    SGRID_STRIDE(i, M) {
        const int32_t p = perm[i];
        key2[i] = key[p];
        ord2[i] = ord[p];
    }
}
template <class W>
__global__ void k_gather_entries(const int32_t *ord, int64_t M, const int32_t *idx_in, const W *w_in, int32_t *idx_out,
                                 W *w_out) {
    SGRID_STRIDE(i, M) {
        const int32_t p = ord[i];
        idx_out[i] = idx_in[p];
        w_out[i] = w_in[p];
    }
}

}  // namespace

size_t sort_rows_tmp_bytes(int64_t cap) {
    const int64_t M = std::min<int64_t>(cap, kSortChunk) + 1;
    // keys x2, ord x2, digit, perm, the entries' copy (4 + 8), partition scratch
    return (size_t)M * (8 + 8 + 4 + 4 + 4 + 4 + 4 + 8) + partition_tmp_bytes(M, 1 << kSortDigitBits) + 256;
}

cudaError_t launch_sort_rows(int64_t n, const int64_t *off, const int32_t *deg, int32_t *idx, WInt *w, int64_t cap,
                             void *tmp, cudaStream_t s) {
    if (n <= 0 || cap <= 1) return cudaSuccess;
    cudaError_t e;
    // row chunks of at most kSortChunk slots (the offsets come to the host
    // only when the graph needs more than one chunk)
    std::vector<int64_t> cut = {0, n}, hoff;
    if (cap > kSortChunk) {
        hoff.resize((size_t)n + 1);
        if ((e = cudaMemcpyAsync(hoff.data(), off, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
        cut = {0};
        for (int64_t r = 0; r < n;) {
            int64_t lo = r + 1, hi = n;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (hoff[(size_t)mid] - hoff[(size_t)r] <= kSortChunk) lo = mid;
                else hi = mid - 1;
            }
            r = lo;
            cut.push_back(r);
        }
    }
    auto at = [&](int64_t r) { return hoff.empty() ? (r == 0 ? (int64_t)0 : cap) : hoff[(size_t)r]; };
    int64_t chunk_max = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k) chunk_max = std::max(chunk_max, at(cut[k + 1]) - at(cut[k]));
    if (chunk_max > kSortChunk) return cudaErrorInvalidValue;  // one row beyond 2^30 slots
    char *p = static_cast<char *>(tmp);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    const int64_t M1 = chunk_max + 1;
    auto *key = reinterpret_cast<unsigned long long *>(take(8 * M1));
    auto *key2 = reinterpret_cast<unsigned long long *>(take(8 * M1));
    auto *ord = reinterpret_cast<int32_t *>(take(4 * M1));
    auto *ord2 = reinterpret_cast<int32_t *>(take(4 * M1));
    auto *digit = reinterpret_cast<int32_t *>(take(4 * M1));
    auto *perm = reinterpret_cast<int32_t *>(take(4 * M1));
    auto *idx_copy = reinterpret_cast<int32_t *>(take(4 * M1));
    auto *w_copy = reinterpret_cast<WInt *>(take(8 * M1));
    int64_t *key_off = reinterpret_cast<int64_t *>(take(8 * ((1 << kSortDigitBits) + 2)));
    void *part_tmp = take(partition_tmp_bytes(M1, 1 << kSortDigitBits));
    int tbits = 1;  // targets are row ids of the same graph: below n <= 2^tbits - 1, the gap marker
    while ((1LL << tbits) - 1 < n) ++tbits;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        const int64_t r0 = cut[k], r1 = cut[k + 1];
        const int64_t e0 = at(r0), M = at(r1) - e0;
        if (M <= 1) continue;
        int rbits = 0;
        while ((1LL << rbits) < r1 - r0) ++rbits;
        if (rbits + tbits > 64) return cudaErrorInvalidValue;
        // warps of about 4096 merged positions each, at most one resident wave's worth of blocks per pass
        const int64_t kb = ((r1 - r0) + M + 8 * 4096 - 1) / (8 * 4096);
        k_row_keys<<<(int)(kb < 1 ? 1 : (kb > 152 * 64 ? 152 * 64 : kb)), 256, 0, s>>>(off, deg, idx, r0, r1, e0, M,
                                                                                      tbits, key, ord);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // the key's bits: targets and the gap marker, then the row
        std::vector<int> shifts;
        for (int sh = 0; sh < tbits + rbits; sh += kSortDigitBits) shifts.push_back(sh);
        unsigned long long *ck = key, *ck2 = key2;
        int32_t *co = ord, *co2 = ord2;
        for (int sh : shifts) {
            k_key_digit<<<sgrid(M), 256, 0, s>>>(ck, M, sh, digit);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = launch_partition(digit, M, 1 << kSortDigitBits, key_off, perm, part_tmp, s)) != cudaSuccess)
                return e;
            k_gather_key_ord<<<sgrid(M), 256, 0, s>>>(ck, co, perm, M, ck2, co2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            std::swap(ck, ck2);
            std::swap(co, co2);
        }
        if ((e = cudaMemcpyAsync(idx_copy, idx + e0, 4 * (size_t)M, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(w_copy, w + e0, 8 * (size_t)M, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        k_gather_entries<WInt><<<sgrid(M), 256, 0, s>>>(co, M, idx_copy, w_copy, idx + e0, w + e0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lgb
