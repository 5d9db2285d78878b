// Aggregation (Algorithm 4): for every community c of the renumbered refined
// membership, accumulate H[C'[j]] += w over all edges (self-loops included)
// of all member vertices and write the merged (d, w) pairs as row c of the
// super-vertex graph G'' (a holey CSR whose row capacity is the community's
// total degree). The row sum is K''[c]. Communities are binned by total
// degree like the sweep kernels: a tile of lanes (<= 32 member edges), one
// warp with a shared-memory table (<= 256), one block with a shared-memory
// table (<= 4096), one block with a global-memory table (larger).
// Row order inside G'' is unspecified; deterministic mode writes exact
// integer sums, so the rows are equal as sets.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

template <class P, class Wi, class Wo> struct AV {
    using A = typename P::acc;
    const int64_t *off;
    const int32_t *deg;
    const int32_t *idx;
    const Wi *w;
    const int32_t *Cd;
    const int64_t *coff;
    const int32_t *members;
    const int64_t *out_off;
    int32_t *out_deg;
    int32_t *out_idx;
    Wo *out_w;
    A *out_K;
    int32_t *hub_keys;
    A *hub_vals;
    const int64_t *tab_off;
    const int32_t *tab_idx;
    int64_t tab_k0, tab_k1, tab_base;
    int64_t ncomm;
    int *err;
    unsigned long long *prof;
};

template <class P, class Wi, class Wo> AV<P, Wi, Wo> aview(const AggCtx &c) {
    using A = typename P::acc;
    AV<P, Wi, Wo> a;
    a.off = c.g.off;
    a.deg = c.g.deg;
    a.idx = c.g.idx;
    a.w = static_cast<const Wi *>(c.g.w);
    a.Cd = c.Cd;
    a.coff = c.coff;
    a.members = c.members;
    a.out_off = c.out_off;
    a.out_deg = c.out_deg;
    a.out_idx = c.out_idx;
    a.out_w = static_cast<Wo *>(c.out_w);
    a.out_K = static_cast<A *>(c.out_K);
    a.hub_keys = c.hub_keys;
    a.hub_vals = static_cast<A *>(c.hub_vals);
    a.tab_off = c.tab_off;
    a.tab_idx = c.tab_idx;
    a.tab_k0 = c.tab_k0;
    a.tab_k1 = c.tab_k1;
    a.tab_base = c.tab_base;
    a.ncomm = c.ncomm;
    a.err = c.err;
    a.prof = c.prof;
    return a;
}

// stored weight of a merged entry, and its value as the next pass sees it
template <class Wo, class A> __device__ __forceinline__ Wo out_weight(A s) { return (Wo)s; }

// ------------------------------------------------------------- tile bins
template <class P, class Wi, class Wo, int T>
__global__ void __launch_bounds__(256) k_agg_tile(AV<P, Wi, Wo> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int base_lane = lane & ~(T - 1);
    const unsigned tmask = (T == 32) ? kFull : (((1u << T) - 1u) << base_lane);
    const int64_t tiles = (int64_t)gridDim.x * (blockDim.x / T);
    ProfCounts pc;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T; t < count; t += tiles) {
        const int32_t c = list[t];
        const int64_t m0 = a.coff[c];
        const int32_t nm = (int32_t)(a.coff[c + 1] - m0);
        // member of this lane and its edge range
        int32_t du = 0;
        int64_t su = 0;
        if (tl < nm) {
            const int32_t u = a.members[m0 + tl];
            du = a.deg[u];
            su = a.off[u];
        }
        int32_t incl = du;
#pragma unroll
        for (int o = 1; o < T; o <<= 1) {
            const int32_t x = __shfl_up_sync(tmask, incl, o, T);
            if (tl >= o) incl += x;
        }
        const int32_t excl = incl - du;
        const int32_t total = __shfl_sync(tmask, incl, T - 1, T);
        // the lane whose member owns edge slot tl
        int owner = 0;
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int32_t ek = __shfl_sync(tmask, excl, k, T);
            const int32_t ik = __shfl_sync(tmask, incl, k, T);
            if (tl >= ek && tl < ik) owner = k;
        }
        const int64_t s_own = __shfl_sync(tmask, su, owner, T);
        const int32_t e_own = __shfl_sync(tmask, excl, owner, T);
        int32_t key = -1;
        A wv = 0;
        if (tl < total) {
            const int64_t e = s_own + (tl - e_own);
            key = a.Cd[a.idx[e]];
            wv = wconv<A>(a.w[e]);
        }
        A sum = 0;
        bool lead = (key >= 0);
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int32_t kk = __shfl_sync(tmask, key, k, T);
            const A wk = __shfl_sync(tmask, wv, k, T);
            if (key >= 0 && kk == key) {
                sum += wk;
                if (k < tl) lead = false;
            }
        }
        const unsigned ball = (__ballot_sync(tmask, lead) & tmask) >> base_lane;
        const int pos = __popc(ball & ((1u << tl) - 1u));
        const int64_t o0 = a.out_off[c];
        A kpart = 0;
        if (lead) {
            const Wo wo = out_weight<Wo>(sum);
            a.out_idx[o0 + pos] = key;
            a.out_w[o0 + pos] = wo;
            kpart = wconv<A>(wo);
        }
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) kpart += __shfl_xor_sync(tmask, kpart, o, T);
        if (tl == 0) {
            a.out_deg[c] = __popc(ball);
            a.out_K[c] = kpart;
            pc.v[0]++;
            pc.v[1] += nm;
            pc.v[2] += total;
            pc.v[3] += __popc(ball);
        }
    }
    pc.flush(a.prof);
}

// insert all member edges of community c into a table (threads of a warp
// take members round-robin; used by the warp bin)
template <class P, class Wi, class Wo>
__device__ __forceinline__ void fill_members_lanes(const AV<P, Wi, Wo> &a, int64_t m0, int32_t nm, int32_t *keys,
                                                   typename P::acc *vals, int bits, int lane) {
    using A = typename P::acc;
    for (int32_t k = lane; k < nm; k += 32) {
        const int32_t u = a.members[m0 + k];
        const int64_t e0 = a.off[u];
        const int32_t du = a.deg[u];
        for (int32_t e = 0; e < du; ++e)
            if (!hash_add(keys, vals, bits, a.Cd[a.idx[e0 + e]], wconv<A>(a.w[e0 + e]))) set_error(a.err, kErrHashFull);
    }
}

// ------------------------------------------------------- warp-table bin
template <class P, class Wi, class Wo>
__global__ void __launch_bounds__(256) k_agg_warp(AV<P, Wi, Wo> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    __shared__ int32_t skeys[8][kWarpSlots];
    __shared__ A svals[8][kWarpSlots];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *keys = skeys[wib];
    A *vals = svals[wib];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    ProfCounts pc;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < count; t += nwarps) {
        const int32_t c = list[t];
        const int64_t m0 = a.coff[c];
        const int32_t nm = (int32_t)(a.coff[c + 1] - m0);
        const int64_t cap = a.out_off[c + 1] - a.out_off[c];
        int bits = ceil_log2(2 * cap);
        if (bits < 6) bits = 6;
        const int S = 1 << bits;
        for (int s = lane; s < S; s += 32) {
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncwarp();
        fill_members_lanes(a, m0, nm, keys, vals, bits, lane);
        __syncwarp();
        const int64_t o0 = a.out_off[c];
        int written = 0;
        A kpart = 0;
        for (int s0 = 0; s0 < S; s0 += 32) {
            const int s = s0 + lane;
            const int32_t k = keys[s];
            const unsigned ball = __ballot_sync(kFull, k >= 0);
            if (k >= 0) {
                const int pos = written + __popc(ball & ((1u << lane) - 1u));
                const Wo wo = out_weight<Wo>(vals[s]);
                a.out_idx[o0 + pos] = k;
                a.out_w[o0 + pos] = wo;
                kpart += wconv<A>(wo);
            }
            written += __popc(ball);
        }
        kpart = warp_sum(kpart);
        if (lane == 0) {
            a.out_deg[c] = written;
            a.out_K[c] = kpart;
            pc.v[0]++;
            pc.v[1] += nm;
            pc.v[2] += cap;
            pc.v[3] += written;
        }
        __syncwarp();
    }
    pc.flush(a.prof);
}

// ------------------------------------------------------ block table bin
constexpr int kAggThreads = 512;
static_assert(4 * kAggThreads >= kBlockMaxDeg, "the block kernel's threads hold four members each");
// shared memory of the block kernel: the table, then the members' entry
// prefix (nm + 1 int32) and row starts (nm int64)
template <class A> constexpr size_t block_smem_bytes() {
    return (sizeof(A) + sizeof(int32_t)) * kBlockSlots + sizeof(int64_t) * kBlockMaxDeg +
           sizeof(int32_t) * (kBlockMaxDeg + 2);
}

// One block per community. Its members' entries are taken as one flat
// range: the members' row starts and the prefix sums of their degrees go to
// shared memory, then the warps take 32 consecutive entries at a time
// across member boundaries (each lane finds its member by binary search
// over the prefix), so every lane has an entry and the loads of different
// chunks overlap. Every member of a community with an edge has one, so a
// community has at most as many members as entries (bin 5: at most
// kBlockMaxDeg); a larger member count takes the members one per warp.
template <class P, class Wi, class Wo>
__global__ void __launch_bounds__(kAggThreads) k_agg_block(AV<P, Wi, Wo> a, const int32_t *__restrict__ list,
                                                          int64_t count) {
    using A = typename P::acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_written;
    __shared__ A s_k[kAggThreads / 32];
    __shared__ int32_t s_part[kAggThreads / 32];
    A *vals = reinterpret_cast<A *>(smem_raw);
    int64_t *mrow = reinterpret_cast<int64_t *>(smem_raw + sizeof(A) * kBlockSlots);
    int32_t *keys = reinterpret_cast<int32_t *>(smem_raw + sizeof(A) * kBlockSlots + sizeof(int64_t) * kBlockMaxDeg);
    int32_t *pre = keys + kBlockSlots;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nw = blockDim.x >> 5;
    ProfCounts pc;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int32_t c = list[t];
        const int64_t m0 = a.coff[c];
        const int32_t nm = (int32_t)(a.coff[c + 1] - m0);
        int64_t cap = a.out_off[c + 1] - a.out_off[c];
        if (cap > a.ncomm) cap = a.ncomm;  // distinct targets <= number of communities
        int bits = ceil_log2(2 * cap);
        if (bits < 6) bits = 6;
        __syncthreads();
        const int64_t S = 1LL << bits;
        for (int64_t s = tid; s < S; s += blockDim.x) {
            keys[s] = -1;
            vals[s] = 0;
        }
        if (tid == 0) s_written = 0;
        if (nm <= kBlockMaxDeg) {
            // members' row starts and the exclusive prefix of their degrees:
            // thread tid holds members [4 tid, 4 tid + 4)
            int32_t d4[4], sum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t k = 4 * tid + q;
                d4[q] = 0;
                if (k < nm) {
                    const int32_t u = a.members[m0 + k];
                    mrow[k] = a.off[u];
                    d4[q] = a.deg[u];
                }
                sum += d4[q];
            }
            int32_t inc = sum;  // inclusive scan of the threads' sums: warps, then the warp totals
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_part[wib] = inc;
            __syncthreads();
            int32_t before = 0;
            for (int w2 = 0; w2 < wib; ++w2) before += s_part[w2];
            int32_t run = before + inc - sum;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t k = 4 * tid + q;
                if (k < nm) pre[k] = run;
                run += d4[q];
                if (k == nm - 1) pre[nm] = run;
            }
            if (nm == 0 && tid == 0) pre[0] = 0;
            __syncthreads();
            const int32_t T = pre[nm];
            for (int32_t x0 = wib * 32; x0 < T; x0 += nw * 32) {
                const int32_t x = x0 + lane;
                if (x < T) {
                    int32_t lo = 0, hi = nm - 1;  // the last member k with pre[k] <= x
                    while (lo < hi) {
                        const int32_t mid = (lo + hi + 1) >> 1;
                        if (pre[mid] <= x) lo = mid;
                        else hi = mid - 1;
                    }
                    const int64_t e = mrow[lo] + (x - pre[lo]);
                    if (!hash_add(keys, vals, bits, a.Cd[a.idx[e]], wconv<A>(a.w[e]))) set_error(a.err, kErrHashFull);
                }
            }
        } else {
            __syncthreads();
            // warps take members round-robin, lanes stride over a member's edges
            for (int32_t k = wib; k < nm; k += nw) {
                const int32_t u = a.members[m0 + k];
                const int64_t e0 = a.off[u];
                const int32_t du = a.deg[u];
                for (int32_t e = lane; e < du; e += 32)
                    if (!hash_add(keys, vals, bits, a.Cd[a.idx[e0 + e]], wconv<A>(a.w[e0 + e])))
                        set_error(a.err, kErrHashFull);
            }
        }
        __syncthreads();
        const int64_t o0 = a.out_off[c];
        A kpart = 0;
        for (int64_t s0 = (int64_t)wib * 32; s0 < S; s0 += (int64_t)nw * 32) {
            const int64_t s = s0 + lane;
            const int32_t k = keys[s];
            const unsigned ball = __ballot_sync(kFull, k >= 0);
            int base = 0;
            if (lane == 0 && ball) base = atomicAdd(&s_written, __popc(ball));
            base = __shfl_sync(kFull, base, 0);
            if (k >= 0) {
                const int pos = base + __popc(ball & ((1u << lane) - 1u));
                const Wo wo = out_weight<Wo>(vals[s]);
                a.out_idx[o0 + pos] = k;
                a.out_w[o0 + pos] = wo;
                kpart += wconv<A>(wo);
            }
        }
        kpart = warp_sum(kpart);
        if (lane == 0) s_k[wib] = kpart;
        __syncthreads();
        if (tid == 0) {
            A ks = 0;
            for (int w2 = 0; w2 < nw; ++w2) ks += s_k[w2];
            a.out_deg[c] = s_written;
            a.out_K[c] = ks;
            pc.v[0]++;
            pc.v[1] += nm;
            pc.v[2] += a.out_off[c + 1] - a.out_off[c];
            pc.v[3] += s_written;
        }
    }
    pc.flush(a.prof);
}

// ------------------------------------------------- bin 6: packed tables
// tab_size[k] = 2^max(6, ceil log2 2 min(tdeg, ncomm)) of community list[k]
// (its distinct targets are at most that many), tab_idx[c] = k, the member
// count tab_nm[k], and out_K[c] = 0 (the write adds into it)
template <class A>
__global__ void k_tab_sizes(const int32_t *list, int64_t count, const int64_t *tdeg, const int64_t *coff,
                            int64_t ncomm, int64_t *tab_size, int32_t *tab_idx, int64_t *tab_nm, A *out_K) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = list[k];
        const int64_t cap = tdeg[c] < ncomm ? tdeg[c] : ncomm;  // distinct targets
        int bits = ceil_log2(2 * cap);
        if (bits < 6) bits = 6;
        tab_size[k] = 1LL << bits;
        tab_idx[c] = (int32_t)k;
        tab_nm[k] = coff[c + 1] - coff[c];
        out_K[c] = 0;
    }
}

// The members of the bin-6 communities as one flat list in table order
// (member t of table k at moff[k] + t): its vertex fm[t], its table ft[t]
// and its degree fd[t] (the row lengths whose scan makes the flat entry
// range of the insertion). Every member of such a community has an edge.
__global__ void k_tab_members(const int32_t *list, int64_t K6, const int64_t *moff, const int64_t *coff,
                              const int32_t *members, const int32_t *deg, int32_t *fm, int32_t *ft, int32_t *fd) {
    const int64_t M6 = moff[K6];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < M6; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = K6 - 1;  // the last table k with moff[k] <= t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (moff[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int32_t u = members[coff[list[lo]] + (t - moff[lo])];
        fm[t] = u;
        ft[t] = (int32_t)lo;
        fd[t] = deg[u];
    }
}

// Insertion of tables [tab_k0, tab_k1): their members' entries form the
// flat range [eoff[moff[k0]], eoff[moff[k1]]) (eoff: the scan of the flat
// members' degrees), cut into chunks of 32 consecutive entries, so rows of
// any length spread over all warps; each warp takes a contiguous run of
// chunks. Lane 0 finds the member of the warp's first entry by binary
// search; 32 entries span at most 32 members (every member has an edge),
// whose ends the lanes hold, and each lane finds its own by a search over
// them; the next chunk starts at the member after the ones that ended. Entries
// of one chunk with the same (table, key) are summed first and inserted
// once, which keeps hot keys (a large community's own entries) from
// serialising on one address. Members come in community order, so a warp's
// run shares a few tables.
template <class P, class Wi, class Wo>
__global__ void __launch_bounds__(256) k_agg_tab_insert(AV<P, Wi, Wo> a, const int32_t *__restrict__ fm,
                                                        const int32_t *__restrict__ ft, const int64_t *__restrict__ eoff,
                                                        const int64_t *__restrict__ moff) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int64_t mlo = moff[a.tab_k0], mhi = moff[a.tab_k1];
    const int64_t x_begin = eoff[mlo], x_end = eoff[mhi];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nch = (x_end - x_begin + 31) / 32;
    const int64_t c0 = nch * wid / warps, c1 = nch * (wid + 1) / warps;
    ProfCounts pc;
    int64_t m0 = 0;
    if (c0 < c1 && lane == 0) {
        const int64_t x0 = x_begin + c0 * 32;
        int64_t lo = mlo, hi = mhi - 1;  // the last member with eoff[m] <= x0
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (eoff[mid] <= x0) lo = mid;
            else hi = mid - 1;
        }
        m0 = lo;
    }
    m0 = __shfl_sync(kFull, m0, 0);
    for (int64_t x0 = x_begin + c0 * 32; x0 < x_begin + c1 * 32; x0 += 32) {
        const int64_t mine = m0 + lane < mhi ? eoff[m0 + lane + 1] : INT64_MAX;  // end of member m0 + lane
        const int64_t x = x0 + lane;
        int own = 0;  // members before x's: lanes whose member ends at or before x
        for (int st = 16; st >= 1; st >>= 1)
            if (__shfl_sync(kFull, mine, own + st - 1) <= x) own += st;
        own &= 31;
        const bool valid = x < x_end;
        int32_t key = -1, tk = -1;
        int64_t tb = 0;
        int tbits = 0;
        A v = 0;
        if (valid) {
            const int64_t m = m0 + own;
            const int32_t u = fm[m];
            const int64_t e = a.off[u] + (x - eoff[m]);
            tk = ft[m];
            tb = a.tab_off[tk] - a.tab_base;
            tbits = __ffsll((long long)(a.tab_off[tk + 1] - a.tab_off[tk])) - 1;
            key = a.Cd[a.idx[e]];
            v = wconv<A>(a.w[e]);
            if (a.prof) {
                pc.v[2]++;
                if (x == eoff[m]) pc.v[1]++;
            }
        }
        const unsigned long long pair = valid ? ((unsigned long long)(uint32_t)tk << 32) | (uint32_t)key : ~0ull;
        const unsigned peers = __match_any_sync(kFull, pair);
        v = peer_sum(peers, v);
        if (valid && lane == __ffs(peers) - 1) {
            bool ok;
            if constexpr (P::det) ok = hash_add(a.hub_keys + tb, a.hub_vals + tb, tbits, key, v);
            else ok = hash_add_kv(reinterpret_cast<unsigned long long *>(a.hub_vals) + tb, tbits, key, v);
            if (!ok) set_error(a.err, kErrHashFull);
        }
        m0 += __popc(__ballot_sync(kFull, mine <= x0 + 32));  // the member of the next chunk's first entry
    }
    pc.flush(a.prof);
}

// The distinct entries of tables [tab_k0, tab_k1) become their communities'
// rows (order unspecified: the slots go in chunks of 32 -- tables are at
// least 64 slots and start at multiples of 64, so a chunk lies in one table
// -- each warp takes a contiguous run of chunks and appends each chunk's
// entries at its row's running fill), out_deg[c] their count and K''[c]
// their sum (both start at 0).
template <class P, class Wi, class Wo>
__global__ void __launch_bounds__(256) k_agg_tab_write(AV<P, Wi, Wo> a, const int32_t *__restrict__ list) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int64_t s_begin = a.tab_off[a.tab_k0], s_end = a.tab_off[a.tab_k1];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nch = (s_end - s_begin) / 32;
    const int64_t c0 = nch * wid / warps, c1 = nch * (wid + 1) / warps;
    ProfCounts pc;
    int64_t k = 0;
    if (c0 < c1 && lane == 0) {
        const int64_t s0 = s_begin + c0 * 32;
        int64_t lo = a.tab_k0, hi = a.tab_k1 - 1;  // the table holding slot s0
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (a.tab_off[mid] <= s0) lo = mid;
            else hi = mid - 1;
        }
        k = lo;
    }
    k = __shfl_sync(kFull, k, 0);
    for (int64_t s0 = s_begin + c0 * 32; s0 < s_begin + c1 * 32; s0 += 32) {
        while (a.tab_off[k + 1] <= s0) ++k;  // the same on every lane
        const int32_t c = list[k];
        const int64_t sl = s0 + lane - a.tab_base;
        int32_t key;
        A val;
        if constexpr (P::det) {
            key = a.hub_keys[sl];
            val = key >= 0 ? a.hub_vals[sl] : (A)0;
        } else {  // key and fp32 value in one word
            const unsigned long long kv = reinterpret_cast<const unsigned long long *>(a.hub_vals)[sl];
            key = (int32_t)(uint32_t)kv;
            val = (A)__uint_as_float((uint32_t)(kv >> 32));
        }
        const unsigned ball = __ballot_sync(kFull, key >= 0);
        if (!ball) continue;
        int pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(&a.out_deg[c], __popc(ball));
        pos0 = __shfl_sync(kFull, pos0, 0);
        A part = 0;
        if (key >= 0) {
            const int64_t o = a.out_off[c] + pos0 + __popc(ball & ((1u << lane) - 1u));
            const Wo wo = out_weight<Wo>(val);
            a.out_idx[o] = key;
            a.out_w[o] = wo;
            part = wconv<A>(wo);
        }
        part = warp_sum(part);
        if (lane == 0) {
            atomic_add_acc(&a.out_K[c], part);
            pc.v[3] += __popc(ball);
            if (s0 == a.tab_off[k]) pc.v[0]++;
        }
    }
    pc.flush(a.prof);
}

template <class P, class Wi, class Wo>
cudaError_t tables_typed(const AggCtx &c, const int32_t *list, int sms, cudaStream_t s) {
    auto a = aview<P, Wi, Wo>(c);
    // one wave: as many blocks as are resident at once (the warps take
    // equal runs of chunks, so a second wave would leave a tail)
    static int bi = 0, bw = 0;
    if (!bi && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, k_agg_tab_insert<P, Wi, Wo>, 256, 0) != cudaSuccess)
        bi = 0;
    if (!bw && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, k_agg_tab_write<P, Wi, Wo>, 256, 0) != cudaSuccess)
        bw = 0;
    k_agg_tab_insert<P, Wi, Wo><<<sms * (bi > 0 ? bi : 4), 256, 0, s>>>(a, c.fm, c.ft, c.eoff, c.moff);
    k_agg_tab_write<P, Wi, Wo><<<sms * (bw > 0 ? bw : 4), 256, 0, s>>>(a, list);
    return cudaGetLastError();
}

template <class P, class Wi, class Wo>
cudaError_t agg_typed(const AggCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks, cudaStream_t s) {
    auto a = aview<P, Wi, Wo>(c);
    auto grid = [&](int64_t per_block) {
        int64_t b = (count + per_block - 1) / per_block;
        return (int)(b < max_blocks ? (b < 1 ? 1 : b) : max_blocks);
    };
    switch (bin) {
        case 1: k_agg_tile<P, Wi, Wo, 8><<<grid(32), 256, 0, s>>>(a, list, count); break;
        case 2: k_agg_tile<P, Wi, Wo, 16><<<grid(16), 256, 0, s>>>(a, list, count); break;
        case 3: k_agg_tile<P, Wi, Wo, 32><<<grid(8), 256, 0, s>>>(a, list, count); break;
        case 4: k_agg_warp<P, Wi, Wo><<<grid(8), 256, 0, s>>>(a, list, count); break;
        case 5: {
            const size_t sm = block_smem_bytes<typename P::acc>();
            auto kern = k_agg_block<P, Wi, Wo>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            kern<<<grid(1), kAggThreads, sm, s>>>(a, list, count);
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_table_sizes(const int32_t *list, int64_t count, const int64_t *tdeg, const int64_t *coff,
                               int64_t ncomm, bool det, int64_t *tab_size, int32_t *tab_idx, int64_t *tab_nm,
                               void *out_K, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t b = (count + 255) / 256;
    const int g = (int)(b < 2432 ? b : 2432);
    if (det)
        k_tab_sizes<long long><<<g, 256, 0, s>>>(list, count, tdeg, coff, ncomm, tab_size, tab_idx, tab_nm,
                                                 static_cast<long long *>(out_K));
    else
        k_tab_sizes<float><<<g, 256, 0, s>>>(list, count, tdeg, coff, ncomm, tab_size, tab_idx, tab_nm,
                                             static_cast<float *>(out_K));
    return cudaGetLastError();
}

cudaError_t launch_table_members(const int32_t *list, int64_t K6, const int64_t *moff, int64_t M6, const int64_t *coff,
                                 const int32_t *members, const int32_t *deg, int32_t *fm, int32_t *ft, int32_t *fd,
                                 cudaStream_t s) {
    if (K6 <= 0 || M6 <= 0) return cudaSuccess;
    const int64_t b = (M6 + 255) / 256;
    k_tab_members<<<(int)(b < 2432 ? b : 2432), 256, 0, s>>>(list, K6, moff, coff, members, deg, fm, ft, fd);
    return cudaGetLastError();
}

cudaError_t launch_aggregate_tables(const AggCtx &c, const int32_t *list, int sms, cudaStream_t s) {
    if (c.tab_k1 <= c.tab_k0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) return tables_typed<Det, WInt, WInt>(c, list, sms, s);
        return tables_typed<Det, float, WInt>(c, list, sms, s);
    }
    return tables_typed<Async, float, float>(c, list, sms, s);
}

cudaError_t launch_aggregate(const AggCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) return agg_typed<Det, WInt, WInt>(c, bin, list, count, max_blocks, s);
        return agg_typed<Det, float, WInt>(c, bin, list, count, max_blocks, s);
    }
    return agg_typed<Async, float, float>(c, bin, list, count, max_blocks, s);
}

}  // namespace lgb
