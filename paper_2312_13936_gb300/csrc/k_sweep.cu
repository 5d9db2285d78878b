// Local-moving (Algorithm 2) and refinement (Algorithm 3) sweep kernels.
//
// One launch evaluates the vertices of one (schedule step, degree bin) list.
// For each vertex i the kernel accumulates K_{i->c} over the neighbour
// communities (scanCommunities / scanBounded), computes the Eq. 2 gain of
// every candidate, takes the best (ties: lowest community id) and compares
// it with staying. The accumulation structure depends on the degree bin:
//   bins 1-4  a tile of 4/8/16/32 lanes holds one edge per lane; equal
//             communities are merged with register shuffles;
//   bin 5     one warp per vertex with an open-addressing table in shared memory;
//   bin 6     one block per vertex with a shared-memory table;
//   bin 7     one block per vertex with a table in global memory (hubs).
// Asynchronous local-moving applies a move at once (atomics on Sigma); the
// deterministic mode and the refinement record proposals that the apply
// kernels below commit after the whole step was evaluated.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

template <class P, class W> struct SV {
    using A = typename P::acc;
    const int64_t *off;
    const int32_t *deg;
    const int32_t *idx;
    const W *w;
    int32_t *C;
    const int32_t *CB;
    const A *K;
    A *Sig;
    int32_t *size;
    uint8_t *unproc;
    int32_t *prop;
    long long *gain;
    const int32_t *step;
    A two_m;
    double gamma;
    int32_t cur_step, cap_step;
    A *dq_acc;
    unsigned long long *moved;
    int32_t *hub_keys;
    A *hub_vals;
    int hub_bits;
    int *err;
    unsigned long long *prof;
};

template <class P, class W> SV<P, W> view(const SweepCtx &c) {
    using A = typename P::acc;
    SV<P, W> a;
    a.off = c.g.off;
    a.deg = c.g.deg;
    a.idx = c.g.idx;
    a.w = static_cast<const W *>(c.g.w);
    a.C = c.C;
    a.CB = c.CB;
    a.K = static_cast<const A *>(c.K);
    a.Sig = static_cast<A *>(c.Sig);
    a.size = c.size;
    a.unproc = c.unproc;
    a.prop = c.prop;
    a.gain = c.gain;
    a.step = c.step;
    a.two_m = P::det ? (A)c.two_m_i : (A)c.two_m_f;
    a.gamma = c.gamma;
    a.cur_step = c.cur_step;
    a.cap_step = c.cap_step;
    a.dq_acc = static_cast<A *>(c.dq_acc);
    a.moved = c.moved;
    a.hub_keys = c.hub_keys;
    a.hub_vals = static_cast<A *>(c.hub_vals);
    a.hub_bits = c.hub_bits;
    a.err = c.err;
    a.prof = c.prof;
    return a;
}

// Community of neighbour j: asynchronous local-moving reads through L2 since
// other SMs move vertices concurrently; elsewhere C is constant in a launch.
template <class P, bool REFINE> __device__ __forceinline__ int32_t comm_of(const int32_t *C, int32_t j) {
    if (P::det || REFINE) return __ldg(&C[j]);
    return __ldcg(&C[j]);
}
template <class P, bool REFINE, class A> __device__ __forceinline__ A sigma_of(const A *Sig, int32_t c) {
    if (P::det || REFINE) return __ldg(&Sig[c]);
    return load_cg(&Sig[c]);
}

// Better candidate: larger key, then smaller community id.
template <class A> __device__ __forceinline__ bool better(A k1, int32_t c1, A k2, int32_t c2) {
    return k1 > k2 || (k1 == k2 && c1 < c2);
}

// Final decision for vertex v with best candidate (key, cand) and
// K_{v->d} = kvd. Run by one thread. Returns true if an asynchronous move was
// applied (its neighbours must then be marked unprocessed).
template <class P, class W, bool REFINE>
__device__ __forceinline__ bool decide(const SV<P, W> &a, int32_t v, int32_t d, typename P::acc Kv,
                                       typename P::acc key, int32_t cand, typename P::acc kvd,
                                       typename P::acc &local_gain) {
    using A = typename P::acc;
    bool mv = false;
    A g = 0;
    if (cand != INT_MAX) {
        const A sd = sigma_of<P, REFINE>(a.Sig, d);
        const A ks = stay_key(a.two_m, kvd, Kv, sd, a.gamma);
        mv = key > ks;
        if (!REFINE && mv && a.cur_step >= a.cap_step) {
            // S2: in steps that may hold adjacent vertices, a single-vertex
            // community does not move into a larger-id single-vertex one.
            const int32_t szd = P::det ? __ldg(&a.size[d]) : __ldcg(&a.size[d]);
            const int32_t szc = P::det ? __ldg(&a.size[cand]) : __ldcg(&a.size[cand]);
            if (szd == 1 && szc == 1 && cand > d) mv = false;
        }
        g = key - ks;
    }
    if (REFINE || P::det) {
        a.prop[v] = mv ? cand : -1;
        if (!REFINE && mv) a.gain[v] = (long long)g;
        return false;
    }
    if (mv) {
        atomic_add_acc(&a.Sig[d], -Kv);
        atomic_add_acc(&a.Sig[cand], Kv);
        atomicSub(&a.size[d], 1);
        atomicAdd(&a.size[cand], 1);
        a.C[v] = cand;
        local_gain += g;
    }
    return mv;
}

// Eligibility: local-moving processes unprocessed vertices (and marks them
// processed, Algorithm 2 pruning); refinement processes isolated vertices
// (the community of v has v as its only member, reading R7).
template <class P, class W, bool REFINE>
__device__ __forceinline__ bool take_vertex(const SV<P, W> &a, int32_t v, int32_t &d) {
    if (REFINE) {
        d = a.C[v];
        return __ldg(&a.size[d]) == 1;
    }
    const bool e = a.unproc[v] != 0;
    if (e) {
        a.unproc[v] = 0;
        d = a.C[v];
    }
    return e;
}

// -------------------------------------------------------------- tile bins
template <class P, class W, int T, bool REFINE>
__global__ void __launch_bounds__(256) k_eval_tile(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const unsigned tmask = (T == 32) ? kFull : (((1u << T) - 1u) << (lane & ~(T - 1)));
    const int64_t tiles = (int64_t)gridDim.x * (blockDim.x / T);
    A local_gain = 0;
    ProfCounts pc;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T; t < count; t += tiles) {
        const int32_t v = list[t];
        int32_t d = 0;
        int elig = 0;
        if (tl == 0) elig = take_vertex<P, W, REFINE>(a, v, d) ? 1 : 0;
        elig = __shfl_sync(tmask, elig, 0, T);
        d = __shfl_sync(tmask, d, 0, T);
        if (!elig) {
            if (tl == 0 && (REFINE || P::det)) a.prop[v] = -1;
            if (tl == 0) pc.v[1]++;
            continue;
        }
        const A Kv = a.K[v];
        const int64_t e0 = a.off[v];
        const int32_t dv = a.deg[v];
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int32_t j = -1, c = -1;
        A wv = 0;
        if (tl < dv) {
            j = a.idx[e0 + tl];
            wv = wconv<A>(a.w[e0 + tl]);
            bool ok = (j != v);
            if (REFINE && ok) ok = (__ldg(&a.CB[j]) == bv);
            if (ok) c = comm_of<P, REFINE>(a.C, j);
        }
        // merge equal communities: every lane sums the lanes of its community
        // in lane order; the first lane of each community leads
        A sum = 0;
        bool lead = (c >= 0);
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int32_t ck = __shfl_sync(tmask, c, k, T);
            const A wk = __shfl_sync(tmask, wv, k, T);
            if (c >= 0 && ck == c) {
                sum += wk;
                if (k < tl) lead = false;
            }
        }
        const unsigned dball = __ballot_sync(tmask, lead && c == d) & tmask;
        const int dsrc = dball ? ((__ffs(dball) - 1) & (T - 1)) : 0;
        const A kvd_b = __shfl_sync(tmask, sum, dsrc, T);
        const A kvd = dball ? kvd_b : (A)0;
        A key = AccLimits<A>::lowest();
        int32_t cand = INT_MAX;
        if (lead && c != d) {
            key = move_key(a.two_m, sum, Kv, sigma_of<P, REFINE>(a.Sig, c), a.gamma);
            cand = c;
        }
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) {
            const A ok = __shfl_xor_sync(tmask, key, o, T);
            const int32_t oc = __shfl_xor_sync(tmask, cand, o, T);
            if (better(ok, oc, key, cand)) {
                key = ok;
                cand = oc;
            }
        }
        int mv = 0;
        if (tl == 0) mv = decide<P, W, REFINE>(a, v, d, Kv, key, cand, kvd, local_gain) ? 1 : 0;
        if (a.prof) {
            const unsigned lb = __ballot_sync(tmask, lead) & tmask;
            if (tl == 0) {
                pc.v[0]++;
                pc.v[2] += dv;
                pc.v[3] += __popc(lb);
                const bool any = (REFINE || P::det) ? (a.prop[v] >= 0) : (mv != 0);
                if (any) {
                    pc.v[4]++;
                    pc.v[5] += dv;
                }
            }
        }
        if (!REFINE && !P::det) {
            mv = __shfl_sync(tmask, mv, 0, T);
            if (mv && tl < dv) a.unproc[j] = 1;  // neighbours (self-loop included) of a mover
        }
    }
    if (!REFINE && !P::det) {
        const A s = warp_sum(local_gain);
        if (lane == 0 && s != (A)0) atomic_add_acc(a.dq_acc, s);
    }
    pc.flush(a.prof);
}

// ------------------------------------------------------- warp-table bin
template <class P, class W, bool REFINE>
__global__ void __launch_bounds__(256) k_eval_warp(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    __shared__ int32_t skeys[8][kWarpSlots];
    __shared__ A svals[8][kWarpSlots];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t *keys = skeys[wib];
    A *vals = svals[wib];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    A local_gain = 0;
    ProfCounts pc;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < count; t += nwarps) {
        const int32_t v = list[t];
        int32_t d = 0;
        int elig = 0;
        if (lane == 0) elig = take_vertex<P, W, REFINE>(a, v, d) ? 1 : 0;
        elig = __shfl_sync(kFull, elig, 0);
        d = __shfl_sync(kFull, d, 0);
        if (!elig) {
            if (lane == 0 && (REFINE || P::det)) a.prop[v] = -1;
            if (lane == 0) pc.v[1]++;
            continue;
        }
        const A Kv = a.K[v];
        const int64_t e0 = a.off[v];
        const int32_t dv = a.deg[v];
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int bits = ceil_log2(2 * (int64_t)dv);
        if (bits < 6) bits = 6;
        const int S = 1 << bits;
        for (int s = lane; s < S; s += 32) {
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncwarp();
        for (int32_t e = lane; e < dv; e += 32) {
            const int32_t j = a.idx[e0 + e];
            if (j == v) continue;
            if (REFINE && __ldg(&a.CB[j]) != bv) continue;
            const int32_t c = comm_of<P, REFINE>(a.C, j);
            if (!hash_add(keys, vals, bits, c, wconv<A>(a.w[e0 + e]))) set_error(a.err, kErrHashFull);
        }
        __syncwarp();
        A key = AccLimits<A>::lowest(), kvd = 0;
        int32_t cand = INT_MAX;
        for (int s = lane; s < S; s += 32) {
            const int32_t k = keys[s];
            if (k < 0) continue;
            pc.v[3]++;
            const A sum = vals[s];
            if (k == d) {
                kvd = sum;
                continue;
            }
            const A kk = move_key(a.two_m, sum, Kv, sigma_of<P, REFINE>(a.Sig, k), a.gamma);
            if (better(kk, k, key, cand)) {
                key = kk;
                cand = k;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const A ok = __shfl_xor_sync(kFull, key, o);
            const int32_t oc = __shfl_xor_sync(kFull, cand, o);
            if (better(ok, oc, key, cand)) {
                key = ok;
                cand = oc;
            }
        }
        kvd = warp_sum(kvd);
        int mv = 0;
        if (lane == 0) {
            mv = decide<P, W, REFINE>(a, v, d, Kv, key, cand, kvd, local_gain) ? 1 : 0;
            pc.v[0]++;
            pc.v[2] += dv;
            if ((REFINE || P::det) ? (a.prop[v] >= 0) : (mv != 0)) {
                pc.v[4]++;
                pc.v[5] += dv;
            }
        }
        if (!REFINE && !P::det) {
            mv = __shfl_sync(kFull, mv, 0);
            if (mv)
                for (int32_t e = lane; e < dv; e += 32) a.unproc[a.idx[e0 + e]] = 1;
        }
        __syncwarp();
    }
    if (!REFINE && !P::det) {
        const A s = warp_sum(local_gain);
        if (lane == 0 && s != (A)0) atomic_add_acc(a.dq_acc, s);
    }
    pc.flush(a.prof);
}

// ------------------------------------------------ block / hub table bins
constexpr int kBlockThreads = 512;

template <class P, class W, bool REFINE, bool HUB>
__global__ void __launch_bounds__(kBlockThreads) k_eval_block(SV<P, W> a, const int32_t *__restrict__ list,
                                                             int64_t count) {
    using A = typename P::acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_elig, s_d, s_mv;
    __shared__ A s_key[kBlockThreads / 32], s_kvd[kBlockThreads / 32];
    __shared__ int32_t s_cand[kBlockThreads / 32];
    int32_t *keys;
    A *vals;
    if (HUB) {
        keys = a.hub_keys + ((int64_t)blockIdx.x << a.hub_bits);
        vals = a.hub_vals + ((int64_t)blockIdx.x << a.hub_bits);
    } else {
        vals = reinterpret_cast<A *>(smem_raw);
        keys = reinterpret_cast<int32_t *>(smem_raw + sizeof(A) * kBlockSlots);
    }
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    A local_gain = 0;
    ProfCounts pc;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int32_t v = list[t];
        __syncthreads();
        if (tid == 0) {
            int32_t d = 0;
            s_elig = take_vertex<P, W, REFINE>(a, v, d) ? 1 : 0;
            s_d = d;
            if (!s_elig && (REFINE || P::det)) a.prop[v] = -1;
            if (!s_elig) pc.v[1]++;
        }
        __syncthreads();
        if (!s_elig) continue;
        const int32_t d = s_d;
        const A Kv = a.K[v];
        const int64_t e0 = a.off[v];
        const int32_t dv = a.deg[v];
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int bits = ceil_log2(2 * (int64_t)dv);
        if (bits < 6) bits = 6;
        if (HUB && bits > a.hub_bits) {
            if (tid == 0) set_error(a.err, kErrHashFull);
            if (tid == 0 && (REFINE || P::det)) a.prop[v] = -1;
            continue;
        }
        const int64_t S = 1LL << bits;
        for (int64_t s = tid; s < S; s += blockDim.x) {
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncthreads();
        for (int64_t e = tid; e < dv; e += blockDim.x) {
            const int32_t j = a.idx[e0 + e];
            if (j == v) continue;
            if (REFINE && __ldg(&a.CB[j]) != bv) continue;
            const int32_t c = comm_of<P, REFINE>(a.C, j);
            if (!hash_add(keys, vals, bits, c, wconv<A>(a.w[e0 + e]))) set_error(a.err, kErrHashFull);
        }
        __syncthreads();
        A key = AccLimits<A>::lowest(), kvd = 0;
        int32_t cand = INT_MAX;
        for (int64_t s = tid; s < S; s += blockDim.x) {
            const int32_t k = keys[s];
            if (k < 0) continue;
            pc.v[3]++;
            const A sum = vals[s];
            if (k == d) {
                kvd = sum;
                continue;
            }
            const A kk = move_key(a.two_m, sum, Kv, sigma_of<P, REFINE>(a.Sig, k), a.gamma);
            if (better(kk, k, key, cand)) {
                key = kk;
                cand = k;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const A ok = __shfl_xor_sync(kFull, key, o);
            const int32_t oc = __shfl_xor_sync(kFull, cand, o);
            if (better(ok, oc, key, cand)) {
                key = ok;
                cand = oc;
            }
        }
        kvd = warp_sum(kvd);
        if (lane == 0) {
            s_key[wib] = key;
            s_cand[wib] = cand;
            s_kvd[wib] = kvd;
        }
        __syncthreads();
        if (tid == 0) {
            A bk = s_key[0], kd = s_kvd[0];
            int32_t bc = s_cand[0];
            for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2) {
                if (better(s_key[w2], s_cand[w2], bk, bc)) {
                    bk = s_key[w2];
                    bc = s_cand[w2];
                }
                kd += s_kvd[w2];
            }
            s_mv = decide<P, W, REFINE>(a, v, d, Kv, bk, bc, kd, local_gain) ? 1 : 0;
            pc.v[0]++;
            pc.v[2] += dv;
            if ((REFINE || P::det) ? (a.prop[v] >= 0) : (s_mv != 0)) {
                pc.v[4]++;
                pc.v[5] += dv;
            }
        }
        __syncthreads();
        if (!REFINE && !P::det && s_mv)
            for (int64_t e = tid; e < dv; e += blockDim.x) a.unproc[a.idx[e0 + e]] = 1;
    }
    if (!REFINE && !P::det) {
        const A s = warp_sum(local_gain);
        if (lane == 0 && s != (A)0) atomic_add_acc(a.dq_acc, s);
    }
    pc.flush(a.prof);
}

// ------------------------------------------------------------ apply steps
// Deterministic local-moving: commit the proposals of one step (all bins).
template <class P, class W>
__global__ void __launch_bounds__(256) k_move_apply(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    long long g = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[t];
        const int32_t c = a.prop[v];
        if (c < 0) continue;
        const int32_t d = a.C[v];
        const auto Kv = a.K[v];
        atomic_add_acc(&a.Sig[d], -Kv);
        atomic_add_acc(&a.Sig[c], Kv);
        atomicSub(&a.size[d], 1);
        atomicAdd(&a.size[c], 1);
        a.C[v] = c;
        g += a.gain[v];
        const int64_t e0 = a.off[v];
        const int32_t dv = a.deg[v];
        for (int32_t e = 0; e < dv; ++e) a.unproc[a.idx[e0 + e]] = 1;
    }
    g = warp_sum(g);
    if ((threadIdx.x & 31) == 0 && g != 0) atomic_add_acc(reinterpret_cast<long long *>(a.dq_acc), g);
}

// Refinement: accept proposal v -> t unless t is a single-vertex community
// whose vertex proposes in the same step; a mutual pair keeps the larger id's
// move (reading S5). Accepted vertices join t.
template <class P, class W>
__global__ void __launch_bounds__(256) k_refine_apply(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    unsigned long long mv = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[t];
        const int32_t tg = a.prop[v];
        if (tg < 0) continue;
        const int32_t pt = (a.step[tg] == a.cur_step) ? a.prop[tg] : -1;
        if (!(pt < 0 || (pt == v && v > tg))) continue;
        const auto Kv = a.K[v];
        atomic_add_acc(&a.Sig[v], -Kv);
        atomic_add_acc(&a.Sig[tg], Kv);
        atomicSub(&a.size[v], 1);
        atomicAdd(&a.size[tg], 1);
        a.C[v] = tg;
        mv++;
    }
    mv = warp_sum(mv);
    if ((threadIdx.x & 31) == 0 && mv) atomicAdd(a.moved, mv);
}

template <class P, class W, bool REFINE>
cudaError_t eval_typed(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                       cudaStream_t s) {
    SV<P, W> a = view<P, W>(c);
    auto grid = [&](int64_t per_block) {
        int64_t b = (count + per_block - 1) / per_block;
        return (int)(b < max_blocks ? (b < 1 ? 1 : b) : max_blocks);
    };
    switch (bin) {
        case 1: k_eval_tile<P, W, 4, REFINE><<<grid(64), 256, 0, s>>>(a, list, count); break;
        case 2: k_eval_tile<P, W, 8, REFINE><<<grid(32), 256, 0, s>>>(a, list, count); break;
        case 3: k_eval_tile<P, W, 16, REFINE><<<grid(16), 256, 0, s>>>(a, list, count); break;
        case 4: k_eval_tile<P, W, 32, REFINE><<<grid(8), 256, 0, s>>>(a, list, count); break;
        case 5: k_eval_warp<P, W, REFINE><<<grid(8), 256, 0, s>>>(a, list, count); break;
        case 6: {
            const size_t sm = (sizeof(typename P::acc) + sizeof(int32_t)) * kBlockSlots;
            auto kern = k_eval_block<P, W, REFINE, false>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            kern<<<grid(1), kBlockThreads, sm, s>>>(a, list, count);
            break;
        }
        case 7: k_eval_block<P, W, REFINE, true><<<grid(1), kBlockThreads, 0, s>>>(a, list, count); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class P, class W>
cudaError_t eval_mode(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks, cudaStream_t s) {
    return c.refine ? eval_typed<P, W, true>(c, bin, list, count, max_blocks, s)
                    : eval_typed<P, W, false>(c, bin, list, count, max_blocks, s);
}

int apply_grid(int64_t count) {
    int64_t b = (count + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t launch_sweep_eval(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) return eval_mode<Det, int32_t>(c, bin, list, count, max_blocks, s);
        return eval_mode<Det, float>(c, bin, list, count, max_blocks, s);
    }
    return eval_mode<Async, float>(c, bin, list, count, max_blocks, s);
}

cudaError_t launch_move_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (!c.det) return cudaErrorInvalidValue;
    if (c.g.w_int) k_move_apply<Det, int32_t><<<apply_grid(count), 256, 0, s>>>(view<Det, int32_t>(c), list, count);
    else k_move_apply<Det, float><<<apply_grid(count), 256, 0, s>>>(view<Det, float>(c), list, count);
    return cudaGetLastError();
}

cudaError_t launch_refine_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) k_refine_apply<Det, int32_t><<<apply_grid(count), 256, 0, s>>>(view<Det, int32_t>(c), list, count);
        else k_refine_apply<Det, float><<<apply_grid(count), 256, 0, s>>>(view<Det, float>(c), list, count);
    } else {
        k_refine_apply<Async, float><<<apply_grid(count), 256, 0, s>>>(view<Async, float>(c), list, count);
    }
    return cudaGetLastError();
}

}  // namespace lgb
