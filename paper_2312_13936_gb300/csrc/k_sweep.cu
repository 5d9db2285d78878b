// Local-moving (Algorithm 2) and refinement (Algorithm 3) sweeps.
//
// For each vertex i the kernels accumulate K_{i->c} over the neighbour
// communities (scanCommunities / scanBounded), compute the Eq. 2 gain of
// every candidate, take the best (ties: lowest community id) and compare it
// with staying. The accumulation structure depends on the degree bin:
//   bin 1     one thread per vertex, up to 8 edges in registers, merged by
//             pairwise comparison (32 vertices per warp, 8 loads in flight each);
//   bins 2-3  a tile of 16/32 lanes holds one edge per lane; equal
//             communities are merged with register shuffles;
//   bin 4     one warp per vertex, open-addressing table in shared memory;
//   bin 5     one block per vertex, shared-memory table;
//   bin 6     one block per vertex, table in global memory (hubs).
//
// A sweep visits the schedule steps in order (reading S0). The main kernel,
// k_sweep_coop, is persistent: one cooperative launch runs every step of a
// sweep and separates steps with a grid barrier, so a sweep costs one launch
// whatever the number of steps. Asynchronous local-moving applies each move
// at once below the capped step (atomics on Sigma, the paper's asynchronous
// execution) and records proposals in the capped steps, where neighbours
// share a step; the deterministic mode records proposals in every step. An
// apply phase after the step's evaluation commits them; the refinement's
// proposals are accepted by reading S5. The per-(step, bin) kernels
// below run the same routines one launch at a time; the engine uses them if
// a cooperative launch is not possible.
//
// State that changes during a sweep (C, Sigma, sizes, flags, proposals) is
// read through L2 (ld.global.cg) so that a step sees every write made before
// the preceding barrier.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace lgb {
namespace {

template <class P, class W> struct SV {
    using A = typename P::acc;
    using T = typename P::tot;
    const int64_t *off;
    const int32_t *deg;
    const int32_t *idx;
    const W *w;
    int32_t *C;
    const int32_t *CB;
    const A *K;
    T *Sig;
    int32_t *size;
    uint8_t *unproc;
    int32_t *prop;
    long long *gain;
    const int32_t *step;
    const int64_t *loff;  // rows and weights in list order (null: by vertex)
    const int32_t *lidx;
    const W *lw;
    const A *lK;
    A kscale;       // 2m (deterministic) or 1/2m (asynchronous), see move_key
    double two_m_d;
    double gamma;
    int32_t cur_step, cap_step, nsteps;
    const int64_t *key_off;
    int32_t max_it, single_sweep;
    double tau;
    T *dq_arr;                     // per-sweep gain sums (persistent phase)
    unsigned long long *moved_arr; // per-sweep refinement moves (persistent phase)
    int32_t *iters_out;
    T *dq_acc;
    unsigned long long *moved;
    int32_t *hub_keys;
    A *hub_vals;
    int hub_bits, hub_regions;
    // bin 6 on the whole grid (persistent sweep)
    const int32_t *hubs;
    int32_t *hj;
    int64_t *htoff, *heoff, *hinfo;
    int32_t *hd, *hcand, *hmv;
    unsigned long long *hkey;
    A *hkvd;
    bool grid_hubs;
    unsigned *bar;
    int *err;
    unsigned long long *prof;
    int32_t block_max;              // rows longer than this are bin 6 (the hubs)
    int32_t stall_block;            // testing aid: this block never arrives at a barrier
    unsigned long long spin_limit;  // barrier polls before giving up
    // persistent sweep: act[k] == it + 1 marks step k as holding an eligible
    // vertex in sweep it (steps without one are skipped); null elsewhere
    int32_t *act;
    // randomized refinement (asynchronous mode): draws from SplitMix64 with
    // state rseed + 0xD1B54A32D192ED03 * (sweep + 1); sweep: the sweep of a
    // per-step launch
    bool rand_refine;
    uint64_t rseed;
    int32_t sweep;
    // batch of graphs (gid == null: one graph)
    const int32_t *gid;
    const A *gks;
    const double *g2m;
    int32_t *gdone;
    int32_t *giters;
    unsigned *gactive;
    const double *gtau;
    int32_t G;
};

// The row and weight of the vertex v at list position t: from the copy in
// list order when the pass made one (a step's rows then lie together), else
// from the vertex's own row.
template <class W> struct RowOf {
    int64_t e0;
    int32_t dv;
    const int32_t *idx;
    const W *w;
};
template <class P, class W> __device__ __forceinline__ RowOf<W> row_of(const SV<P, W> &a, int32_t v, int64_t t) {
    if (a.loff) {
        const int64_t e0 = a.loff[t];
        return {e0, (int32_t)(a.loff[t + 1] - e0), a.lidx, a.lw};
    }
    return {a.off[v], a.deg[v], a.idx, a.w};
}
template <class P, class W> __device__ __forceinline__ typename P::acc k_of(const SV<P, W> &a, int32_t v, int64_t t) {
    return a.lK ? a.lK[t] : a.K[v];
}

// A thread's sweep sums: gains or joins (asynchronous), applied gains
// (deterministic local-moving), applied proposals (refinement), and this
// sweep's per-graph slots they go to.
template <class P> struct Sums {
    GAcc<typename P::acc> gain;
    GAcc<unsigned __int128> dgain;  // deterministic gains (dq: two words per slot)
    GAcc<unsigned long long> moved;
    typename P::tot *dq;
    unsigned long long *mv;
    int32_t stamp = 0;  // this sweep's mark in act (persistent sweep)
};

template <class P, class W> SV<P, W> view(const SweepCtx &c) {
    using A = typename P::acc;
    using T = typename P::tot;
    SV<P, W> a;
    a.off = c.g.off;
    a.deg = c.g.deg;
    a.idx = c.g.idx;
    a.w = static_cast<const W *>(c.g.w);
    a.C = c.C;
    a.CB = c.CB;
    a.K = static_cast<const A *>(c.K);
    a.Sig = static_cast<T *>(c.Sig);
    a.size = c.size;
    a.unproc = c.unproc;
    a.prop = c.prop;
    a.gain = c.gain;
    a.step = c.step;
    a.loff = c.loff;
    a.lidx = c.lidx;
    a.lw = static_cast<const W *>(c.lw);
    a.lK = static_cast<const A *>(c.lK);
    a.kscale = P::det ? (A)c.two_m_i : (A)(1.0 / c.two_m_f);
    a.two_m_d = P::det ? (double)c.two_m_i : c.two_m_f;
    a.gamma = c.gamma;
    a.cur_step = c.cur_step;
    a.cap_step = c.cap_step;
    a.nsteps = c.nsteps;
    a.key_off = c.key_off;
    a.max_it = c.max_it;
    a.single_sweep = c.single_sweep;
    a.tau = c.tau;
    a.dq_arr = static_cast<T *>(c.dq_arr);
    a.moved_arr = c.moved_arr;
    a.iters_out = c.iters_out;
    a.dq_acc = static_cast<T *>(c.dq_acc);
    a.moved = c.moved;
    a.hub_keys = c.hub_keys;
    a.hub_vals = static_cast<A *>(c.hub_vals);
    a.hub_bits = c.hub_bits;
    a.hub_regions = c.hub_regions;
    a.hubs = c.hubs;
    a.hj = c.hj;
    a.htoff = c.htoff;
    a.heoff = c.heoff;
    a.hinfo = c.hinfo;
    a.hd = c.hd;
    a.hcand = c.hcand;
    a.hmv = c.hmv;
    a.hkey = c.hkey;
    a.hkvd = static_cast<A *>(c.hkvd);
    a.grid_hubs = c.grid_hubs;
    a.bar = c.bar;
    a.err = c.err;
    a.prof = c.prof;
    a.block_max = c.block_max;
    a.stall_block = c.stall_block;
    a.spin_limit = c.spin_limit;
    a.act = c.act;
    a.rand_refine = c.rand_refine;
    a.rseed = c.rseed;
    a.sweep = c.sweep;
    a.gid = c.gid;
    a.gks = static_cast<const A *>(c.gks);
    a.g2m = c.g2m;
    a.gdone = c.gdone;
    a.giters = c.giters;
    a.gactive = c.gactive;
    a.gtau = c.gtau;
    a.G = c.G;
    return a;
}

__device__ __forceinline__ int32_t ldm(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ double ldm(const double *p) { return __ldcg(p); }
__device__ __forceinline__ long long ldm(const long long *p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldm(const uint8_t *p) { return __ldcg(p); }

// Better candidate: larger key, then smaller community id.
template <class A> __device__ __forceinline__ bool better(A k1, int32_t c1, A k2, int32_t c2) {
    return k1 > k2 || (k1 == k2 && c1 < c2);
}

// graph of vertex v and its key scale
// (B: the kernel serves a batch of graphs; the single-graph instantiations
// carry no per-graph code)
template <bool B, class P, class W> __device__ __forceinline__ int32_t graph_of(const SV<P, W> &a, int32_t v) {
    return B ? __ldg(&a.gid[v]) : 0;
}
template <bool B, class P, class W>
__device__ __forceinline__ typename P::acc kscale_of(const SV<P, W> &a, int32_t gv) {
    return B ? __ldg(&a.gks[gv]) : a.kscale;
}

// Whether a step decides by proposals that an apply phase commits after
// the step's evaluation, rather than moving at once: always in the
// deterministic mode and in the refinement, and in the asynchronous
// local-moving in the capped steps, where neighbours may share a step (on
// heavy-tailed graphs most vertices are there, and moving at once let
// neighbours chase each other).
template <class P, bool REFINE> __device__ __forceinline__ bool proposing(int32_t cur_step, int32_t cap_step) {
    return REFINE || P::det || cur_step >= cap_step;
}
// the gain of a local-moving proposal, in the key's own type (a 128-bit
// gain takes the two words gain[2v], gain[2v+1])
__device__ __forceinline__ void store_gain(long long *gain, int32_t v, __int128 g) {
    gain[2 * (int64_t)v] = (long long)(unsigned long long)g;
    gain[2 * (int64_t)v + 1] = (long long)(g >> 64);
}
__device__ __forceinline__ void store_gain(long long *gain, int32_t v, float g) {
    reinterpret_cast<float *>(gain)[v] = g;
}
__device__ __forceinline__ unsigned __int128 load_gain128(const long long *gain, int32_t v) {
    const unsigned long long lo = (unsigned long long)__ldcg(&gain[2 * (int64_t)v]);
    const unsigned long long hi = (unsigned long long)__ldcg(&gain[2 * (int64_t)v + 1]);
    return ((unsigned __int128)hi << 64) | lo;
}

// Decision for vertex v (one thread, graph gv, key scale kscale) with best
// candidate (key, cand), K_{v->d} = kvd and Sigma_d = sd. Returns true if
// an asynchronous local-moving move was applied (its neighbours must then be
// marked unprocessed).
template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ bool decide_sd(const SV<P, W> &a, int32_t v, int32_t d, typename P::acc Kv,
                                          typename P::key key, int32_t cand, typename P::acc kvd,
                                          typename P::tot sd, Sums<P> &sm, int32_t cur_step, int32_t gv,
                                          typename P::acc kscale) {
    using A = typename P::acc;
    using T = typename P::tot;
    using K = typename P::key;
    bool mv = false;
    K g = 0;
    if (cand != INT_MAX) {
        const K ks = stay_key(kscale, kvd, Kv, sd, a.gamma);
        mv = key > ks;
        if (!REFINE && mv && cur_step >= a.cap_step) {
            // S2: where neighbours may move together, a single-vertex
            // community does not move into a larger-id single-vertex one.
            if (ldm(&a.size[d]) == 1 && ldm(&a.size[cand]) == 1 && cand > d) mv = false;
        }
        g = key - ks;
    }
    if constexpr (P::det) {
        // the deterministic mode always proposes (an apply phase commits)
        a.prop[v] = mv ? cand : -1;
        if (!REFINE && mv) store_gain(a.gain, v, g);
        return false;
    } else {
        if (REFINE && cur_step < a.cap_step) {
            // Asynchronous refinement below the capped step: no two vertices
            // of a step are adjacent, so the neighbour through which v saw
            // cand stays in cand and nobody joins v while it leaves: the join
            // is applied at once (the gain sum counts joins in this phase).
            if (mv) {
                atomic_add_acc(&a.Sig[d], -(T)Kv);
                atomic_add_acc(&a.Sig[cand], (T)Kv);
                atomicSub(&a.size[d], 1);
                atomicAdd(&a.size[cand], 1);
                a.C[v] = cand;
                gacc_add(sm.gain, B, gv, (A)1, sm.mv);
            }
            return false;
        }
        if (proposing<P, REFINE>(cur_step, a.cap_step)) {
            a.prop[v] = mv ? cand : -1;
            if (!REFINE && mv) store_gain(a.gain, v, g);
            return false;
        }
        if (mv) {
            atomic_add_acc(&a.Sig[d], -(T)Kv);
            atomic_add_acc(&a.Sig[cand], (T)Kv);
            atomicSub(&a.size[d], 1);
            atomicAdd(&a.size[cand], 1);
            a.C[v] = cand;
            gacc_add(sm.gain, B, gv, g, sm.dq);
        }
    }
    return mv;
}
template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ bool decide(const SV<P, W> &a, int32_t v, int32_t d, typename P::acc Kv,
                                       typename P::key key, int32_t cand, typename P::acc kvd, Sums<P> &sm,
                                       int32_t cur_step, int32_t gv, typename P::acc kscale) {
    return decide_sd<P, W, REFINE, B>(a, v, d, Kv, key, cand, kvd, ldm(&a.Sig[d]), sm, cur_step, gv, kscale);
}

// Key of candidate community c for vertex v. The randomized refinement
// (asynchronous mode) replaces the gain key > 0 of an isolated vertex (whose
// staying key is 0) by 1 / (1 - ln(U) / key), U uniform in (0, 1) from the
// vertex, the community and the sweep: the largest of these keys is a draw
// with probability proportional to the gain (Efraimidis and Spirakis'
// weighted sampling, in an order-preserving form), and it stays positive, so
// the vertex moves exactly when some gain is positive.
template <class P, class W, bool REFINE>
__device__ __forceinline__ typename P::key cand_key(const SV<P, W> &a, const Sums<P> &sm, int32_t v, int32_t c,
                                                    typename P::key kk) {
    if constexpr (P::det || !REFINE) {
        return kk;
    } else {
        if (!a.rand_refine) return kk;
        if (!(kk > 0)) return AccLimits<typename P::key>::lowest();
        const uint64_t h = splitmix64_at(a.rseed + 0xD1B54A32D192ED03ULL * (uint64_t)sm.stamp,
                                         ((uint64_t)(uint32_t)v << 32) | (uint32_t)c);
        const float u = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
        return 1.0f / (1.0f - logf(u) / kk);
    }
}

// act[k] = stamp, written only when it differs (a step's mark is read by
// many threads and written about once)
__device__ __forceinline__ void mark_step(int32_t *act, int32_t k, int32_t stamp) {
    if (__ldcg(&act[k]) != stamp) act[k] = stamp;
}
// A neighbour u of a mover becomes unprocessed (Algorithm 2 pruning); its
// step is marked active for the rest of this sweep.
template <class P, class W>
__device__ __forceinline__ void flag_unproc(const SV<P, W> &a, const Sums<P> &sm, int32_t u) {
    a.unproc[u] = 1;
    if (a.act) mark_step(a.act, a.step[u], sm.stamp);
}

// Eligibility: local-moving takes unprocessed vertices and marks them
// processed (Algorithm 2 pruning); refinement takes isolated vertices (the
// community of v has v as its only member, reading R7). In a batch, the
// vertices of a graph whose phase has converged are left alone.
template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ bool take_vertex(const SV<P, W> &a, int32_t v, int32_t &d, int32_t gv) {
    if (REFINE) {
        d = ldm(&a.C[v]);
        return ldm(&a.size[d]) == 1 && !(B && ldm(&a.gdone[gv]));
    }
    const bool e = ldm(&a.unproc[v]) != 0 && !(B && ldm(&a.gdone[gv]));
    if (e) {
        a.unproc[v] = 0;
        d = ldm(&a.C[v]);
    }
    return e;
}

// --------------------------------------------------------- thread bin
template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ void run_thread(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo, int64_t hi,
                                           int32_t cur_step, Sums<P> &sm, ProfCounts &pc) {
    using A = typename P::acc;
    constexpr int E = kThreadMaxDeg;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < hi; t += nthreads) {
        const int32_t v = list[t];
        // eligibility first (Algorithm 2 pruning: the unprocessed flag;
        // refinement: the size of the vertex's community), so that a pruned
        // vertex costs one flag load and none of the header loads below
        int32_t d = 0;
        bool elig;
        if (REFINE) {
            d = ldm(&a.C[v]);
            elig = ldm(&a.size[d]) == 1;
        } else {
            elig = ldm(&a.unproc[v]) != 0;
        }
        const int32_t gv = (B && elig) ? graph_of<B>(a, v) : 0;
        if (B && elig) elig = !ldm(&a.gdone[gv]);
        if (!elig) {
            if (proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
            pc.v[1]++;
            continue;
        }
        if (!REFINE) {
            a.unproc[v] = 0;  // processed (Algorithm 2 pruning)
            d = ldm(&a.C[v]);
        }
        const A Kv = k_of(a, v, t);
        const RowOf<W> row = row_of(a, v, t);
        const int64_t e0 = row.e0;
        const int32_t dv = row.dv;
        const typename P::tot sd = ldm(&a.Sig[d]);
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int32_t jj[E];
        A wt[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            jj[k] = -1;
            wt[k] = 0;
            if (k < dv) {
                jj[k] = row.idx[e0 + k];
                wt[k] = wconv<A>(row.w[e0 + k]);
            }
        }
        int32_t c[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            c[k] = -1;
            bool ok = k < dv && jj[k] != v;
            if (REFINE && ok) ok = (__ldg(&a.CB[jj[k]]) == bv);
            if (ok) c[k] = ldm(&a.C[jj[k]]);
        }
        // merge equal communities into their first entry, in edge order
#pragma unroll
        for (int k = 1; k < E; ++k)
#pragma unroll
            for (int k2 = 0; k2 < k; ++k2)
                if (c[k] >= 0 && c[k2] == c[k]) {
                    wt[k2] += wt[k];
                    c[k] = -1;
                }
        A kvd = 0;
        typename P::key key = AccLimits<typename P::key>::lowest();
        int32_t cand = INT_MAX;
        int distinct = 0;
        const A ks = kscale_of<B>(a, gv);
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if (c[k] < 0) continue;
            distinct++;
            if (c[k] == d) {
                kvd = wt[k];
                continue;
            }
            const typename P::key kk =
                cand_key<P, W, REFINE>(a, sm, v, c[k], move_key(ks, wt[k], Kv, ldm(&a.Sig[c[k]]), a.gamma));
            if (better(kk, c[k], key, cand)) {
                key = kk;
                cand = c[k];
            }
        }
        const bool mv = decide_sd<P, W, REFINE, B>(a, v, d, Kv, key, cand, kvd, sd, sm, cur_step, gv, ks);
        if (a.prof) {
            pc.v[0]++;
            pc.v[2] += dv;
            pc.v[3] += distinct;
            if (proposing<P, REFINE>(cur_step, a.cap_step) ? (a.prop[v] >= 0) : mv) {
                pc.v[4]++;
                pc.v[5] += dv;
            }
        }
        if (!REFINE && !P::det && mv) {
#pragma unroll
            for (int k = 0; k < E; ++k)
                if (k < dv) flag_unproc(a, sm, jj[k]);  // neighbours (self-loop included) of a mover
        }
    }
}

// ----------------------------------------------------------- tile bins
template <class P, class W, int T, bool REFINE, bool B>
__device__ __forceinline__ void run_tile(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo, int64_t hi,
                                         int32_t cur_step, Sums<P> &sm, ProfCounts &pc) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const unsigned tmask = (T == 32) ? kFull : (((1u << T) - 1u) << (lane & ~(T - 1)));
    const int64_t tiles = (int64_t)gridDim.x * (blockDim.x / T);
    for (int64_t t = lo + (int64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T; t < hi; t += tiles) {
        const int32_t v = list[t];
        const int32_t gv = graph_of<B>(a, v);
        int32_t d = 0;
        int elig = 0;
        if (tl == 0) elig = take_vertex<P, W, REFINE, B>(a, v, d, gv) ? 1 : 0;
        elig = __shfl_sync(tmask, elig, 0, T);
        d = __shfl_sync(tmask, d, 0, T);
        if (!elig) {
            if (tl == 0 && proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
            if (tl == 0) pc.v[1]++;
            continue;
        }
        const A Kv = k_of(a, v, t);
        const RowOf<W> row = row_of(a, v, t);
        const int64_t e0 = row.e0;
        const int32_t dv = row.dv;
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int32_t j = -1, c = -1;
        A wv = 0;
        if (tl < dv) {
            j = row.idx[e0 + tl];
            wv = wconv<A>(row.w[e0 + tl]);
            bool ok = (j != v);
            if (REFINE && ok) ok = (__ldg(&a.CB[j]) == bv);
            if (ok) c = ldm(&a.C[j]);
        }
        // merge equal communities: each lane sums the lanes of its community
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
        typename P::key key = AccLimits<typename P::key>::lowest();
        int32_t cand = INT_MAX;
        const A ks = kscale_of<B>(a, gv);
        if (lead && c != d) {
            key = cand_key<P, W, REFINE>(a, sm, v, c, move_key(ks, sum, Kv, ldm(&a.Sig[c]), a.gamma));
            cand = c;
        }
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) {
            const typename P::key ok = kshfl_xor(tmask, key, o, T);
            const int32_t oc = __shfl_xor_sync(tmask, cand, o, T);
            if (better(ok, oc, key, cand)) {
                key = ok;
                cand = oc;
            }
        }
        int mv = 0;
        if (tl == 0) mv = decide<P, W, REFINE, B>(a, v, d, Kv, key, cand, kvd, sm, cur_step, gv, ks) ? 1 : 0;
        if (a.prof) {
            const unsigned lb = __ballot_sync(tmask, lead) & tmask;
            if (tl == 0) {
                pc.v[0]++;
                pc.v[2] += dv;
                pc.v[3] += __popc(lb);
                if (proposing<P, REFINE>(cur_step, a.cap_step) ? (a.prop[v] >= 0) : (mv != 0)) {
                    pc.v[4]++;
                    pc.v[5] += dv;
                }
            }
        }
        if (!REFINE && !P::det) {
            mv = __shfl_sync(tmask, mv, 0, T);
            if (mv && tl < dv) flag_unproc(a, sm, j);  // neighbours (self-loop included) of a mover
        }
    }
}

// ------------------------------------------------------- warp-table bin
template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ void run_warp(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo, int64_t hi,
                                         int32_t cur_step, int32_t *keys, typename P::acc *vals, Sums<P> &sm,
                                         ProfCounts &pc) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = lo + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < hi; t += nwarps) {
        const int32_t v = list[t];
        const int32_t gv = graph_of<B>(a, v);
        int32_t d = 0;
        int elig = 0;
        if (lane == 0) elig = take_vertex<P, W, REFINE, B>(a, v, d, gv) ? 1 : 0;
        elig = __shfl_sync(kFull, elig, 0);
        d = __shfl_sync(kFull, d, 0);
        if (!elig) {
            if (lane == 0 && proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
            if (lane == 0) pc.v[1]++;
            continue;
        }
        const A Kv = k_of(a, v, t);
        const RowOf<W> row = row_of(a, v, t);
        const int64_t e0 = row.e0;
        const int32_t dv = row.dv;
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
            const int32_t j = row.idx[e0 + e];
            if (j == v) continue;
            if (REFINE && __ldg(&a.CB[j]) != bv) continue;
            if (!hash_add(keys, vals, bits, ldm(&a.C[j]), wconv<A>(row.w[e0 + e]))) set_error(a.err, kErrHashFull);
        }
        __syncwarp();
        typename P::key key = AccLimits<typename P::key>::lowest();
        A kvd = 0;
        int32_t cand = INT_MAX;
        const A ks = kscale_of<B>(a, gv);
        for (int s = lane; s < S; s += 32) {
            const int32_t k = keys[s];
            if (k < 0) continue;
            pc.v[3]++;
            const A sum = vals[s];
            if (k == d) {
                kvd = sum;
                continue;
            }
            const typename P::key kk =
                cand_key<P, W, REFINE>(a, sm, v, k, move_key(ks, sum, Kv, ldm(&a.Sig[k]), a.gamma));
            if (better(kk, k, key, cand)) {
                key = kk;
                cand = k;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const typename P::key ok = kshfl_xor(kFull, key, o);
            const int32_t oc = __shfl_xor_sync(kFull, cand, o);
            if (better(ok, oc, key, cand)) {
                key = ok;
                cand = oc;
            }
        }
        kvd = warp_sum(kvd);
        int mv = 0;
        if (lane == 0) {
            mv = decide<P, W, REFINE, B>(a, v, d, Kv, key, cand, kvd, sm, cur_step, gv, ks) ? 1 : 0;
            pc.v[0]++;
            pc.v[2] += dv;
            if (proposing<P, REFINE>(cur_step, a.cap_step) ? (a.prop[v] >= 0) : (mv != 0)) {
                pc.v[4]++;
                pc.v[5] += dv;
            }
        }
        if (!REFINE && !P::det) {
            mv = __shfl_sync(kFull, mv, 0);
            if (mv)
                for (int32_t e = lane; e < dv; e += 32) flag_unproc(a, sm, row.idx[e0 + e]);
        }
        __syncwarp();
    }
}

// ------------------------------------------------ block / hub table bins
// One block per vertex (HUB: a global-memory table per block; only blocks
// below hub_regions take part).
template <class P, class W, bool REFINE, bool HUB, bool B>
__device__ __forceinline__ void run_block(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo, int64_t hi,
                                          int32_t cur_step, int32_t *keys, typename P::acc *vals, int max_bits,
                                          Sums<P> &sm, ProfCounts &pc) {
    using A = typename P::acc;
    __shared__ int s_elig, s_d, s_mv;
    __shared__ typename P::key s_key[32];
    __shared__ A s_kvd[32];
    __shared__ int32_t s_cand[32];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nw = blockDim.x >> 5;
    const int64_t nblk = HUB ? (int64_t)a.hub_regions : (int64_t)gridDim.x;
    if (HUB && (int64_t)blockIdx.x >= nblk) return;
    for (int64_t t = lo + blockIdx.x; t < hi; t += nblk) {
        const int32_t v = list[t];
        const int32_t gv = graph_of<B>(a, v);
        __syncthreads();
        if (tid == 0) {
            int32_t d = 0;
            s_elig = take_vertex<P, W, REFINE, B>(a, v, d, gv) ? 1 : 0;
            s_d = d;
            if (!s_elig && proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
            if (!s_elig) pc.v[1]++;
        }
        __syncthreads();
        if (!s_elig) continue;
        const int32_t d = s_d;
        const A Kv = k_of(a, v, t);
        const RowOf<W> row = row_of(a, v, t);
        const int64_t e0 = row.e0;
        const int32_t dv = row.dv;
        const int32_t bv = REFINE ? a.CB[v] : 0;
        int bits = ceil_log2(2 * (int64_t)dv);
        if (bits < 6) bits = 6;
        if (bits > max_bits) {
            if (tid == 0) {
                set_error(a.err, kErrHashFull);
                if (proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
            }
            continue;
        }
        const int64_t S = 1LL << bits;
        for (int64_t s = tid; s < S; s += blockDim.x) {
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncthreads();
        for (int64_t e = tid; e < dv; e += blockDim.x) {
            const int32_t j = row.idx[e0 + e];
            if (j == v) continue;
            if (REFINE && __ldg(&a.CB[j]) != bv) continue;
            if (!hash_add(keys, vals, bits, ldm(&a.C[j]), wconv<A>(row.w[e0 + e]))) set_error(a.err, kErrHashFull);
        }
        __syncthreads();
        typename P::key key = AccLimits<typename P::key>::lowest();
        A kvd = 0;
        int32_t cand = INT_MAX;
        const A ks = kscale_of<B>(a, gv);
        for (int64_t s = tid; s < S; s += blockDim.x) {
            const int32_t k = keys[s];
            if (k < 0) continue;
            pc.v[3]++;
            const A sum = vals[s];
            if (k == d) {
                kvd = sum;
                continue;
            }
            const typename P::key kk =
                cand_key<P, W, REFINE>(a, sm, v, k, move_key(ks, sum, Kv, ldm(&a.Sig[k]), a.gamma));
            if (better(kk, k, key, cand)) {
                key = kk;
                cand = k;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const typename P::key ok = kshfl_xor(kFull, key, o);
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
            typename P::key bk = s_key[0];
            A kd = s_kvd[0];
            int32_t bc = s_cand[0];
            for (int w2 = 1; w2 < nw; ++w2) {
                if (better(s_key[w2], s_cand[w2], bk, bc)) {
                    bk = s_key[w2];
                    bc = s_cand[w2];
                }
                kd += s_kvd[w2];
            }
            s_mv = decide<P, W, REFINE, B>(a, v, d, Kv, bk, bc, kd, sm, cur_step, gv, ks) ? 1 : 0;
            pc.v[0]++;
            pc.v[2] += dv;
            if (proposing<P, REFINE>(cur_step, a.cap_step) ? (a.prop[v] >= 0) : (s_mv != 0)) {
                pc.v[4]++;
                pc.v[5] += dv;
            }
        }
        __syncthreads();
        if (!REFINE && !P::det && s_mv)
            for (int64_t e = tid; e < dv; e += blockDim.x) flag_unproc(a, sm, row.idx[e0 + e]);
    }
    __syncthreads();
}

// -------------------------------------------- bin 6 on the whole grid
// In the persistent sweep the vertices of bin 6 (rows of more than
// kBlockMaxDeg entries) of a step are evaluated by every block together:
// degree-first schedules put a few hubs in each of many steps, and one block
// per hub would leave the rest of the GPU waiting on the largest. Hub j of
// the pass (its ordinal in list order) is hubs[j]. Phases, each ended by a
// grid barrier: block 0 takes the eligibility of the step's hubs and lays
// out the eligible ones (hj[p] = j; table slots [htoff[p], htoff[p+1]), a
// power of two of at least 2 deg; row entries [heoff[p], heoff[p+1]) of the
// flat walk); clearing; insertion of the rows (entries of one warp step
// with equal (hub, community) summed first); the largest key per hub
// (atomicMax on an order-preserving encoding); the smallest community id
// among those with that key (atomicMin), which is the candidate a block's
// own scan finds; the decision, one thread per hub; for an asynchronous
// local-moving move, the neighbours' flags. A step whose hubs are all
// ineligible ends after the first phase.
// order-preserving unsigned encodings of the keys: a 128-bit key as (high
// word with its sign bit flipped, low word), compared high word first; an
// fp32 key in the low 32 bits
__device__ __forceinline__ void key_order(__int128 k, unsigned long long &hi, unsigned long long &lo) {
    hi = (unsigned long long)(long long)(k >> 64) ^ 0x8000000000000000ULL;
    lo = (unsigned long long)k;
}
__device__ __forceinline__ __int128 key_of_order(unsigned long long hi, unsigned long long lo, __int128) {
    return (__int128)(((unsigned __int128)(hi ^ 0x8000000000000000ULL) << 64) | lo);
}
__device__ __forceinline__ void key_order(float k, unsigned long long &hi, unsigned long long &lo) {
    const unsigned u = __float_as_uint(k);
    hi = (unsigned long long)((u & 0x80000000u) ? ~u : (u | 0x80000000u));
    lo = 0ULL;
}
__device__ __forceinline__ float key_of_order(unsigned long long e, unsigned long long, float) {
    const unsigned u = (unsigned)e;
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// the p in [0, np) whose range [off[p], off[p+1]) holds x (off ascending)
__device__ __forceinline__ int64_t range_at(const int64_t *off, int64_t np, int64_t x) {
    int64_t lo = 0, hi = np - 1;  // the last p with off[p] <= x
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldcg(&off[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// exclusive block scan of x (every thread of the block calls it); returns
// the block total in *total
__device__ __forceinline__ long long block_scan_excl(long long x, long long *total) {
    __shared__ long long s_w[32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) s_w[wib] = inc;
    __syncthreads();
    long long before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < wib) before += s_w[w];
        all += s_w[w];
    }
    *total = all;
    return before + inc - x;
}

// The neighbours of the step's moving hubs become unprocessed (Algorithm 2
// pruning), the whole grid walking the hubs' rows as one flat range (the
// layout of run_hubs_grid: eligible hub p owns entries [heoff[p],
// heoff[p+1]) of hub hj[p]). A hub moved when hmv[j] is set (a move made at
// once) or, in an apply phase (by_prop), when its proposal is set.
template <class P, class W>
__device__ __forceinline__ void hub_flags(const SV<P, W> &a, const Sums<P> &sm, int64_t np, int64_t E, bool by_prop) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // a contiguous range of entries per warp, following the hub as it goes
    // (a row is longer than 32 entries: 32 consecutive ones span at most two)
    const int64_t per = ((E + warps - 1) / warps + 31) & ~(int64_t)31;
    const int64_t x1 = (gw + 1) * per < E ? (gw + 1) * per : E;
    if (gw * per >= x1) return;
    int64_t p = 0;
    if (lane == 0) p = range_at(a.heoff, np, gw * per);
    p = __shfl_sync(kFull, p, 0);
    int64_t nb = __ldcg(&a.heoff[p + 1]);
    for (int64_t x0 = gw * per; x0 < x1; x0 += 32) {
        while (x0 >= nb) nb = __ldcg(&a.heoff[++p + 1]);
        const int64_t x = x0 + lane;
        if (x >= x1) continue;
        const int64_t pl = x >= nb ? p + 1 : p;
        const int64_t j = __ldcg(&a.hj[pl]);
        const int32_t v = __ldg(&a.hubs[j]);
        if (by_prop ? (ldm(&a.prop[v]) < 0) : !__ldcg(&a.hmv[j])) continue;
        flag_unproc(a, sm, a.idx[a.off[v] + (x - __ldcg(&a.heoff[pl]))]);
    }
}

// the asynchronous mode's whole-grid hub tables: one 8-byte word per slot
// (key and fp32 value, hash_add_kv) in the value buffer, which holds 8 bytes
// per slot
template <class P, class W> __device__ __forceinline__ unsigned long long *hub_kv(const SV<P, W> &a) {
    return reinterpret_cast<unsigned long long *>(a.hub_vals);
}

template <class P, class W, bool REFINE, bool B>
__device__ __forceinline__ bool run_hubs_grid(const SV<P, W> &a, int64_t j0, int64_t nh, int32_t cur_step,
                                              Sums<P> &sm, ProfCounts &pc) {
    using A = typename P::acc;
    const int lane = threadIdx.x & 31;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t warps = nthreads >> 5, gw = tid >> 5;
    // A layered step (below cap_step: no two of its vertices are adjacent)
    // with one hub: every block reads the hub's eligibility itself -- no
    // vertex of the step can change it (a flag is set, or a community joined,
    // only by a neighbour), and the grid barriers of the previous step made
    // its last writes visible -- so the layout needs no barrier of its own.
    // Block 0 records the layout and resets the hub's state before the
    // insertion barrier, and clears the pruning flag after it, once every
    // block has read the flag.
    const bool single = nh == 1 && cur_step < a.cap_step;
    int64_t np, S, E;
    int32_t sv = -1, sbits = 0;  // single: the hub and its table's log2 size
    if (single) {
        const int32_t v = __ldg(&a.hubs[j0]);
        const int32_t gv = graph_of<B>(a, v);
        int32_t d = 0;
        bool e;
        if (REFINE) {
            d = ldm(&a.C[v]);
            e = ldm(&a.size[d]) == 1 && !(B && ldm(&a.gdone[gv]));
        } else {
            e = ldm(&a.unproc[v]) != 0 && !(B && ldm(&a.gdone[gv]));
            if (e) d = ldm(&a.C[v]);
        }
        const int32_t dv = e ? a.deg[v] : 0;
        sbits = ceil_log2(2 * (int64_t)dv);
        if (sbits < 6) sbits = 6;
        np = e ? 1 : 0;
        S = e ? (1LL << sbits) : 0;
        E = dv;
        sv = v;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (!e) {
                if (proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
                pc.v[1]++;
            } else {
                if (P::det) {
                    a.hkey[2 * j0] = 0ULL;
                    a.hkey[2 * j0 + 1] = 0ULL;
                } else {
                    a.hkey[j0] = 0ULL;
                }
                a.hcand[j0] = INT_MAX;
                a.hkvd[j0] = 0;
                a.hmv[j0] = 0;
                a.hj[0] = (int32_t)j0;
                a.htoff[0] = 0;
                a.heoff[0] = 0;
                a.htoff[1] = S;
                a.heoff[1] = E;
                a.hinfo[0] = np;
                a.hinfo[1] = S;
                a.hinfo[2] = E;
            }
            a.hd[j0] = e ? d : -1;
        }
        if (np == 0) return true;  // the same in every block
    } else {
        // eligibility and layout (block 0)
        if (blockIdx.x == 0) {
            long long np = 0, ns = 0, ne = 0;
            for (int64_t i0 = 0; i0 < nh; i0 += blockDim.x) {
                const int64_t i = i0 + threadIdx.x;
                bool e = false;
                int64_t sz = 0, dv = 0;
                if (i < nh) {
                    const int64_t j = j0 + i;
                    const int32_t v = __ldg(&a.hubs[j]);
                    const int32_t gv = graph_of<B>(a, v);
                    int32_t d = 0;
                    e = take_vertex<P, W, REFINE, B>(a, v, d, gv);
                    if (!e) {
                        if (proposing<P, REFINE>(cur_step, a.cap_step)) a.prop[v] = -1;
                        pc.v[1]++;
                    } else {
                        dv = a.deg[v];
                        int bits = ceil_log2(2 * dv);
                        if (bits < 6) bits = 6;
                        sz = 1LL << bits;
                        if (P::det) {
                            a.hkey[2 * j] = 0ULL;
                            a.hkey[2 * j + 1] = 0ULL;
                        } else {
                            a.hkey[j] = 0ULL;
                        }
                        a.hcand[j] = INT_MAX;
                        a.hkvd[j] = 0;
                        a.hmv[j] = 0;
                    }
                    a.hd[j] = e ? d : -1;
                }
                long long tp, ts, te;
                const long long p = block_scan_excl(e ? 1 : 0, &tp);
                const long long so = block_scan_excl(sz, &ts);
                const long long eo = block_scan_excl(dv, &te);
                if (e) {
                    a.hj[np + p] = (int32_t)(j0 + i);
                    a.htoff[np + p] = ns + so;
                    a.heoff[np + p] = ne + eo;
                }
                np += tp;
                ns += ts;
                ne += te;
            }
            if (threadIdx.x == 0) {
                a.htoff[np] = ns;
                a.heoff[np] = ne;
                a.hinfo[0] = np;
                a.hinfo[1] = ns;
                a.hinfo[2] = ne;
            }
        }
        if (!grid_barrier(a.bar, a.err, a.spin_limit)) return false;
        np = __ldcg(&a.hinfo[0]);
        S = __ldcg(&a.hinfo[1]);
        E = __ldcg(&a.hinfo[2]);
        if (np == 0) return true;
    }
    // Each warp takes one contiguous range of entries (insertion) or slots
    // (key passes), 32 at a time, and follows the hub they belong to as it
    // goes: one binary search at the start of its range, then a step to the
    // next hub when a boundary is passed. A hub's row is longer than 32
    // entries, so 32 consecutive entries span at most two hubs; its table is
    // a power of two of at least 8192 slots, so 32 aligned slots lie in one.
    // insertion (the tables are clean: the last scan of a step clears every
    // slot it reads, and the engine clears them before the first sweep)
    if (single) {  // one hub: its entries [0, E), its table [0, S); the layout in registers
        const int64_t per = ((E + warps - 1) / warps + 31) & ~(int64_t)31;
        const int64_t x1 = (gw + 1) * per < E ? (gw + 1) * per : E;
        const int64_t e0 = a.off[sv];
        const int32_t bv = REFINE ? __ldg(&a.CB[sv]) : 0;
        for (int64_t x0 = gw * per; x0 < x1; x0 += 32) {
            const int64_t x = x0 + lane;
            int32_t key = -1;
            A val = 0;
            if (x < x1) {
                const int32_t u = a.idx[e0 + x];
                if (u != sv && (!REFINE || __ldg(&a.CB[u]) == bv)) {
                    key = ldm(&a.C[u]);
                    val = wconv<A>(a.w[e0 + x]);
                }
            }
            const unsigned peers = __match_any_sync(kFull, key);
            val = peer_sum(peers, val);
            if (key >= 0 && lane == __ffs(peers) - 1) {
                bool ok;
                if constexpr (P::det) ok = hash_add(a.hub_keys, a.hub_vals, sbits, key, val);
                else ok = hash_add_kv(hub_kv<P>(a), sbits, key, val);
                if (!ok) set_error(a.err, kErrHashFull);
            }
        }
    } else {
        const int64_t per = ((E + warps - 1) / warps + 31) & ~(int64_t)31;
        const int64_t x1 = (gw + 1) * per < E ? (gw + 1) * per : E;
        int64_t p = 0, nb = 0;  // hub of the warp's current entry and the end of its row
        if (gw * per < x1) {
            if (lane == 0) p = range_at(a.heoff, np, gw * per);
            p = __shfl_sync(kFull, p, 0);
            nb = __ldcg(&a.heoff[p + 1]);
        }
        for (int64_t x0 = gw * per; x0 < x1; x0 += 32) {
            while (x0 >= nb) nb = __ldcg(&a.heoff[++p + 1]);  // the same on every lane
            const int64_t x = x0 + lane;
            const int64_t pl = x >= nb ? p + 1 : p;
            int32_t key = -1, bits = 0;
            int64_t tbase = 0;
            A val = 0;
            if (x < x1) {
                const int32_t v = __ldg(&a.hubs[__ldcg(&a.hj[pl])]);
                const int64_t e = a.off[v] + (x - (pl == p ? nb - a.deg[v] : nb));
                const int32_t u = a.idx[e];
                if (u != v && (!REFINE || __ldg(&a.CB[u]) == __ldg(&a.CB[v]))) {
                    key = ldm(&a.C[u]);
                    val = wconv<A>(a.w[e]);
                    tbase = __ldcg(&a.htoff[pl]);
                    bits = __ffsll((long long)(__ldcg(&a.htoff[pl + 1]) - tbase)) - 1;
                }
            }
            const unsigned long long pair = key >= 0 ? ((unsigned long long)pl << 32) | (uint32_t)key : ~0ULL;
            const unsigned peers = __match_any_sync(kFull, pair);
            val = peer_sum(peers, val);
            if (key >= 0 && lane == __ffs(peers) - 1) {
                bool ok;
                if constexpr (P::det) ok = hash_add(a.hub_keys + tbase, a.hub_vals + tbase, bits, key, val);
                else ok = hash_add_kv(hub_kv<P>(a) + tbase, bits, key, val);
                if (!ok) set_error(a.err, kErrHashFull);
            }
        }
    }
    if (!grid_barrier(a.bar, a.err, a.spin_limit)) return false;
    // every block has read the single hub's pruning flag: it is processed
    if (single && !REFINE && blockIdx.x == 0 && threadIdx.x == 0) a.unproc[sv] = 0;
    // deterministic mode: the largest key per hub -- its high word (pass 0),
    // then its low word among the slots with that high word (pass 1) --
    // then the smallest community id with that key (pass 2); asynchronous
    // mode: one pass, key and id packed in one word (fp32 key above the
    // complemented id, so that the largest word is the largest key with the
    // smallest id). K_{v->d} from the slot of v's own community. The last
    // pass clears the slots. The lanes of a warp read one hub's table, so
    // each pass needs one reduction over the warp and one atomic.
    constexpr int npass = P::det ? 3 : 1;
    constexpr int Q = 4;  // slots per lane and iteration: 128 aligned slots lie in one table
    using T = typename P::tot;
    const int64_t sper = ((S + warps - 1) / warps + 32 * Q - 1) & ~(int64_t)(32 * Q - 1);
    const int64_t s1 = (gw + 1) * sper < S ? (gw + 1) * sper : S;
    for (int pass = 0; pass < npass; ++pass) {
        int64_t p = 0, nb = 0;  // table of the warp's current slots and its end
        if (gw * sper < s1) {
            if (lane == 0) p = range_at(a.htoff, np, gw * sper);
            p = __shfl_sync(kFull, p, 0);
            nb = __ldcg(&a.htoff[p + 1]);
        }
        int64_t j = -1;
        int32_t d = -1, v = 0;
        typename P::acc kv = 0, ks = 0;
        unsigned long long hhi = 0, hlo = 0;  // the hub's largest key so far (passes 1 and 2)
        for (int64_t s0 = gw * sper; s0 < s1; s0 += 32 * Q) {
            if (s0 >= nb || j < 0) {  // the warp enters a table: its hub's constants
                while (s0 >= nb) nb = __ldcg(&a.htoff[++p + 1]);
                j = __ldcg(&a.hj[p]);
                d = __ldcg(&a.hd[j]);
                v = __ldg(&a.hubs[j]);
                kv = a.K[v];
                ks = kscale_of<B>(a, graph_of<B>(a, v));
                if (P::det && pass > 0) {
                    hhi = __ldcg(&a.hkey[2 * j]);
                    hlo = __ldcg(&a.hkey[2 * j + 1]);
                }
            }
            // the lane's slots s0 + lane + 32 q: keys first, then the sums
            // and the candidates' totals, all loads of a round in flight
            int32_t kq[Q];
            A vq[Q];
            T sq[Q];
            if constexpr (P::det) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t sl = s0 + 32 * q + lane;
                    kq[q] = sl < s1 ? __ldcg(&a.hub_keys[sl]) : -1;
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    vq[q] = 0;
                    if (kq[q] >= 0) vq[q] = __ldcg(&a.hub_vals[s0 + 32 * q + lane]);
                }
            } else {  // key and value in one word
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t sl = s0 + 32 * q + lane;
                    const unsigned long long kv = sl < s1 ? __ldcg(&hub_kv<P>(a)[sl]) : kEmptyKV;
                    kq[q] = (int32_t)(uint32_t)kv;
                    vq[q] = (A)__uint_as_float((uint32_t)(kv >> 32));
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                sq[q] = 0;
                if (kq[q] >= 0 && kq[q] != d) sq[q] = ldm(&a.Sig[kq[q]]);
            }
            unsigned long long lmax = 0ULL;
            int32_t lmin = INT_MAX;
            bool any = false;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int32_t k = kq[q];
                if (k < 0) continue;
                if (pass == npass - 1) {
                    if constexpr (P::det) {
                        a.hub_keys[s0 + 32 * q + lane] = -1;
                        a.hub_vals[s0 + 32 * q + lane] = 0;
                    } else {
                        hub_kv<P>(a)[s0 + 32 * q + lane] = kEmptyKV;
                    }
                }
                if (k == d) {
                    if (pass == 0) a.hkvd[j] = vq[q];
                    continue;
                }
                unsigned long long enc, enc_lo;
                key_order(cand_key<P, W, REFINE>(a, sm, v, k, move_key(ks, vq[q], kv, sq[q], a.gamma)), enc, enc_lo);
                if (!P::det) enc = (enc << 32) | (unsigned long long)(~(uint32_t)k);
                any = true;
                if (pass == 0) {
                    pc.v[3]++;
                    lmax = enc > lmax ? enc : lmax;
                } else if (pass == 1) {
                    if (enc == hhi) lmax = enc_lo > lmax ? enc_lo : lmax;
                } else if (enc == hhi && enc_lo == hlo) {
                    lmin = k < lmin ? k : lmin;
                }
            }
            if (!__any_sync(kFull, any)) continue;
            if (pass < 2) {
                // the largest high word (pass 0), the largest low word among
                // the slots with the hub's largest high word (pass 1)
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(kFull, lmax, o);
                    lmax = y > lmax ? y : lmax;
                }
                if (lane == 0) {
                    if (pass == 0) atomicMax(&a.hkey[P::det ? 2 * j : j], lmax);
                    else if (lmax) atomicMax(&a.hkey[2 * j + 1], lmax);
                }
            } else {
                for (int o = 16; o > 0; o >>= 1) {
                    const int32_t y = __shfl_xor_sync(kFull, lmin, o);
                    lmin = y < lmin ? y : lmin;
                }
                if (lane == 0 && lmin != INT_MAX) atomicMin(&a.hcand[j], lmin);
            }
        }
        if (!grid_barrier(a.bar, a.err, a.spin_limit)) return false;
    }
    // decisions
    for (int64_t p = tid; p < np; p += nthreads) {
        const int64_t j = __ldcg(&a.hj[p]);
        const int32_t d = __ldcg(&a.hd[j]);
        const int32_t v = __ldg(&a.hubs[j]);
        const int32_t gv = graph_of<B>(a, v);
        using K = typename P::key;
        int32_t c;
        K bk;
        if (P::det) {
            c = __ldcg(&a.hcand[j]);
            bk = c == INT_MAX ? AccLimits<K>::lowest()
                              : key_of_order(__ldcg(&a.hkey[2 * j]), __ldcg(&a.hkey[2 * j + 1]), K(0));
        } else {
            const unsigned long long best = __ldcg(&a.hkey[j]);
            c = best == 0ULL ? INT_MAX : (int32_t)~(uint32_t)best;
            bk = best == 0ULL ? AccLimits<K>::lowest() : key_of_order(best >> 32, 0ULL, K(0));
        }
        const A kd = __ldcg(&a.hkvd[j]);
        const bool mv = decide<P, W, REFINE, B>(a, v, d, a.K[v], bk, c, kd, sm, cur_step, gv, kscale_of<B>(a, gv));
        const int32_t dv = a.deg[v];
        pc.v[0]++;
        pc.v[2] += dv;
        if (proposing<P, REFINE>(cur_step, a.cap_step) ? (ldm(&a.prop[v]) >= 0) : mv) {
            pc.v[4]++;
            pc.v[5] += dv;
        }
        if (!REFINE && !P::det && mv) a.hmv[j] = 1;
    }
    if (!REFINE && !P::det) {
        // an asynchronous local-moving move flags the hub's neighbours
        if (!grid_barrier(a.bar, a.err, a.spin_limit)) return false;
        hub_flags<P, W>(a, sm, np, E, false);
    }
    return true;
}

// ------------------------------------------------------------ apply steps
// Local-moving proposals of one step (deterministic mode; asynchronous mode
// in the capped steps): commit them.
// (grid_hub_flags: the neighbours of rows longer than kBlockMaxDeg are
// flagged by hub_flags over the step's hub layout instead of by one warp)
template <class P, class W, bool B>
__device__ __forceinline__ void run_move_apply(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo,
                                               int64_t hi, Sums<P> &sm, bool grid_hub_flags) {
    // whole warps step through the list, so that the neighbours of a mover
    // with a long row are flagged by the whole warp
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < hi; t0 += stride) {
        const int64_t t = t0 + lane;
        int32_t v = -1, c = -1;
        if (t < hi) {
            v = list[t];
            c = ldm(&a.prop[v]);
        }
        int64_t e0 = 0;
        int32_t dv = 0;
        const int32_t *ridx = a.idx;
        if (c >= 0) {
            const int32_t d = ldm(&a.C[v]);
            const auto Kv = (typename P::tot)k_of(a, v, t);
            atomic_add_acc(&a.Sig[d], -Kv);
            atomic_add_acc(&a.Sig[c], Kv);
            atomicSub(&a.size[d], 1);
            atomicAdd(&a.size[c], 1);
            a.C[v] = c;
            if (P::det)
                gacc_add(sm.dgain, B, graph_of<B>(a, v), load_gain128(a.gain, v),
                         reinterpret_cast<unsigned long long *>(sm.dq));
            else
                gacc_add(sm.gain, B, graph_of<B>(a, v),
                         (typename P::acc)__ldcg(reinterpret_cast<const float *>(a.gain) + v), sm.dq);
            const RowOf<W> row = row_of(a, v, t);
            e0 = row.e0;
            dv = row.dv;
            ridx = row.idx;
            if (dv <= 32)
                for (int32_t e = 0; e < dv; ++e) flag_unproc(a, sm, ridx[e0 + e]);
        }
        unsigned longs = __ballot_sync(kFull, c >= 0 && dv > 32 && !(grid_hub_flags && dv > a.block_max));
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t es = __shfl_sync(kFull, e0, src);
            const int32_t ds = __shfl_sync(kFull, dv, src);
            const int32_t *is = a.loff ? a.lidx : a.idx;  // the same on every lane
            for (int32_t e = lane; e < ds; e += 32) flag_unproc(a, sm, is[es + e]);
        }
    }
}

// Refinement: accept proposal v -> t unless t is a single-vertex community
// whose vertex proposes in the same step; of a mutual pair the larger id
// moves (reading S5). Accepted vertices join t.
template <class P, class W, bool B>
__device__ __forceinline__ void run_refine_apply(const SV<P, W> &a, const int32_t *__restrict__ list, int64_t lo,
                                                 int64_t hi, int32_t cur_step, Sums<P> &sm) {
    for (int64_t t = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < hi;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[t];
        const int32_t tg = ldm(&a.prop[v]);
        if (tg < 0) continue;
        const int32_t pt = (__ldg(&a.step[tg]) == cur_step) ? ldm(&a.prop[tg]) : -1;
        if (!(pt < 0 || (pt == v && v > tg))) continue;
        const auto Kv = (typename P::tot)k_of(a, v, t);
        atomic_add_acc(&a.Sig[v], -Kv);
        atomic_add_acc(&a.Sig[tg], Kv);
        atomicSub(&a.size[v], 1);
        atomicAdd(&a.size[tg], 1);
        a.C[v] = tg;
        gacc_add(sm.moved, B, graph_of<B>(a, v), 1ULL, sm.mv);
    }
}

// ------------------------------------------------------- persistent sweep
constexpr int kCoopThreads = 256;

// a sweep's gain sum of graph g: two words per slot (deterministic, 128 bits)
// or one fp64 word
__device__ __forceinline__ double gain_sum(long long *dq, int64_t g) {
    const unsigned long long *w = reinterpret_cast<const unsigned long long *>(dq) + 2 * g;
    return u128_words_to_double(__ldcg(&w[0]), __ldcg(&w[1]));
}
__device__ __forceinline__ double gain_sum(double *dq, int64_t g) { return __ldcg(&dq[g]); }

// shared-memory tables: 8 warp tables of kWarpSlots slots, or one block table
// of kBlockSlots slots (values first, then keys)
template <class A> constexpr size_t table_bytes() { return (sizeof(A) + sizeof(int32_t)) * kBlockSlots; }
template <class A> __device__ __forceinline__ A *table_vals() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<A *>(smem_raw);
}
template <class A> __device__ __forceinline__ int32_t *table_keys() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<int32_t *>(smem_raw + sizeof(A) * kBlockSlots);
}

// One whole phase: sweeps until the phase converges -- local-moving stops
// when a sweep's delta-modularity (reading S4 for the deterministic mode) is
// at most tau (Algorithm 2), refinement when a sweep moves nobody (reading
// R6) -- or max_it sweeps ran. The test reads per-sweep sums after a grid
// barrier, so every block takes the same decision. In a batch every graph
// takes the test on its own sums; the phase ends when no graph is left.
template <class P, class W, bool REFINE, bool B>
__global__ void __launch_bounds__(kCoopThreads, 4) k_sweep_coop(SV<P, W> a, const int32_t *__restrict__ list) {
    using A = typename P::acc;
    using T = typename P::tot;
    int32_t *skeys = table_keys<A>();
    A *svals = table_vals<A>();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool batch = B;
    // testing aid: this block ends without arriving at any barrier, so the
    // others' bounded wait runs out (kErrTimeout) and the launch ends
    if ((int32_t)blockIdx.x == a.stall_block) return;
    __shared__ int64_t s_ko[2][kNumBins + 2];
    ProfCounts pc;
    int32_t it = 0;
    bool ok = true;
    while (ok && it < a.max_it) {
        Sums<P> sm;
        sm.dq = a.dq_arr + (size_t)it * a.G * (P::det ? 2 : 1);  // deterministic: two words per slot
        sm.mv = a.moved_arr + (size_t)it * a.G;
        sm.stamp = it + 1;
        if (a.act) {
            // steps holding an eligible vertex at the start of the sweep
            // (unprocessed, or isolated in the refinement); moves mark the
            // steps of the neighbours they flag as the sweep goes on, and
            // nothing makes a vertex isolated during the refinement
            const int64_t nl = __ldcg(&a.key_off[(int64_t)a.nsteps * kNumBins]);
            for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl;
                 t += (int64_t)gridDim.x * blockDim.x) {
                const int32_t v = list[t];
                if (B && ldm(&a.gdone[graph_of<B>(a, v)])) continue;
                const bool e = REFINE ? ldm(&a.size[ldm(&a.C[v])]) == 1 : ldm(&a.unproc[v]) != 0;
                if (e) mark_step(a.act, a.step[v], sm.stamp);
            }
            if (!(ok = grid_barrier(a.bar, a.err, a.spin_limit))) break;
        }
        int64_t hub_j0 = 0;  // ordinal of the step's first hub
        for (int32_t k = 0; k < a.nsteps && ok; ++k) {
            // the step's nine (step, bin) offsets and its eligibility mark in
            // one round trip, to shared memory: lanes of warp 0 load one
            // each (the bins' work below stores to global memory, so loads
            // issued between them would wait for one another). Two buffers:
            // a warp reads step k's values before the barrier of step k + 1.
            const int64_t *ko = a.key_off + (int64_t)k * kNumBins;
            int64_t *sko = s_ko[k & 1];
            if (wib == 0 && lane <= kNumBins + 1)
                sko[lane] = lane <= kNumBins ? __ldcg(&ko[lane]) : (a.act ? (int64_t)__ldcg(&a.act[k]) : 0);
            __syncthreads();
            const int64_t b0 = sko[0], b8 = sko[8];
            if (b0 == b8) continue;  // empty step: every block sees the same counts
            if (a.act && (int32_t)sko[kNumBins + 1] != sm.stamp) {  // nothing eligible: the same in every block
                hub_j0 += sko[7] - sko[6];
                continue;
            }
            run_thread<P, W, REFINE, B>(a, list, sko[1], sko[2], k, sm, pc);
            run_tile<P, W, 16, REFINE, B>(a, list, sko[2], sko[3], k, sm, pc);
            run_tile<P, W, 32, REFINE, B>(a, list, sko[3], sko[4], k, sm, pc);
            run_warp<P, W, REFINE, B>(a, list, sko[4], sko[5], k, skeys + wib * kWarpSlots, svals + wib * kWarpSlots,
                                   sm, pc);
            const int64_t b5 = sko[5], b6 = sko[6], b7 = sko[7];
            if (b6 > b5) {
                __syncthreads();  // the warp tables become one block table
                run_block<P, W, REFINE, false, B>(a, list, b5, b6, k, skeys, svals, ceil_log2(kBlockSlots), sm, pc);
            }
            if (b7 > b6) {
                if (a.grid_hubs) {
                    if (!(ok = run_hubs_grid<P, W, REFINE, B>(a, hub_j0, b7 - b6, k, sm, pc))) break;
                } else {
                    const int64_t base = (int64_t)blockIdx.x << a.hub_bits;
                    run_block<P, W, REFINE, true, B>(a, list, b6, b7, k, a.hub_keys + base, a.hub_vals + base,
                                                     a.hub_bits, sm, pc);
                }
                hub_j0 += b7 - b6;
            }
            if (!(ok = grid_barrier(a.bar, a.err, a.spin_limit))) break;
            // apply phase: deterministic mode, and proposals where neighbours
            // may share a step (below the capped step the asynchronous mode
            // moves and joins at once)
            if (P::det || k >= a.cap_step) {
                if (REFINE) {
                    run_refine_apply<P, W, B>(a, list, b0, b8, k, sm);
                } else {
                    const bool hub_layout = a.grid_hubs && b7 > b6;  // run_hubs_grid laid out this step's hubs
                    run_move_apply<P, W, B>(a, list, b0, b8, sm, hub_layout);
                    if (hub_layout) hub_flags<P, W>(a, sm, __ldcg(&a.hinfo[0]), __ldcg(&a.hinfo[2]), true);
                }
                if (!(ok = grid_barrier(a.bar, a.err, a.spin_limit))) break;
            }
        }
        if (!ok) break;
        // this sweep's sums: one graph reduces per warp, a batch flushes
        // every thread's running sum into its graph's slot
        if (batch) {
            if (REFINE) {
                if (!P::det) gacc_flush(sm.gain, sm.mv);
                gacc_flush(sm.moved, sm.mv);
            } else if (P::det) {
                gacc_flush(sm.dgain, reinterpret_cast<unsigned long long *>(sm.dq));
            } else {
                gacc_flush(sm.gain, sm.dq);
            }
        } else if (REFINE) {
            unsigned long long moved = sm.moved.v;
            if (!P::det) moved += (unsigned long long)(sm.gain.v + (A)0.5);
            moved = warp_sum(moved);
            if (lane == 0 && moved) atomicAdd(&sm.mv[0], moved);
        } else if (P::det) {
            const unsigned __int128 g = warp_sum_u128(sm.dgain.v);
            if (lane == 0 && g) atomic_add_u128(reinterpret_cast<unsigned long long *>(sm.dq), g);
        } else {
            const A g = warp_sum(sm.gain.v);
            if (lane == 0 && g != (A)0) atomic_add_acc(&sm.dq[0], (T)g);
        }
        if (!(ok = grid_barrier(a.bar, a.err, a.spin_limit))) break;
        bool stop;
        if (batch) {
            // every graph still running takes its own test; graphs that
            // stop record their sweep count, the others are counted
            unsigned running = 0;
            for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.G;
                 g += (int64_t)gridDim.x * blockDim.x) {
                if (__ldcg(&a.gdone[g])) continue;
                bool sg;
                if (REFINE) {
                    sg = __ldcg(&sm.mv[g]) == 0ULL || a.single_sweep;
                } else {
                    const double tm = a.g2m[g];
                    const double sum = gain_sum(sm.dq, g);
                    // a graph without edges (2m = 0) has nothing to move
                    const double tau = a.gtau ? a.gtau[g] : a.tau;
                    sg = !(tm > 0) || (P::det ? 2.0 * sum / (tm * tm) : 2.0 * sum / tm) <= tau;
                }
                if (sg) {
                    a.gdone[g] = 1;
                    a.giters[g] = it + 1;
                } else {
                    running++;
                }
            }
            running = warp_sum(running);
            if (lane == 0 && running) atomicAdd(&a.gactive[it], running);
            if (!(ok = grid_barrier(a.bar, a.err, a.spin_limit))) break;
            stop = __ldcg(&a.gactive[it]) == 0u;
        } else if (REFINE) {
            stop = __ldcg(&sm.mv[0]) == 0ULL || a.single_sweep;
        } else {
            // sweep delta-modularity from the summed gains: 2 num / (2m)^2
            // (deterministic, reading S4) or 2 sum / 2m (asynchronous)
            const double tm = a.two_m_d;
            const double sum = gain_sum(sm.dq, 0);
            const double dq = P::det ? 2.0 * sum / (tm * tm) : 2.0 * sum / tm;
            stop = dq <= a.tau;
        }
        ++it;
        if (stop) break;
    }
    if (batch) {
        // graphs still running when the phase ends ran every sweep
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.G; g += (int64_t)gridDim.x * blockDim.x)
            if (!__ldcg(&a.gdone[g])) a.giters[g] = it;
    } else if (blockIdx.x == 0 && threadIdx.x == 0 && a.giters) {
        a.giters[0] = it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters_out = it;
    pc.flush(a.prof);
}

// ------------------------------------------- one (step, bin) per launch
// (one graph only) local-moving gains into the sweep's delta-modularity sum;
// asynchronous refinement joins into the move count
template <class P, class W> __device__ __forceinline__ Sums<P> scalar_sums(const SV<P, W> &a) {
    Sums<P> sm;
    sm.dq = a.dq_acc;
    sm.mv = a.moved;
    sm.stamp = a.sweep + 1;
    return sm;
}
template <class P, class W, bool REFINE>
__device__ __forceinline__ void flush_gain(const SV<P, W> &a, Sums<P> &sm) {
    using A = typename P::acc;
    if (P::det) return;
    if (REFINE) {
        const unsigned long long c = warp_sum((unsigned long long)(sm.gain.v + (A)0.5));
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.moved, c);
    } else {
        const A s = warp_sum(sm.gain.v);
        if ((threadIdx.x & 31) == 0 && s != (A)0) atomic_add_acc(a.dq_acc, (typename P::tot)s);
    }
}

template <class P, class W, bool REFINE>
__global__ void __launch_bounds__(256) k_eval_thread(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    Sums<P> sm = scalar_sums(a);
    ProfCounts pc;
    run_thread<P, W, REFINE, false>(a, list, 0, count, a.cur_step, sm, pc);
    flush_gain<P, W, REFINE>(a, sm);
    pc.flush(a.prof);
}
template <class P, class W, int T, bool REFINE>
__global__ void __launch_bounds__(256) k_eval_tile(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    Sums<P> sm = scalar_sums(a);
    ProfCounts pc;
    run_tile<P, W, T, REFINE, false>(a, list, 0, count, a.cur_step, sm, pc);
    flush_gain<P, W, REFINE>(a, sm);
    pc.flush(a.prof);
}
template <class P, class W, bool REFINE>
__global__ void __launch_bounds__(256) k_eval_warp(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    int32_t *skeys = table_keys<A>();
    A *svals = table_vals<A>();
    const int wib = threadIdx.x >> 5;
    Sums<P> sm = scalar_sums(a);
    ProfCounts pc;
    run_warp<P, W, REFINE, false>(a, list, 0, count, a.cur_step, skeys + wib * kWarpSlots, svals + wib * kWarpSlots, sm,
                           pc);
    flush_gain<P, W, REFINE>(a, sm);
    pc.flush(a.prof);
}
template <class P, class W, bool REFINE, bool HUB>
__global__ void __launch_bounds__(256) k_eval_block(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    using A = typename P::acc;
    int32_t *skeys = table_keys<A>();
    A *svals = table_vals<A>();
    Sums<P> sm = scalar_sums(a);
    ProfCounts pc;
    if (HUB) {
        const int64_t base = (int64_t)blockIdx.x << a.hub_bits;
        run_block<P, W, REFINE, true, false>(a, list, 0, count, a.cur_step, a.hub_keys + base, a.hub_vals + base, a.hub_bits,
                                      sm, pc);
    } else {
        run_block<P, W, REFINE, false, false>(a, list, 0, count, a.cur_step, skeys, svals, ceil_log2(kBlockSlots), sm, pc);
    }
    flush_gain<P, W, REFINE>(a, sm);
    pc.flush(a.prof);
}
template <class P, class W>
__global__ void __launch_bounds__(256) k_move_apply(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    Sums<P> sm = scalar_sums(a);
    run_move_apply<P, W, false>(a, list, 0, count, sm, false);
    if (P::det) {
        const unsigned __int128 g = warp_sum_u128(sm.dgain.v);
        if ((threadIdx.x & 31) == 0 && g) atomic_add_u128(reinterpret_cast<unsigned long long *>(a.dq_acc), g);
    } else {
        flush_gain<P, W, false>(a, sm);
    }
}
template <class P, class W>
__global__ void __launch_bounds__(256) k_refine_apply(SV<P, W> a, const int32_t *__restrict__ list, int64_t count) {
    Sums<P> sm = scalar_sums(a);
    run_refine_apply<P, W, false>(a, list, 0, count, a.cur_step, sm);
    const unsigned long long mv = warp_sum(sm.moved.v);
    if ((threadIdx.x & 31) == 0 && mv) atomicAdd(a.moved, mv);
}

// raise the dynamic shared-memory limit of a kernel (a host-side attribute:
// cheap, and set before every launch so no kernel can miss it)
template <class K> cudaError_t allow_table_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class P, class W, bool REFINE>
cudaError_t eval_typed(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                       cudaStream_t s) {
    SV<P, W> a = view<P, W>(c);
    constexpr size_t tb = table_bytes<typename P::acc>();
    auto grid = [&](int64_t per_block) {
        int64_t b = (count + per_block - 1) / per_block;
        return (int)(b < max_blocks ? (b < 1 ? 1 : b) : max_blocks);
    };
    switch (bin) {
        case 1: k_eval_thread<P, W, REFINE><<<grid(256), 256, 0, s>>>(a, list, count); break;
        case 2: k_eval_tile<P, W, 16, REFINE><<<grid(16), 256, 0, s>>>(a, list, count); break;
        case 3: k_eval_tile<P, W, 32, REFINE><<<grid(8), 256, 0, s>>>(a, list, count); break;
        case 4: {
            cudaError_t e = allow_table_smem(k_eval_warp<P, W, REFINE>, tb);
            if (e != cudaSuccess) return e;
            k_eval_warp<P, W, REFINE><<<grid(8), 256, tb, s>>>(a, list, count);
            break;
        }
        case 5: {
            cudaError_t e = allow_table_smem(k_eval_block<P, W, REFINE, false>, tb);
            if (e != cudaSuccess) return e;
            k_eval_block<P, W, REFINE, false><<<grid(1), 256, tb, s>>>(a, list, count);
            break;
        }
        case 6:
            a.hub_regions = max_blocks;
            k_eval_block<P, W, REFINE, true><<<grid(1), 256, 0, s>>>(a, list, count);
            break;
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

template <class P, class W, bool REFINE, bool B>
cudaError_t coop_launch(const SweepCtx &c, const int32_t *list, int grid, cudaStream_t s) {
    SV<P, W> a = view<P, W>(c);
    constexpr size_t tb = table_bytes<typename P::acc>();
    cudaError_t e = allow_table_smem(k_sweep_coop<P, W, REFINE, B>, tb);
    if (e != cudaSuccess) return e;
    void *args[] = {&a, (void *)&list};
    return cudaLaunchCooperativeKernel((const void *)k_sweep_coop<P, W, REFINE, B>, dim3(grid), dim3(kCoopThreads),
                                       args, tb, s);
}
template <class P, class W, bool REFINE>
cudaError_t coop_typed(const SweepCtx &c, const int32_t *list, int grid, cudaStream_t s) {
    return c.gid ? coop_launch<P, W, REFINE, true>(c, list, grid, s) : coop_launch<P, W, REFINE, false>(c, list, grid, s);
}
template <class P, class W, bool REFINE, bool B> int coop_blocks_b() {
    constexpr size_t tb = table_bytes<typename P::acc>();
    if (allow_table_smem(k_sweep_coop<P, W, REFINE, B>, tb) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_coop<P, W, REFINE, B>, kCoopThreads, tb) !=
        cudaSuccess)
        return 0;
    return per_sm;
}
template <class P, class W, bool REFINE> int coop_blocks_typed() {
    // both forms share the launch bounds; take the smaller occupancy
    const int a = coop_blocks_b<P, W, REFINE, false>(), b = coop_blocks_b<P, W, REFINE, true>();
    return a < b ? a : b;
}

}  // namespace

cudaError_t launch_sweep_eval(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) return eval_mode<Det, WInt>(c, bin, list, count, max_blocks, s);
        return eval_mode<Det, float>(c, bin, list, count, max_blocks, s);
    }
    return eval_mode<Async, float>(c, bin, list, count, max_blocks, s);
}

cudaError_t launch_move_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (!c.det) k_move_apply<Async, float><<<apply_grid(count), 256, 0, s>>>(view<Async, float>(c), list, count);
    else if (c.g.w_int) k_move_apply<Det, WInt><<<apply_grid(count), 256, 0, s>>>(view<Det, WInt>(c), list, count);
    else k_move_apply<Det, float><<<apply_grid(count), 256, 0, s>>>(view<Det, float>(c), list, count);
    return cudaGetLastError();
}

cudaError_t launch_refine_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (c.det) {
        if (c.g.w_int) k_refine_apply<Det, WInt><<<apply_grid(count), 256, 0, s>>>(view<Det, WInt>(c), list, count);
        else k_refine_apply<Det, float><<<apply_grid(count), 256, 0, s>>>(view<Det, float>(c), list, count);
    } else {
        k_refine_apply<Async, float><<<apply_grid(count), 256, 0, s>>>(view<Async, float>(c), list, count);
    }
    return cudaGetLastError();
}

int sweep_coop_blocks_per_sm(bool det, bool w_int, bool refine) {
    if (det) {
        if (w_int) return refine ? coop_blocks_typed<Det, WInt, true>() : coop_blocks_typed<Det, WInt, false>();
        return refine ? coop_blocks_typed<Det, float, true>() : coop_blocks_typed<Det, float, false>();
    }
    return refine ? coop_blocks_typed<Async, float, true>() : coop_blocks_typed<Async, float, false>();
}

cudaError_t launch_sweep_coop(const SweepCtx &c, const int32_t *list, int grid, cudaStream_t s) {
    if (c.det) {
        if (c.g.w_int)
            return c.refine ? coop_typed<Det, WInt, true>(c, list, grid, s) : coop_typed<Det, WInt, false>(c, list, grid, s);
        return c.refine ? coop_typed<Det, float, true>(c, list, grid, s) : coop_typed<Det, float, false>(c, list, grid, s);
    }
    return c.refine ? coop_typed<Async, float, true>(c, list, grid, s) : coop_typed<Async, float, false>(c, list, grid, s);
}

}  // namespace lgb
