// Device-side building blocks shared by the Leiden kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lgb {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Arithmetic policies. acc is the type of per-edge sums (K_{i->c}) and
// vertex weights K_i; key the type of move keys and their gains; tot the
// type of community totals Sigma_c and of the asynchronous sweep's
// delta-modularity sums. The deterministic mode decides moves in exact
// integer arithmetic on integer weights: sums, K and Sigma in int64, keys
// (products of two such sums) in 128 bits, and a sweep's gain sum in 128
// bits (two 64-bit words, lo then hi). The asynchronous mode keeps Sigma
// and 2m in fp64 and everything per edge in fp32: on this GPU the fp64 pipe
// is a small fraction of the fp32 rate, and the move key
// K_{i->c} - gamma K_i Sigma_c / 2m has terms of the order of K_i, so fp32
// keeps its relative precision.
struct Det {
    using acc = long long;
    using tot = long long;
    using key = __int128;
    static constexpr bool det = true;
};
struct Async {
    using acc = float;
    using tot = double;
    using key = float;
    static constexpr bool det = false;
};

template <class A> struct AccLimits;
template <> struct AccLimits<long long> {
    __device__ static constexpr long long lowest() { return (long long)0x8000000000000000ULL; }
};
template <> struct AccLimits<double> {
    __device__ static double lowest() { return __longlong_as_double(0xfff0000000000000LL); }  // -inf
};
template <> struct AccLimits<float> {
    __device__ static float lowest() { return __int_as_float(0xff800000); }  // -inf
};
template <> struct AccLimits<__int128> {
    __device__ static __int128 lowest() { return (__int128)((unsigned __int128)1 << 127); }
};

// Register shuffles of the key types (a 128-bit key moves as two words).
__device__ __forceinline__ float kshfl_xor(unsigned mask, float x, int o, int w = 32) {
    return __shfl_xor_sync(mask, x, o, w);
}
__device__ __forceinline__ __int128 kshfl_xor(unsigned mask, __int128 x, int o, int w = 32) {
    const unsigned long long lo = __shfl_xor_sync(mask, (unsigned long long)x, o, w);
    const long long hi = __shfl_xor_sync(mask, (long long)(x >> 64), o, w);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}
__device__ __forceinline__ float kshfl(unsigned mask, float x, int src, int w = 32) {
    return __shfl_sync(mask, x, src, w);
}
__device__ __forceinline__ __int128 kshfl(unsigned mask, __int128 x, int src, int w = 32) {
    const unsigned long long lo = __shfl_sync(mask, (unsigned long long)x, src, w);
    const long long hi = __shfl_sync(mask, (long long)(x >> 64), src, w);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// A 128-bit unsigned sum held as two words (lo, hi) in global memory:
// atomically add x, carrying into hi when lo wraps. Every addition that
// wraps lo adds exactly one carry, so the pair is the exact sum mod 2^128
// in any order.
__device__ __forceinline__ void atomic_add_u128(unsigned long long *p, unsigned __int128 x) {
    const unsigned long long lo = (unsigned long long)x;
    unsigned long long hi = (unsigned long long)(x >> 64);
    if (lo) {
        const unsigned long long old = atomicAdd(&p[0], lo);
        if (old + lo < old) hi += 1ULL;
    }
    if (hi) atomicAdd(&p[1], hi);
}


template <class A, class W> __device__ __forceinline__ A wconv(W w) { return (A)w; }

__device__ __forceinline__ void atomic_add_acc(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void atomic_add_acc(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_acc(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_acc(unsigned long long *p, unsigned long long v) { atomicAdd(p, v); }

// Running per-graph sum of one thread (sweep gains, move counts). In a batch
// of graphs the sum of the previous graph goes to its slot base[g] when the
// thread reaches a vertex of another graph; a single graph never flushes
// here and reduces per warp at the end of the sweep instead.
template <class V> struct GAcc {
    V v = 0;
    int32_t g = 0;
};
template <class V, class D>
__device__ __forceinline__ void gacc_add(GAcc<V> &acc, bool batch, int32_t g, V x, D *base) {
    if (batch && g != acc.g) {
        if (acc.v != (V)0) atomic_add_acc(&base[acc.g], (D)acc.v);
        acc.v = 0;
        acc.g = g;
    }
    acc.v += x;
}
template <class V, class D> __device__ __forceinline__ void gacc_flush(GAcc<V> &acc, D *base) {
    if (acc.v != (V)0) atomic_add_acc(&base[acc.g], (D)acc.v);
    acc.v = 0;
}

// The deterministic mode's gain sums: 128 bits per thread, flushed into
// per-graph slots of two words (lo, hi) at base + 2 g.
__device__ __forceinline__ void gacc_add(GAcc<unsigned __int128> &acc, bool batch, int32_t g, unsigned __int128 x,
                                         unsigned long long *base) {
    if (batch && g != acc.g) {
        if (acc.v) atomic_add_u128(base + 2 * (size_t)acc.g, acc.v);
        acc.v = 0;
        acc.g = g;
    }
    acc.v += x;
}
__device__ __forceinline__ void gacc_flush(GAcc<unsigned __int128> &acc, unsigned long long *base) {
    if (acc.v) atomic_add_u128(base + 2 * (size_t)acc.g, acc.v);
    acc.v = 0;
}
__device__ __forceinline__ unsigned __int128 warp_sum_u128(unsigned __int128 v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
        v += ((unsigned __int128)hi << 64) | lo;
    }
    return v;
}

// Σ reads: the async mode sees concurrent atomics from other SMs, so it reads
// through L2 (ld.global.cg); deterministic mode reads a snapshot.
template <class A> __device__ __forceinline__ A load_cg(const A *p) { return __ldcg(p); }

// Move keys (Eq. 2). Deterministic mode, Eq. 2 times 2m^2 (kscale = 2m), in
// 128 bits (each product is below (2m)^2):
//   key(c) = 2m K_{i->c} - K_i Sigma_c,  stay = 2m K_{i->d} - K_i (Sigma_d - K_i).
// Asynchronous mode, Eq. 2 times m (kscale = 1/2m):
//   key(c) = K_{i->c} - gamma K_i Sigma_c / 2m,  stay = K_{i->d} - gamma K_i (Sigma_d - K_i) / 2m.
// The vertex moves to c* iff key(c*) > stay; the gain key(c*) - stay is
// 2m^2 dQ (deterministic) or m dQ (asynchronous).
__device__ __forceinline__ __int128 move_key(long long two_m, long long kic, long long ki, long long sc, double) {
    return (__int128)two_m * kic - (__int128)ki * sc;
}
__device__ __forceinline__ float move_key(float inv2m, float kic, float ki, double sc, double gamma) {
    return kic - (float)gamma * ki * ((float)sc * inv2m);
}
__device__ __forceinline__ __int128 stay_key(long long two_m, long long kid, long long ki, long long sd, double) {
    return (__int128)two_m * kid - (__int128)ki * (sd - ki);
}
__device__ __forceinline__ float stay_key(float inv2m, float kid, float ki, double sd, double gamma) {
    return kid - (float)gamma * ki * (((float)sd - ki) * inv2m);
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number i+1 of the
// generator whose state starts at s. Vertex priorities of the sweep schedule.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t i) {
    uint64_t z = s + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// u precedes v in the schedule order: higher priority first, ties by id.
__device__ __forceinline__ bool precedes(uint64_t pu, int32_t u, uint64_t pv, int32_t v) {
    return pu > pv || (pu == pv && u < v);
}

// Open-addressing hash table with linear probing (keys -1 = empty).
__device__ __forceinline__ uint32_t hslot(int32_t key, int bits) {
    return ((uint32_t)key * 0x9E3779B1u) >> (32 - bits);
}
template <class A>
__device__ __forceinline__ bool hash_add(int32_t *keys, A *vals, int bits, int32_t k, A v) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hslot(k, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        int32_t cur = *((volatile int32_t *)&keys[s]);
        if (cur == k) {
            atomic_add_acc(&vals[s], v);
            return true;
        }
        if (cur == -1) {
            int32_t prev = atomicCAS(&keys[s], -1, k);
            if (prev == -1 || prev == k) {
                atomic_add_acc(&vals[s], v);
                return true;
            }
        }
        s = (s + 1u) & mask;
    }
    return false;
}

// Open-addressing table whose slot is one 8-byte word: the key in the low
// half (-1: empty), an fp32 value in the high half, so that an insertion
// touches one memory sector (the asynchronous mode's global tables). A new
// key goes in with its value by one 64-bit compare-and-swap against the
// empty word; a failed swap returns the slot's word, and if its key is ours
// the value is added to the high half. A slot's key never changes once set,
// so the key half of a returned word is exact even while other threads add
// to its value half.
constexpr unsigned long long kEmptyKV = 0x00000000ffffffffULL;  // key -1, value 0.0f
__device__ __forceinline__ bool hash_add_kv(unsigned long long *kv, int bits, int32_t k, float v) {
    const uint32_t mask = (1u << bits) - 1u;
    const unsigned long long mine = ((unsigned long long)__float_as_uint(v) << 32) | (uint32_t)k;
    uint32_t s = hslot(k, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = atomicCAS(&kv[s], kEmptyKV, mine);
        if (cur == kEmptyKV) return true;
        if ((int32_t)(uint32_t)cur == k) {
            atomicAdd(reinterpret_cast<float *>(&kv[s]) + 1, v);
            return true;
        }
        s = (s + 1u) & mask;
    }
    return false;
}

__device__ __forceinline__ int ceil_log2(int64_t x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Row i of a CSR against labels C: K_i (sum of weights) and the weight to
// vertices labelled ci, over entries [from, to) of the row with stride step.
__device__ __forceinline__ void row_part(const int32_t *idx, const float *w, const int32_t *C, int64_t e0,
                                         int64_t from, int64_t to, int step, int32_t ci, double &k, double &in) {
    for (int64_t e = e0 + from; e < e0 + to; e += step) {
        const double x = w ? (double)w[e] : 1.0;
        k += x;
        if (C[idx[e]] == ci) in += x;
    }
}
// the same for every lane's row of a full warp: short rows by their lane,
// rows longer than 64 entries (LONG) by the whole warp in turn (valid: the
// lane has a row)
template <bool LONG>
__device__ __forceinline__ void warp_rows(const int64_t *off, const int32_t *idx, const float *w, const int32_t *C,
                                          bool valid, int64_t i, int32_t ci, double &k, double &in) {
    const int lane = threadIdx.x & 31;
    int64_t e0 = 0, d = 0;
    if (valid) {
        e0 = off[i];
        d = off[i + 1] - e0;
        if (!LONG || d <= 64) row_part(idx, w, C, e0, 0, d, 1, ci, k, in);
    }
    unsigned longs = LONG ? __ballot_sync(kFull, valid && d > 64) : 0u;
    while (longs) {
        const int src = __ffs(longs) - 1;
        longs &= longs - 1;
        double kl = 0, il = 0;
        row_part(idx, w, C, __shfl_sync(kFull, e0, src), lane, __shfl_sync(kFull, d, src), 32,
                 __shfl_sync(kFull, ci, src), kl, il);
        kl = warp_sum(kl);
        il = warp_sum(il);
        if (lane == src) {
            k = kl;
            in = il;
        }
    }
}

// arr[key] += x for every lane of a full warp (key < 0: nothing), with one
// atomic per distinct key: lanes that share a key sum first. Cheap when a
// warp's keys repeat (labels of nearby vertices).
__device__ __forceinline__ void warp_add_by_key(double *arr, int64_t key, double x) {
    unsigned todo = __ballot_sync(kFull, key >= 0);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const int64_t k = __shfl_sync(kFull, key, lead);
        const unsigned same = __ballot_sync(kFull, key == k);
        const double s = warp_sum(key == k ? x : 0.0);
        if ((int)(threadIdx.x & 31) == lead && s != 0.0) atomicAdd(&arr[k], s);
        todo &= ~same;
    }
}

// Sum of v over the lanes of peers (every lane of peers calls it, with the
// same peers).
template <class A>
__device__ __forceinline__ A peer_sum(unsigned peers, A v) {
    if (peers == kFull) return warp_sum(v);
    A s = 0;
    for (unsigned m = peers; m; m &= m - 1) s += __shfl_sync(peers, v, __ffs(m) - 1);
    return s;
}

// Profiling counters: every lane holds partial counts; one atomic per warp.
struct ProfCounts {
    unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
    __device__ __forceinline__ void flush(unsigned long long *dst) {
        if (!dst) return;
        for (int k = 0; k < 6; ++k) {
            const unsigned long long s = warp_sum(v[k]);
            if ((threadIdx.x & 31) == 0 && s) atomicAdd(&dst[k], s);
        }
    }
};

// Device error word: kernels record the first failure here instead of
// trapping; the host reads it after each phase.
enum : int { kErrNone = 0, kErrHashFull = 1, kErrBadIndex = 2, kErrTimeout = 3 };
__device__ __forceinline__ void set_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// Grid-wide barrier of a cooperative launch. bar[0] counts the arrivals of
// the launch and bar[1] the barriers completed; both are zero when the launch
// begins (the launcher clears them). Thread 0 of each block arrives with a
// release add on bar[0]: an arrival that returns old learns its barrier
// r = old / G + 1 (no block arrives at barrier r + 1 before all G blocks
// arrived at barrier r), and the G-th arrival publishes r in bar[1] with a
// release store, which the others poll with acquire loads. Compared with
// resetting a counter and advancing a generation (three dependent atomics
// on the last arrival) this took a barrier of 608 blocks from 3.1 to 2.2
// microseconds on this GPU. Spins are bounded: after spin_limit polls (2^24,
// about a second, by default) without progress the kernel records
// kErrTimeout and every later barrier returns at once, so the launch always
// ends. A grid of one block needs only __syncthreads.
constexpr unsigned long long kSpinLimit = 1ULL << 24;
__device__ __forceinline__ unsigned bar_arrive(unsigned *p) {
    unsigned r;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(r) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ unsigned bar_poll(const unsigned *p) {
    unsigned r;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ void bar_publish(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, unsigned long long spin_limit = kSpinLimit) {
    __shared__ int s_ok;
    __syncthreads();
    if (gridDim.x == 1) return true;
    if (threadIdx.x == 0) {
        int ok = *((volatile int *)err) == 0;
        if (ok) {
            const unsigned G = gridDim.x;
            const unsigned old = bar_arrive(&bar[0]);
            const unsigned r = old / G + 1;
            if (old == r * G - 1) {
                bar_publish(&bar[1], r);
            } else {
                unsigned long long spins = 0;
                while (bar_poll(&bar[1]) < r) {
                    if (++spins > spin_limit) {
                        set_error(err, kErrTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace lgb
