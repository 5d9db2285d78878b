// Internals of the host engine shared by its translation units (engine.cu,
// serve.cu): the scalar block read back per phase, the state of one run,
// and the handle's device workspace.
#pragma once
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "engine.h"
#include "kernels.h"

namespace lgb {

namespace detail {

struct Scalars {  // device scalars, read back in one copy
    int err;
    int nonint;
    unsigned long long vsum[2];
    double two_m_f;
    long long two_m_i;
    double dq_f;
    unsigned long long dq_i[2];  // deterministic gain sum: 128 bits, lo then hi
    unsigned long long moved;
    double wsum;
    double msum[4];
    int32_t maxdeg;
    int32_t iters;
    unsigned long long maxtdeg;
};

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t _e = (x);                                                              \
        if (_e != cudaSuccess) {                                                           \
            set_last_error(std::string(#x) + ": " + cudaGetErrorString(_e));              \
            return (_e == cudaErrorMemoryAllocation) ? LEIDEN_ERR_OOM : LEIDEN_ERR_CUDA;   \
        }                                                                                  \
    } while (0)
#define ST(x)                                  \
    do {                                       \
        leiden_status _s = (x);                \
        if (_s != LEIDEN_OK) return _s;        \
    } while (0)

// barrier polls before a persistent launch gives up (kSpinLimit of the
// device code, about a second)
constexpr unsigned long long kSpinLimitDefault = 1ULL << 24;

// allocations left before an injected failure (leiden_test_fail_allocation;
// negative: none)
extern std::atomic<int64_t> g_fail_alloc_after;

// the deterministic mode's bound on 2m (reading S1): weight sums are then
// exact in fp64, and every key and a sweep's sum of gains fit in 128 bits
constexpr double kDetMaxTwoM = 9007199254740992.0;  // 2^53

inline int ceil_log2_h(int64_t x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

}  // namespace detail
using namespace detail;

// State of one run (or one serving step) that the passes share.
struct Run {
    const leiden_params *prm = nullptr;
    bool det = false, trace = false, profile = false, batch = false;
    int32_t L = 0, B = 0, NG = 1;  // L: the largest layer cap of the run's graphs
    leiden_stats st{};
    std::vector<std::pair<cudaEvent_t, int>> marks;  // phase boundary events (phase id of the span that starts)
    GraphView G;                  // current graph G'
    int64_t Gcap = 0;             // entry capacity of G' (holey after aggregation)
    int cur_agg = 1;              // the next aggregation writes agg[cur_agg ^ 1]
    const int32_t *cur_gid = nullptr;  // graph of every vertex of G' (batches)
    double tau = 0;
    int passes = 0;
    bool no_edges = false;
    int64_t n0 = 0;               // vertices of the dendrogram C0
    int64_t deg_bound = INT64_MAX;  // bound on the degrees of G' (picks the long-row kernels)
    // graphs at different passes (serving): the first n_cont vertices of G'
    // continue with move-based labels, the others start as singletons;
    // gpass/gtau are per-graph pass indices and tolerances; a graph stops at
    // graph_max_passes
    int64_t n_cont = -1;
    const int32_t *gpass = nullptr;
    const double *gtau = nullptr;
    int32_t graph_max_passes = 0;
    const int32_t *gL = nullptr;  // layer cap of every graph (batches; L is the largest)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // start and end of a whole run

    Run() = default;
    Run(const Run &) = delete;
    Run &operator=(const Run &) = delete;
    ~Run() {  // the run's events go on every return path, errors included
        for (auto &m : marks) cudaEventDestroy(m.first);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

// One graph submitted to a serving handle.
struct Request {
    int64_t id = 0, n = 0, m = 0;
    // host copy while the graph waits for device memory
    std::vector<int64_t> hoff;
    std::vector<int32_t> hidx;
    std::vector<float> hw;
    bool on_device = false;
    int64_t *off = nullptr;  // device copy: offsets, local indices, weights
    int32_t *idx = nullptr;
    float *w = nullptr;
    int32_t *memb = nullptr;  // result: canonical labels
    int64_t bytes = 0;        // device bytes held
    int32_t L = 0;            // layer cap of its schedule (reading S0)
    // in flight
    int32_t pass = 0;
    int32_t fresh = 1;        // its next pass begins from singletons (reading R5')
    int64_t n_cur = 0;        // vertices in the union
    int64_t arena = 0;        // first entry in the dendrogram arena
    // result
    leiden_status status = LEIDEN_OK;
    double q = 0;
    int32_t passes = 0;
    int64_t communities = 0;
    int64_t fin_seq = 0;      // place in the server's finishing order
};

// Counters shared by the lanes of one server: request ids, the finishing
// order, and the device bytes charged against the one budget.
struct ServeShared {
    int64_t next_id = 1;
    int64_t fin_seq = 0;
    int64_t budget = 0, used = 0;  // device bytes of the requests' own buffers
};

// Serving state (continuous batching): graphs wait, join the union at a pass
// boundary when slots and memory allow, run one pass per step with the
// others, and leave with their results when they stop.
struct Serve {
    leiden_params prm{};
    int64_t cap_v = 0, cap_e = 0;  // union capacity: vertices (also the dendrogram arena), entries
    int32_t cap_g = 0;             // graphs in flight
    ServeShared own;               // counters when the union serves alone
    ServeShared *sh = &own;        // else those of the server it is a lane of
    std::map<int64_t, Request> reqs;
    std::deque<int64_t> waiting;   // submitted, not yet in the union (first come, first served)
    int32_t on_host = 0;           // waiting graphs still held on the host
    std::vector<int64_t> inflight; // in union order
    std::deque<int64_t> finished;  // results not yet read
    int64_t steps = 0;
    int64_t n_union = 0, e_union = 0, n_cont = 0, arena_n = 0;
    int cur = 0;                   // the union lives in agg[cur]
    int32_t *arena[2] = {nullptr, nullptr};
    int arena_cur = 0;
    int32_t *gpass = nullptr;
    double *gtau = nullptr;
    // host mirrors of the per-graph arrays of a step
    std::vector<int64_t> hvseg, hvseg0;
    std::vector<int32_t> hpass, hstate, hL, hfresh;
    std::vector<double> htau;
    int32_t *gL = nullptr;
};

struct Handle::Impl {
    int64_t n0 = 0, m0 = 0;
    leiden_tuning tune = [] {
        leiden_tuning t;
        tuning_default(t);
        return t;
    }();
    BinBounds bins() const {
        BinBounds b;
        b.thread_max = tune.thread_max_deg;
        b.warp_max = tune.warp_max_deg;
        b.block_max = tune.block_max_deg;
        return b;
    }
    int64_t maxdeg0 = INT64_MAX;  // largest degree of the input graph
    Serve *srv = nullptr;
    cudaStream_t s = nullptr;
    int sm = 152;
    bool nonint = false;
    double wsum = 0;
    // input CSR
    int64_t *off0 = nullptr;
    int32_t *idx0 = nullptr, *deg0 = nullptr;
    float *w0 = nullptr;
    // aggregated graphs (ping-pong)
    struct Agg {
        int64_t *off = nullptr;
        int32_t *deg = nullptr, *idx = nullptr;
        void *w = nullptr;
        int64_t cap = 0;
        int wsz = 0;  // bytes per weight: 4 (fp32) or 8 (WInt)
    } agg[2];
    // per-vertex workspace
    int32_t *C0 = nullptr, *Cp = nullptr, *CB = nullptr, *Cd = nullptr, *size = nullptr, *prop = nullptr,
            *step = nullptr, *key = nullptr, *list = nullptr, *flag = nullptr, *members = nullptr, *cursor = nullptr,
            *bnd = nullptr, *rep = nullptr, *label = nullptr, *minv = nullptr, *out = nullptr, *scnt = nullptr,
            *slayer = nullptr, *sfcount = nullptr, *act = nullptr;
    int64_t *pos = nullptr, *pos2 = nullptr, *coff = nullptr, *cnt = nullptr, *tdeg = nullptr, *key_cnt = nullptr,
            *key_off = nullptr;
    int64_t *tnm = nullptr, *tmoff = nullptr, *teoff = nullptr;  // bin-6 aggregation: member counts and scans
    void *K = nullptr, *Sig = nullptr, *Kagg = nullptr, *scan_tmp = nullptr, *part_tmp = nullptr;
    long long *gain = nullptr;
    uint8_t *unproc = nullptr;
    double *sigtot = nullptr;
    Scalars *dsc = nullptr, *hsc = nullptr;
    // hub tables
    int32_t *hub_keys = nullptr;
    void *hub_vals = nullptr;
    size_t hub_bytes = 0;
    int key_cap = 0;
    std::vector<int64_t> hkey_off;
    long long launches = 0;
    // trace
    std::map<std::pair<int, int>, std::vector<char>> trace;
    std::map<std::pair<int, int>, int64_t> trace_count;
    std::vector<void *> allocs;
    // profiling (LEIDEN_FLAG_PROFILE)
    unsigned long long *prof_cnt = nullptr;  // LEIDEN_PROFILE_CLASSES x kProfCounters
    unsigned *bar = nullptr;                 // grid barrier of the persistent sweep kernel
    long long *phase_dq = nullptr;           // per-sweep sums of a persistent phase
    unsigned long long *phase_moved = nullptr;
    int32_t phase_cap = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_spans;  // (class, index of the start event)
    std::vector<int64_t> prof_launches;
    leiden_kernel_profile prof_out[LEIDEN_PROFILE_CLASSES];
    bool prof_valid = false;
    bool prof_det = false;
    // batch of graphs (per-vertex graph ids only when G > 1)
    int32_t G = 1;
    std::vector<int64_t> hvseg0;           // vertex offsets of the graphs in the input
    std::vector<double> hgw;               // weight sum of every graph (fp64)
    std::vector<int32_t> hgmaxdeg;         // largest degree of every graph
    std::vector<int64_t> hgnnz;            // CSR entries of every graph
    int32_t *gL = nullptr;                 // layer cap of every graph (device)
    int64_t *vseg0 = nullptr, *vseg = nullptr, *vseg2 = nullptr;  // G+1 each: input, this pass, next pass
    int32_t *gid0 = nullptr, *gidA = nullptr, *gidB = nullptr;
    int32_t *gstate = nullptr, *gdone = nullptr, *gli = nullptr, *glj = nullptr, *gpasses = nullptr,
            *gfresh = nullptr;  // gfresh: the graph's pass began from singletons (reading R5')
    int64_t *gkeep = nullptr, *gcomm = nullptr;
    unsigned long long *gzero = nullptr;  // vertices without edges of every graph (reading R4)
    long long *gsumk = nullptr;            // per-graph sums of K (int64 or fp64 bits)
    long long *gks = nullptr;              // per-graph key scale (int64 2m or fp32 1/2m)
    double *g2m = nullptr, *gq = nullptr, *gmsum = nullptr;
    unsigned *gactive = nullptr;
    std::vector<int32_t> hpasses;          // per graph, after a run
    std::vector<int64_t> hcomm;

    leiden_status pass(Run &r, int32_t lp, bool &stop);
    // per-sweep sums of a persistent phase: max_it x ng
    leiden_status ensure_phase(int32_t max_it, int32_t ng) {
        if (max_it <= phase_cap) return LEIDEN_OK;
        if (phase_dq) free_one(phase_dq);
        if (phase_moved) free_one(phase_moved);
        if (gactive) free_one(gactive);
        phase_dq = nullptr;
        phase_moved = nullptr;
        gactive = nullptr;
        phase_cap = 0;  // nothing held until every array is in place
        ST(alloc(&phase_dq, 2 * (int64_t)max_it * ng));  // deterministic sums take two words
        ST(alloc(&phase_moved, (int64_t)max_it * ng));
        ST(alloc(&gactive, max_it));
        phase_cap = max_it;
        return LEIDEN_OK;
    }
    // the current device, its SM count, the stream-ordered pool (kept warm)
    // and the scalar block
    leiden_status init_device() {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
        cudaMemPool_t pool;
        CK(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t thr = UINT64_MAX;
        CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        CK(cudaMallocHost(&hsc, sizeof(Scalars)));
        ST(alloc(&dsc, 1));
        CK(cudaMemsetAsync(dsc, 0, sizeof(Scalars), s));
        return LEIDEN_OK;
    }
    // workspace for graphs of up to n vertices (later graphs are smaller) and
    // per-graph state for ng graphs
    leiden_status alloc_workspace(int64_t n, int32_t ng) {
        for (int32_t **a : {&C0, &Cp, &CB, &Cd, &size, &prop, &step, &key, &list, &flag, &members, &cursor, &bnd,
                            &rep, &label, &minv, &out, &scnt, &slayer})
            ST(alloc(a, n));
        for (int64_t **a : {&pos, &pos2, &coff, &tnm, &tmoff, &teoff}) ST(alloc(a, n + 1));
        for (int64_t **a : {&cnt, &tdeg}) ST(alloc(a, n));
        long long *k1, *k2, *k3;
        ST(alloc(&k1, n));
        ST(alloc(&k2, n));
        ST(alloc(&k3, n));
        K = k1;
        Sig = k2;
        Kagg = k3;
        ST(alloc(&gain, 2 * n));  // a deterministic gain takes two words
        ST(alloc(&unproc, n));
        ST(alloc(&sigtot, n));
        char *tmp;
        ST(alloc(&tmp, (int64_t)scan_tmp_bytes((n > ng ? n : ng) + 8192)));
        scan_tmp = tmp;
        ST(ensure_part_tmp(partition_tmp_bytes(n, (32 - 1 + 16) * kNumBins + 1)));  // default schedule
        ST(alloc(&prof_cnt, (int64_t)LEIDEN_PROFILE_CLASSES * kProfCounters));
        ST(alloc(&bar, 2));
        CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
        key_cap = 8192;
        ST(alloc(&key_cnt, key_cap));
        ST(alloc(&key_off, key_cap + 1));
        ST(alloc(&sfcount, 4096 + 1));
        ST(alloc(&act, 1024));
        CK(cudaMemsetAsync(act, 0, sizeof(int32_t) * 1024, s));
        for (int64_t **a : {&vseg0, &vseg, &vseg2}) ST(alloc(a, ng + 1));
        for (int32_t **a : {&gstate, &gdone, &gli, &glj, &gpasses, &gfresh}) ST(alloc(a, ng));
        for (int64_t **a : {&gkeep, &gcomm}) ST(alloc(a, ng));
        ST(alloc(&gzero, ng));
        ST(alloc(&gsumk, ng));
        ST(alloc(&gks, ng));
        ST(alloc(&g2m, ng));
        ST(alloc(&gq, ng));
        ST(alloc(&gmsum, 3 * (int64_t)ng));
        return LEIDEN_OK;
    }
    // brackets one profiled launch of class cls with events on the run's stream
    unsigned long long *prof_begin(Run &r, int cls) {
        if (!r.profile) return nullptr;
        prof_spans.push_back({cls, ev_used});
        cudaEventRecord(next_event(), s);
        prof_launches[cls]++;
        return prof_cnt + (size_t)cls * kProfCounters;
    }
    void prof_end(Run &r) {
        if (r.profile) cudaEventRecord(next_event(), s);
    }
    // phase boundary for the per-phase times of the statistics
    leiden_status mark(Run &r, int phase) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        r.marks.push_back({e, phase});  // owned by the run from here
        CK(cudaEventRecord(e, s));
        return LEIDEN_OK;
    }
    cudaEvent_t next_event() {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }

    ~Impl() {
        if (srv) {
            for (auto &kv : srv->reqs)
                for (void *b : {(void *)kv.second.off, (void *)kv.second.idx, (void *)kv.second.w,
                                (void *)kv.second.memb})
                    if (b) cudaFreeAsync(b, s);
            delete srv;
        }
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (void *p : allocs) cudaFreeAsync(p, s);
        if (hsc) cudaFreeHost(hsc);
        cudaStreamSynchronize(s);
    }
    template <class T> leiden_status alloc(T **p, int64_t count) {
        void *q = nullptr;
        if (g_fail_alloc_after.load() >= 0 && g_fail_alloc_after.fetch_sub(1) == 0) {
            set_last_error("injected device allocation failure (leiden_test_fail_allocation)");
            return LEIDEN_ERR_OOM;
        }
        cudaError_t e = cudaMallocAsync(&q, (size_t)(count > 0 ? count : 1) * sizeof(T), s);
        if (e != cudaSuccess) {
            set_last_error(std::string("device allocation of ") + std::to_string(count * (int64_t)sizeof(T)) +
                           " bytes failed: " + cudaGetErrorString(e));
            return LEIDEN_ERR_OOM;
        }
        allocs.push_back(q);
        *p = static_cast<T *>(q);
        return LEIDEN_OK;
    }
    leiden_status free_one(void *p) {
        for (size_t i = 0; i < allocs.size(); ++i)
            if (allocs[i] == p) {
                cudaFreeAsync(p, s);
                allocs.erase(allocs.begin() + i);
                break;
            }
        return LEIDEN_OK;
    }
    leiden_status sync_scalars() {
        CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hsc->err) {
            const int code = hsc->err;
            set_last_error(code == 3 ? "a grid barrier of the persistent sweep kernel timed out"
                                     : "device error word " + std::to_string(code));
            return code == 3 ? LEIDEN_ERR_TIMEOUT : LEIDEN_ERR_CUDA;
        }
        return LEIDEN_OK;
    }
    template <class T> void record(int pass, int what, const T *dev, int64_t count) {
        std::vector<char> buf((size_t)count * sizeof(T));
        if (count > 0) {
            cudaMemcpyAsync(buf.data(), dev, buf.size(), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
        }
        trace[{pass, what}] = std::move(buf);
        trace_count[{pass, what}] = count;
    }
    leiden_status ensure_hub(int bits, int regions, bool det) {
        const size_t per = ((size_t)1 << bits) * (sizeof(int32_t) + 8);
        const size_t need = per * (size_t)regions;
        if (need <= hub_bytes) return LEIDEN_OK;
        if (hub_keys) free_one(hub_keys);
        if (hub_vals) free_one(hub_vals);
        hub_keys = nullptr;
        hub_vals = nullptr;
        hub_bytes = 0;
        ST(alloc(&hub_keys, ((int64_t)1 << bits) * regions));
        char *v = nullptr;
        ST(alloc(&v, ((int64_t)1 << bits) * regions * 8));
        hub_vals = v;
        hub_bytes = need;
        (void)det;
        return LEIDEN_OK;
    }
    // Sum the event spans per class and turn the work counters into
    // algorithmic bytes (element sizes of what each kernel reads and writes).
    leiden_status finish_profile() {
        std::vector<unsigned long long> c((size_t)LEIDEN_PROFILE_CLASSES * kProfCounters);
        CK(cudaMemcpyAsync(c.data(), prof_cnt, c.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::memset(prof_out, 0, sizeof(prof_out));
        for (auto &sp : prof_spans) {
            float t = 0;
            cudaEventElapsedTime(&t, ev_pool[sp.second], ev_pool[sp.second + 1]);
            prof_out[sp.first].ms += t;
        }
        for (int k = 0; k < LEIDEN_PROFILE_CLASSES; ++k) {
            const unsigned long long *v = &c[(size_t)k * kProfCounters];
            leiden_kernel_profile &o = prof_out[k];
            o.launches = prof_launches[k];
            const int phase = k / 8;
            if (phase < 2) {
                o.items = (int64_t)v[0];
                o.skipped = (int64_t)v[1];
                o.edges = (int64_t)v[2];
                o.distinct = (int64_t)v[3];
                o.moved = (int64_t)v[4];
                const double ksz = prof_det ? 8.0 : 4.0;  // K' is int64 or fp32
                if (phase == 0)  // list, flag r/w, C, K, offset, degree, Sigma_d | idx, w, C[j] | Sigma_c | move
                    o.bytes = (30.0 + ksz) * v[0] + 5.0 * v[1] + 12.0 * v[2] + 8.0 * v[3] + 28.0 * v[4] + 1.0 * v[5];
                else  // + bound C'_B of i and of every neighbour, isolation test, proposal write
                    o.bytes = (40.0 + ksz) * v[0] + 16.0 * v[1] + 16.0 * v[2] + 8.0 * v[3];
            } else {
                o.items = (int64_t)v[0];
                o.edges = (int64_t)v[2];
                o.moved = (int64_t)v[3];
                o.skipped = 0;
                o.distinct = (int64_t)v[3];
                // community: list, offsets in/out, fill, K''; member: id, offset, degree;
                // edge: idx, w, label; written entry: idx, w
                o.bytes = 48.0 * v[0] + 16.0 * v[1] + 12.0 * v[2] + 8.0 * v[3];
            }
        }
        prof_valid = true;
        return LEIDEN_OK;
    }
    // whole-grid bin 6 of the persistent sweep: per-hub arrays of a pass
    int32_t *hubs = nullptr, *hd = nullptr, *hcand = nullptr, *hmv = nullptr, *hj = nullptr;
    int64_t *htoff = nullptr, *heoff = nullptr, *hinfo = nullptr;
    unsigned long long *hkey = nullptr, *hspan = nullptr;
    long long *hkvd = nullptr;
    int64_t hubs_cap = -1;
    // the rows and vertex weights of a pass's graph in list order
    // (leiden_tuning.list_order_min_vertices): offsets (nv + 1), row
    // lengths (nv), entries (ne, weights of wsz bytes) and weights (asz bytes)
    int64_t *lo_off = nullptr;
    int32_t *lo_len = nullptr, *lo_idx = nullptr;
    void *lo_w = nullptr, *lo_K = nullptr;
    int64_t lo_cap_v = 0, lo_cap_e = 0;
    leiden_status ensure_list_order(int64_t nv, int64_t ne) {
        if (nv > lo_cap_v) {
            for (void *p : {(void *)lo_off, (void *)lo_len, lo_K})
                if (p) free_one(p);
            lo_off = nullptr;
            lo_len = nullptr;
            lo_K = nullptr;
            lo_cap_v = 0;
            ST(alloc(&lo_off, nv + 1));
            ST(alloc(&lo_len, nv));
            long long *k = nullptr;
            ST(alloc(&k, nv));  // 8 bytes: int64 (deterministic) or fp32 weights
            lo_K = k;
            lo_cap_v = nv;
        }
        if (ne > lo_cap_e) {
            for (void *p : {(void *)lo_idx, lo_w})
                if (p) free_one(p);
            lo_idx = nullptr;
            lo_w = nullptr;
            lo_cap_e = 0;
            ST(alloc(&lo_idx, ne > 0 ? ne : 1));
            long long *w = nullptr;
            ST(alloc(&w, ne > 0 ? ne : 1));  // 8 bytes: WInt or fp32 weights
            lo_w = w;
            lo_cap_e = ne;
        }
        return LEIDEN_OK;
    }
    leiden_status ensure_hubs(int64_t nh) {
        if (!hinfo) {
            ST(alloc(&hinfo, 4));  // a step's eligible hubs, table slots, entries
            ST(alloc(&hspan, 1));
        }
        if (nh <= hubs_cap) return LEIDEN_OK;
        for (void *p : {(void *)hubs, (void *)hd, (void *)hcand, (void *)hmv, (void *)hj, (void *)htoff,
                        (void *)heoff, (void *)hkey, (void *)hkvd})
            if (p) free_one(p);
        hubs = hd = hcand = hmv = hj = nullptr;
        htoff = heoff = nullptr;
        hkey = nullptr;
        hkvd = nullptr;
        hubs_cap = -1;
        for (int32_t **a : {&hubs, &hd, &hcand, &hmv, &hj}) ST(alloc(a, nh));
        ST(alloc(&htoff, nh + 1));
        ST(alloc(&heoff, nh + 1));
        ST(alloc(&hkey, 2 * nh));  // a deterministic key takes two words
        ST(alloc(&hkvd, nh));
        hubs_cap = nh;
        return LEIDEN_OK;
    }
    size_t part_tmp_bytes = 0;
    leiden_status ensure_part_tmp(size_t bytes) {
        if (bytes <= part_tmp_bytes) return LEIDEN_OK;
        if (part_tmp) free_one(part_tmp);
        part_tmp = nullptr;
        part_tmp_bytes = 0;
        char *p = nullptr;
        ST(alloc(&p, (int64_t)bytes));
        part_tmp = p;
        part_tmp_bytes = bytes;
        return LEIDEN_OK;
    }
    // aggregated graph x with room for cap entries, its weights fp32
    // (asynchronous) or WInt (deterministic)
    leiden_status ensure_agg(int x, int64_t cap, bool det) {
        Agg &a = agg[x];
        if (!a.off) {
            ST(alloc(&a.off, n0 + 1));
            ST(alloc(&a.deg, n0));
        }
        const int wsz = det ? (int)sizeof(WInt) : (int)sizeof(float);
        if (a.cap >= cap && a.idx && a.wsz >= wsz) return LEIDEN_OK;
        if (a.cap < cap && a.idx) {
            free_one(a.idx);
            a.idx = nullptr;
        }
        if (a.w) free_one(a.w);
        a.w = nullptr;
        a.wsz = 0;
        if (!a.idx) ST(alloc(&a.idx, cap));
        a.cap = a.cap > cap ? a.cap : cap;
        char *w = nullptr;
        ST(alloc(&w, a.cap * wsz));
        a.w = w;
        a.wsz = wsz;
        return LEIDEN_OK;
    }
};

}  // namespace lgb
