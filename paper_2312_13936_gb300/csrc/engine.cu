// Host engine: one handle per graph or per batch of graphs. leiden_create
// copies the CSR to the device; leiden_run drives the pass loop of
// Algorithm 1 (local-moving, refinement, stop tests, renumbering, dendrogram
// lookup, aggregation, move-based labels, threshold scaling) with the kernels
// of kernels.h. All state stays on the device; each phase is one persistent
// launch that tests convergence itself, and per pass the host reads back a
// handful of counts.
//
// A batch of G graphs runs as one disjoint union: one set of launches per
// pass serves every graph, each graph keeps its own 2m, convergence tests,
// stop tests and pass count (per-graph arrays of k_batch.cu), and a graph
// that stops leaves the union at the next renumbering. A single graph is the
// case G = 1 without per-vertex graph ids.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "engine_impl.h"

namespace lgb {

thread_local std::string g_last_error;
std::atomic<int64_t> detail::g_fail_alloc_after{-1};  // leiden_test_fail_allocation
void set_last_error(const std::string &s) { g_last_error = s; }
const char *last_error() { return g_last_error.c_str(); }

// The persistent sweeps' grid barrier counts arrivals in 32 bits, from zero
// at every launch. One phase takes at most max_iterations sweeps of at most
// 8 barriers per schedule step (layout, insertion, three key passes, hub
// flags, step end, apply) and 4 more per sweep, on at most the resident
// grid; a limit under which that count could pass 2^32 - 1 is refused
// rather than let the count wrap.
leiden_status check_barrier_budget(int32_t max_iterations, int32_t nsteps, bool det, int sm) {
    int per_sm = 0;
    for (int w = 0; w < 2; ++w)
        for (int r = 0; r < 2; ++r) {
            const int b = sweep_coop_blocks_per_sm(det, w != 0, r != 0);
            per_sm = b > per_sm ? b : per_sm;
        }
    const int64_t arrivals = (int64_t)max_iterations * (8 * (int64_t)nsteps + 4) * per_sm * sm;
    if (arrivals > (int64_t)0xffffffffLL) {
        set_last_error("max_iterations too large for this schedule: one phase could take more than 2^32 - 1 "
                       "grid-barrier arrivals");
        return LEIDEN_ERR_INVALID;
    }
    return LEIDEN_OK;
}

Handle::Handle() : p(new Impl) {}
Handle::~Handle() { delete p; }

leiden_status Handle::create(int64_t n, int64_t nnz, const int64_t *offsets, const int32_t *indices,
                             const float *weights, int where, int validate, void *stream, int32_t num_graphs,
                             const int64_t *vtx_seg) {
    Impl &q = *p;
    q.s = static_cast<cudaStream_t>(stream);
    q.n0 = n;
    q.m0 = nnz;
    q.G = num_graphs;
    if (vtx_seg) q.hvseg0.assign(vtx_seg, vtx_seg + num_graphs + 1);
    else q.hvseg0 = {0, n};
    ST(q.init_device());
    ST(q.alloc(&q.off0, n + 1));
    ST(q.alloc(&q.idx0, nnz));
    ST(q.alloc(&q.w0, nnz));
    ST(q.alloc(&q.deg0, n));
    const cudaMemcpyKind kind = where == LEIDEN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(q.off0, offsets, sizeof(int64_t) * (n + 1), kind, q.s));
    if (nnz > 0) CK(cudaMemcpyAsync(q.idx0, indices, sizeof(int32_t) * nnz, kind, q.s));
    if (nnz > 0) {
        if (weights) CK(cudaMemcpyAsync(q.w0, weights, sizeof(float) * nnz, kind, q.s));
        else CK(launch_fill_i32(reinterpret_cast<int32_t *>(q.w0), 0x3f800000, nnz, q.s));  // unit weights: 1.0f
    }
    ST(q.alloc_workspace(n, num_graphs));
    CK(launch_degrees(q.off0, q.deg0, n, &q.dsc->err, q.s));
    CK(launch_max_i32(q.deg0, n, &q.dsc->maxdeg, q.s));
    const int32_t G = q.G;
    CK(cudaMemcpyAsync(q.vseg0, q.hvseg0.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, q.s));
    if (G > 1) {
        for (int32_t **a : {&q.gid0, &q.gidA, &q.gidB}) ST(q.alloc(a, n));
        CK(launch_graph_ids(q.vseg0, G, n, q.gid0, q.s));
        // indices arrive local to each graph
        CK(launch_globalize_indices(q.vseg0, q.gid0, n, q.off0, nnz, q.idx0, &q.dsc->err, q.s));
    }
    if (validate) CK(launch_validate(n, q.off0, q.idx0, q.w0, &q.dsc->err, q.s));
    CK(cudaMemsetAsync(&q.dsc->wsum, 0, sizeof(double), q.s));
    CK(launch_weight_props(q.w0, nnz, &q.dsc->nonint, &q.dsc->wsum, q.s));
    CK(cudaMemcpyAsync(q.hsc, q.dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, q.s));
    CK(cudaStreamSynchronize(q.s));
    if (q.hsc->err) {
        const int e = q.hsc->err;
        set_last_error(e == 2 ? "CSR is not symmetric (w_ij != w_ji)" : "malformed CSR (offsets, indices or weights)");
        return e == 2 ? LEIDEN_ERR_NOT_SYMMETRIC : LEIDEN_ERR_INVALID;
    }
    q.nonint = q.hsc->nonint != 0;
    q.wsum = q.hsc->wsum;
    q.maxdeg0 = q.hsc->maxdeg;
    // launch shape from the autotuner cache named by LEIDEN_TUNING_CACHE,
    // for this GPU and this graph's class (the defaults otherwise)
    if (const char *cache = std::getenv("LEIDEN_TUNING_CACHE")) {
        int dev = 0;
        cudaDeviceProp prop;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
            leiden_tuning t;
            const std::string keep = last_error();
            if (tuning_lookup(cache, prop.name, n, nnz, q.maxdeg0, t) == LEIDEN_OK) q.tune = t;
            set_last_error(keep);
        }
    }
    if (G > 1) {  // weight sum of every graph, for the deterministic mode's 2m < 2^53 rule
        GraphView g0;
        g0.n = n;
        g0.off = q.off0;
        g0.deg = q.deg0;
        g0.idx = q.idx0;
        g0.w = q.w0;
        CK(cudaMemsetAsync(q.gmsum, 0, sizeof(double) * G, q.s));
        CK(cudaMemsetAsync(&q.dsc->wsum, 0, sizeof(double), q.s));
        CK(launch_vertex_weights(g0, false, q.K, &q.dsc->wsum, q.s));  // fp32 row sums into K
        CK(launch_graph_sums(q.K, false, q.gid0, n, q.gmsum, q.s));
        q.hgw.assign(G, 0.0);
        CK(cudaMemcpyAsync(q.hgw.data(), q.gmsum, sizeof(double) * G, cudaMemcpyDeviceToHost, q.s));
        // largest degree and entry count of every graph (the default layer
        // cap of its schedule, reading S0)
        q.hgnnz.assign(G, 0);
        CK(launch_graph_counts(q.off0, q.vseg0, G, q.gcomm, q.s));
        CK(cudaMemcpyAsync(q.hgnnz.data(), q.gcomm, sizeof(int64_t) * G, cudaMemcpyDeviceToHost, q.s));
        ST(q.alloc(&q.gL, G));
        CK(cudaMemsetAsync(q.gL, 0, sizeof(int32_t) * G, q.s));
        CK(launch_graph_max_deg(q.deg0, q.gid0, n, q.gL, q.s));
        q.hgmaxdeg.assign(G, 0);
        CK(cudaMemcpyAsync(q.hgmaxdeg.data(), q.gL, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, q.s));
        CK(cudaStreamSynchronize(q.s));
    }
    return LEIDEN_OK;
}

// One pass of Algorithm 1 over the current graph G' (every graph of a
// batch at once): vertex weights, schedule, local-moving, refinement, the
// stop tests, renumbering, dendrogram lookup and, for the graphs that go on,
// aggregation and move-based labels. Sets stop when no graph goes on.
leiden_status Handle::Impl::pass(Run &r, int32_t lp, bool &stop) {
    Impl &q = *this;
    cudaStream_t s = q.s;
    const leiden_params &prm = *r.prm;
    const bool det = r.det, trace = r.trace, batch = r.batch;
    const int32_t L = r.L, B = r.B, NG = r.NG;
    const int64_t n0 = r.n0;
    const int tile_blocks = q.sm * 8, big_blocks = q.sm * 2;
    GraphView &G = r.G;
    int64_t &Gcap = r.Gcap;
    int &cur_agg = r.cur_agg;
    const int32_t *&cur_gid = r.cur_gid;
    double &tau = r.tau;
    int &passes = r.passes;
    bool &no_edges = r.no_edges;
    leiden_stats &st = r.st;
    const size_t accsz = 8;
    auto mark = [&](int phase) { return q.mark(r, phase); };
    auto prof_begin = [&](int cls) { return q.prof_begin(r, cls); };
    auto prof_end = [&]() { q.prof_end(r); };
    stop = false;

    const int64_t n = G.n;
    if (n == 0) {
        stop = true;
        return LEIDEN_OK;
    }
    ST(mark(3));
    // vertexWeights(G') and 2m (of every graph of a batch)
    CK(cudaMemsetAsync(&q.dsc->two_m_f, 0, sizeof(double) + sizeof(long long), s));
    CK(launch_vertex_weights(G, det, q.K, det ? (void *)&q.dsc->two_m_i : (void *)&q.dsc->two_m_f, s));
    if (batch) {
        CK(cudaMemsetAsync(q.gsumk, 0, sizeof(long long) * NG, s));
        CK(launch_graph_sums(q.K, det, cur_gid, n, q.gsumk, s));
        CK(launch_graph_scales(q.gsumk, det, NG, q.gks, q.g2m, s));
        q.launches += 2;
    } else {
        CK(launch_graph_scales(det ? (void *)&q.dsc->two_m_i : (void *)&q.dsc->two_m_f, det, 1, q.gks, q.g2m, s));
        q.launches += 1;
    }
    q.launches += 2;  // the vertex weights' two kernels
    // schedule and (step, bin) lists
    // (the schedule's order arrays are the list and key buffers, rewritten below)
    SchedWork sw{q.scnt, q.slayer, q.list, q.key, q.sfcount, &q.dsc->err};
    CK(launch_schedule(G, prm.seed + (r.gpass ? 0 : (uint64_t)lp), L, B, sw, q.step, s, cur_gid,
                       batch ? q.vseg : nullptr, r.gpass, r.deg_bound > kLongRow, batch ? r.gL : nullptr));
    q.launches += 1;
    // steps used: the layers produced, then the buckets if any vertex was
    // not placed below L-1 (only steps that can hold vertices get lists)
    int32_t sinfo[2] = {0, 0};
    CK(cudaMemcpyAsync(sinfo, q.sfcount + 9, sizeof(sinfo), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int32_t nsteps = sinfo[1] > 0 ? L - 1 + B : std::max<int32_t>(1, std::min<int32_t>(sinfo[0], L - 1));
    const int32_t nkeys = nsteps * kNumBins;
    ST(q.ensure_part_tmp(partition_tmp_bytes(n, nkeys + 1)));
    // one vertex list per (schedule step, degree bin), step-major
    CK(launch_step_bin_keys(q.step, G.deg, n, nsteps, false, q.bins(), q.key, s));
    CK(launch_partition(q.key, n, nkeys + 1, q.key_off, q.list, q.part_tmp, s));  // + edgeless bucket
    CK(launch_max_i32(G.deg, n, &q.dsc->maxdeg, s));
    q.launches += 7;
    q.hkey_off.assign(nkeys + 2, 0);
    CK(cudaMemcpyAsync(q.hkey_off.data(), q.key_off, sizeof(int64_t) * (nkeys + 2), cudaMemcpyDeviceToHost, s));
    ST(q.sync_scalars());
    const double two_m_f = q.hsc->two_m_f;
    const long long two_m_i = q.hsc->two_m_i;
    if (!batch && (det ? (two_m_i == 0) : !(two_m_f > 0))) {  // reading R12: no edges
        CK(launch_iota(q.Cp, n, s));
        no_edges = true;
        passes++;
        stop = true;
        return LEIDEN_OK;
    }
    passes++;
    // C' and Sigma' at the start of local-moving (reading R3)
    if (r.n_cont >= 0) CK(launch_init_labels(q.label, r.n_cont, n, q.Cp, s));
    else if (lp == 0) CK(launch_iota(q.Cp, n, s));
    else CK(cudaMemcpyAsync(q.Cp, q.label, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    if (trace) q.record(lp, 1, q.Cp, n);
    // the sweeps' graph and arrays
    const GraphView sG = G;
    int32_t *sC = q.Cp, *sCB = q.CB, *sStep = q.step;
    const int32_t *sList = q.list;
    void *sK = q.K;
    CK(cudaMemsetAsync(q.Sig, 0, accsz * n, s));
    CK(cudaMemsetAsync(q.size, 0, sizeof(int32_t) * n, s));
    CK(launch_community_totals(sC, sK, det, n, q.Sig, q.size, s));
    q.launches += 1;
    const bool step_launches = (prm.flags & LEIDEN_FLAG_STEP_LAUNCHES) != 0;
    // bin 6: in the persistent sweep the whole grid takes each step's hubs
    // (tables of one step at a time); per-step launches keep a global table
    // per block
    const std::vector<int64_t> &ko = q.hkey_off;
    int64_t nhubs = 0;
    for (int32_t k = 0; k < nsteps; ++k) nhubs += ko[(size_t)k * kNumBins + 7] - ko[(size_t)k * kNumBins + 6];
    const bool grid_hubs = nhubs > 0 && !step_launches && sweep_coop_blocks_per_sm(det, sG.w_int, false) > 0 &&
                           sweep_coop_blocks_per_sm(det, sG.w_int, true) > 0;
    if (grid_hubs) {
        ST(q.ensure_hubs(nhubs));
        CK(launch_hub_prep(q.key_off, nsteps, sList, sG.deg, q.hubs, q.hspan, s));
        q.launches += 1;
        unsigned long long span = 0;
        CK(cudaMemcpyAsync(&span, q.hspan, sizeof(span), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (span > (unsigned long long)INT32_MAX) {
            set_last_error("hub tables of one step exceed 2^31 slots");
            return LEIDEN_ERR_OOM;
        }
        ST(q.ensure_hub(0, (int)span, det));
        // clean tables; every step's last scan leaves them clean again. The
        // asynchronous mode keeps key and fp32 value in one 8-byte word per
        // slot (key -1 and value 0 when empty), in the value buffer.
        if (det) {
            CK(cudaMemsetAsync(q.hub_keys, 0xff, sizeof(int32_t) * span, s));
            CK(cudaMemsetAsync(q.hub_vals, 0, 8 * span, s));
        } else {
            CK(launch_fill_u64(static_cast<unsigned long long *>(q.hub_vals), 0x00000000ffffffffULL, (int64_t)span,
                               s));
            q.launches += 1;
        }
    }
    // global tables for bin 6 (one per block)
    int hub_bits = 0, hub_regions = 0;
    if (!grid_hubs) {
        const int maxdeg = q.hsc->maxdeg;
        if (maxdeg > q.tune.block_max_deg) {
            hub_bits = ceil_log2_h(2 * (int64_t)maxdeg);
            const size_t per = ((size_t)1 << hub_bits) * 12;
            hub_regions = (int)std::max<size_t>(1, std::min<size_t>((size_t)q.sm, ((size_t)4 << 30) / per));
            ST(q.ensure_hub(hub_bits, hub_regions, det));
        }
    }
    // the rows and vertex weights in the order of the (step, bin) lists, so
    // that a sweep step reads them contiguously instead of one sector per
    // vertex spread over the whole graph (one graph without rows beyond the
    // block bin, from list_order_min_vertices vertices; values unchanged)
    const int64_t nl = q.hkey_off[(size_t)nkeys];
    const bool list_order = !batch && q.tune.list_order_min_vertices > 0 &&
                            n >= (int64_t)q.tune.list_order_min_vertices &&
                            (int64_t)q.hsc->maxdeg <= (int64_t)q.tune.block_max_deg && nl > 0;
    if (list_order) {
        ST(q.ensure_list_order(nl, 0));
        CK(launch_list_lens(q.list, nl, G.deg, q.lo_len, s));
        CK(launch_exclusive_scan_i32(q.lo_len, q.lo_off, nl, q.scan_tmp, s));
        int64_t ne = 0;
        CK(cudaMemcpyAsync(&ne, q.lo_off + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ST(q.ensure_list_order(nl, ne));
        CK(launch_list_rows(q.list, nl, G, q.K, det, q.lo_off, q.lo_idx, q.lo_w, q.lo_K, s));
        q.launches += 3;
    }
    SweepCtx sc;
    sc.g = sG;
    if (list_order) {
        sc.loff = q.lo_off;
        sc.lidx = q.lo_idx;
        sc.lw = q.lo_w;
        sc.lK = q.lo_K;
    }
    sc.det = det;
    sc.C = sC;
    sc.CB = sCB;
    sc.K = sK;
    sc.Sig = q.Sig;
    sc.size = q.size;
    sc.unproc = q.unproc;
    sc.prop = q.prop;
    sc.gain = q.gain;
    sc.step = sStep;
    sc.two_m_f = two_m_f;
    sc.two_m_i = two_m_i;
    sc.gamma = prm.resolution;
    sc.cap_step = L - 1;
    sc.dq_acc = det ? (void *)q.dsc->dq_i : (void *)&q.dsc->dq_f;
    sc.moved = &q.dsc->moved;
    sc.hub_keys = q.hub_keys;
    sc.hub_vals = q.hub_vals;
    sc.hub_bits = hub_bits;
    sc.err = &q.dsc->err;
    sc.grid_hubs = grid_hubs;
    sc.hubs = q.hubs;
    sc.hj = q.hj;
    sc.hinfo = q.hinfo;
    sc.htoff = q.htoff;
    sc.heoff = q.heoff;
    sc.hd = q.hd;
    sc.hcand = q.hcand;
    sc.hmv = q.hmv;
    sc.hkey = q.hkey;
    sc.hkvd = q.hkvd;
    sc.nsteps = nsteps;
    sc.key_off = q.key_off;
    sc.bar = q.bar;
    sc.block_max = q.tune.block_max_deg;
    sc.hub_regions = hub_regions;
    sc.gid = batch ? cur_gid : nullptr;
    sc.gks = q.gks;
    sc.g2m = q.g2m;
    sc.gdone = q.gdone;
    sc.gactive = q.gactive;
    sc.gtau = r.gtau;
    sc.G = NG;
    // one sweep as per-(step, bin) launches (fallback and test path)
    auto run_steps = [&](bool refine) -> leiden_status {
        sc.refine = refine;
        for (int32_t k = 0; k < nsteps; ++k) {
            sc.cur_step = k;
            const int64_t a0 = ko[k * kNumBins], a1 = ko[(k + 1) * kNumBins];
            if (a1 == a0) continue;
            for (int b = 1; b < kNumBins; ++b) {
                const int64_t lo = ko[k * kNumBins + b], hi = ko[k * kNumBins + b + 1];
                if (hi == lo) continue;
                const int mb = b <= 4 ? tile_blocks : (b == 5 ? big_blocks : hub_regions);
                sc.prof = prof_begin((refine ? 8 : 0) + b);
                CK(launch_sweep_eval(sc, b, sList + lo, hi - lo, mb, s));
                prof_end();
                q.launches++;
            }
            // apply phase: deterministic mode, and proposals where
            // neighbours may share a step (below the capped step the
            // asynchronous mode moves and joins at once)
            if (det || k >= sc.cap_step) {
                if (refine) CK(launch_refine_apply(sc, sList + a0, a1 - a0, s));
                else CK(launch_move_apply(sc, sList + a0, a1 - a0, s));
                q.launches++;
            }
        }
        return LEIDEN_OK;
    };
    // One phase (Algorithm 2 or 3): sweeps until convergence. Normally one
    // persistent cooperative launch that tests convergence on the device;
    // otherwise one host-driven sweep at a time. Returns the sweeps run.
    auto run_phase = [&](bool refine, int *iters, int32_t *giters) -> leiden_status {
        sc.refine = refine;
        // randomized refinement (asynchronous mode; run() refuses it otherwise)
        sc.rand_refine = refine && (prm.flags & LEIDEN_FLAG_RANDOM_REFINE) != 0;
        sc.rseed = prm.seed + 0xD1B54A32D192ED03ULL * (uint64_t)(64 * (r.gpass ? 0 : lp));
        const bool single = refine && (prm.flags & LEIDEN_FLAG_REFINE_SINGLE_SWEEP);
        int per_sm = step_launches ? 0 : sweep_coop_blocks_per_sm(det, sG.w_int, refine);
        if (per_sm > 0 && q.tune.coop_blocks_per_sm > 0 && q.tune.coop_blocks_per_sm < per_sm)
            per_sm = q.tune.coop_blocks_per_sm;  // the handle's launch shape
        CK(launch_phase_init(q.gstate, NG, q.gdone, giters, s));
        sc.giters = giters;
        if (batch && per_sm <= 0) {
            set_last_error("a batch of graphs needs the cooperative sweep kernel");
            return LEIDEN_ERR_UNSUPPORTED;
        }
        if (per_sm > 0) {
            // enough blocks for the graph (about vertices_per_block each),
            // so small graphs do not pay a full-GPU barrier per step and
            // graphs of one block synchronise with __syncthreads only
            int grid = per_sm * q.sm;
            const int64_t vpb = q.tune.vertices_per_block;
            const int64_t want = (n + vpb - 1) / vpb;
            if (want < grid) grid = (int)(want < 1 ? 1 : want);
            sc.hub_regions = hub_regions > grid ? grid : hub_regions;
            sc.max_it = prm.max_iterations;
            sc.single_sweep = single ? 1 : 0;
            sc.tau = tau;
            sc.dq_arr = q.phase_dq;
            sc.moved_arr = q.phase_moved;
            sc.iters_out = &q.dsc->iters;
            CK(cudaMemsetAsync(q.phase_dq, 0, 2 * sizeof(long long) * prm.max_iterations * NG, s));
            CK(cudaMemsetAsync(q.phase_moved, 0, sizeof(unsigned long long) * prm.max_iterations * NG, s));
            CK(cudaMemsetAsync(q.gactive, 0, sizeof(unsigned) * prm.max_iterations, s));
            CK(cudaMemsetAsync(q.bar, 0, 2 * sizeof(unsigned), s));  // barrier state starts clean
            sc.prof = prof_begin(refine ? 8 : 0);
            // steps without an eligible vertex are skipped where there are
            // many steps (heavy-tailed schedules): in the refinement, and in
            // the local-moving of a union of graphs, whose converged graphs
            // leave whole steps idle (for one graph the marks of flagged
            // neighbours cost about what they save)
            sc.act = (nsteps > 64 && (refine || batch)) ? q.act : nullptr;
            const bool stall = (prm.flags & LEIDEN_FLAG_TEST_STALL_BARRIER) != 0;
            sc.stall_block = (stall && grid > 1) ? 1 : -1;
            sc.spin_limit = stall ? (1ULL << 14) : kSpinLimitDefault;
            CK(launch_sweep_coop(sc, sList, grid, s));
            sc.act = nullptr;
            prof_end();
            q.launches++;
            ST(q.sync_scalars());
            *iters = q.hsc->iters;
            sc.hub_regions = hub_regions;
            return LEIDEN_OK;
        }
        int k = 0;
        for (int32_t it = 0; it < prm.max_iterations; ++it) {
            k++;
            CK(cudaMemsetAsync(&q.dsc->dq_f, 0, sizeof(double), s));
            CK(cudaMemsetAsync(q.dsc->dq_i, 0, sizeof(q.dsc->dq_i), s));
            CK(cudaMemsetAsync(&q.dsc->moved, 0, sizeof(unsigned long long), s));
            sc.sweep = it;
            ST(run_steps(refine));
            ST(q.sync_scalars());
            if (refine) {
                if (q.hsc->moved == 0 || single) break;
            } else {
                // reading S4: the 128-bit gain sum with the oracle's roundings
                const double dq = det ? 2.0 * u128_words_to_double(q.hsc->dq_i[0], q.hsc->dq_i[1]) /
                                            ((double)two_m_i * (double)two_m_i)
                                      : 2.0 * q.hsc->dq_f / two_m_f;
                if (dq <= tau) break;  // locally converged
            }
        }
        *iters = k;
        CK(launch_fill_i32(giters, k, 1, s));
        return LEIDEN_OK;
    };
    // ---- local-moving phase (Algorithm 2)
    ST(mark(0));
    CK(cudaMemsetAsync(q.unproc, 1, (size_t)n, s));  // mark all vertices unprocessed
    int li = 0;
    ST(run_phase(false, &li, q.gli));
    st.move_iterations += li;
    if (trace) q.record(lp, 2, q.Cp, n);
    // ---- refinement phase (Algorithm 3); the Louvain variant has none and
    // takes its local-moving communities as the refined ones
    ST(mark(1));
    CK(cudaMemcpyAsync(sCB, sC, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    int lj = 0;
    if (!(prm.flags & LEIDEN_FLAG_LOUVAIN)) {
        CK(launch_iota(sC, n, s));
        CK(cudaMemsetAsync(q.Sig, 0, accsz * n, s));
        CK(cudaMemsetAsync(q.size, 0, sizeof(int32_t) * n, s));
        CK(launch_community_totals(sC, sK, det, n, q.Sig, q.size, s));  // Sigma' <- K', one member each
        q.launches += 2;
        ST(run_phase(true, &lj, q.glj));
    }
    st.refine_iterations += lj;
    if (trace) q.record(lp, 3, q.Cp, n);
    // ---- stop tests (readings R4, R5')
    ST(mark(3));
    // non-empty refined communities: the labels present in C' (ids of G')
    CK(launch_fill_i32(q.flag, 0, n, s));
    CK(launch_mark_labels(q.Cp, n, q.flag, s));
    CK(launch_exclusive_scan_i32(q.flag, q.pos, n, q.scan_tmp, s));
    CK(launch_fill_i32(q.rep, 0, n, s));
    CK(launch_mark_labels(q.CB, n, q.rep, s));
    CK(launch_exclusive_scan_i32(q.rep, q.pos2, n, q.scan_tmp, s));
    // every graph takes Algorithm 1's two break tests on its own counts;
    // the graphs that go on keep their refined communities, densely
    // renumbered after those of the graphs before them
    CK(launch_graph_stop(q.vseg, q.pos, q.pos2, q.gli, q.g2m, prm.aggregation_tolerance, NG, q.gstate, q.gkeep,
                         q.gpasses, s, r.gpass, r.graph_max_passes, G.deg, batch ? cur_gid : nullptr, n, q.gzero,
                         q.gfresh, (prm.flags & LEIDEN_FLAG_REFINE_LABELS) != 0));
    CK(launch_exclusive_scan(q.gkeep, q.vseg2, NG, q.scan_tmp, s));
    q.launches += 14;
    int64_t counts[3];
    CK(cudaMemcpyAsync(&counts[0], q.pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&counts[1], q.pos2 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&counts[2], q.vseg2 + NG, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ST(q.sync_scalars());
    const int64_t ncomm_all = counts[0];
    const int64_t ncomm = counts[2];  // communities of the graphs that go on: vertices of the next graph
    if (trace) {
        int64_t c4[4] = {n, li, lj, ncomm_all};
        std::vector<char> buf(sizeof(c4));
        std::memcpy(buf.data(), c4, sizeof(c4));
        q.trace[{lp, 4}] = buf;
        q.trace_count[{lp, 4}] = 4;
    }
    // ---- renumber communities; lookup dendrogram (graphs that stop take
    // their refined labels, reading R8)
    CK(launch_renumber_batch(q.Cp, q.pos, cur_gid, q.vseg, q.vseg2, q.gstate, q.Cd, n, s));
    CK(launch_lookup_batch(q.C0, batch ? q.gid0 : nullptr, q.vseg0, q.vseg, q.gstate, q.Cd, q.Cp, n0, s));
    CK(launch_commit_states(q.gstate, NG, s));
    q.launches += 3;
    if (ncomm == 0) {  // every graph stopped (globally converged or low shrink)
        stop = true;
        return LEIDEN_OK;
    }
    if (trace) {
        q.record(lp, 5, q.Cd, n);
        q.record(lp, 10, q.C0, n0);
    }
    // ---- aggregation phase (Algorithm 4)
    ST(mark(2));
    const int dst = cur_agg ^ 1;
    CK(cudaMemsetAsync(q.cnt, 0, sizeof(int64_t) * ncomm, s));
    CK(cudaMemsetAsync(q.tdeg, 0, sizeof(int64_t) * ncomm, s));
    CK(launch_comm_counts(q.Cd, G.deg, n, q.cnt, q.tdeg, s));
    CK(launch_exclusive_scan(q.cnt, q.coff, ncomm, q.scan_tmp, s));
    CK(cudaMemsetAsync(q.cursor, 0, sizeof(int32_t) * ncomm, s));
    CK(launch_comm_fill(q.Cd, n, q.coff, q.cursor, q.members, s));
    if (!q.agg[dst].off) {  // sized for the largest graph the handle takes
        ST(q.alloc(&q.agg[dst].off, q.n0 + 1));
        ST(q.alloc(&q.agg[dst].deg, q.n0));
    }
    CK(launch_exclusive_scan(q.tdeg, q.agg[dst].off, ncomm, q.scan_tmp, s));
    CK(launch_comm_bin_keys(q.tdeg, ncomm, q.bins(), q.key, s));
    CK(launch_partition(q.key, ncomm, kNumBins, q.key_off, q.list, q.part_tmp, s));
    CK(launch_max_i64(q.tdeg, ncomm, &q.dsc->maxtdeg, s));
    q.launches += 16;
    int64_t cap = 0;
    int64_t ako[kNumBins + 1];
    CK(cudaMemcpyAsync(&cap, q.agg[dst].off + ncomm, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ako, q.key_off, sizeof(ako), cudaMemcpyDeviceToHost, s));
    ST(q.sync_scalars());
    ST(q.ensure_agg(dst, cap, det));
    // rows of communities without edges (bin 0) are never visited: empty
    CK(cudaMemsetAsync(q.agg[dst].deg, 0, sizeof(int32_t) * ncomm, s));
    {
        const int64_t mt = (int64_t)q.hsc->maxtdeg;
        r.deg_bound = mt < ncomm ? mt : ncomm;  // degrees of G'' (the next graph)
        AggCtx ac;
        ac.g = G;
        ac.det = det;
        ac.Cd = q.Cd;
        ac.coff = q.coff;
        ac.members = q.members;
        ac.out_off = q.agg[dst].off;
        ac.out_deg = q.agg[dst].deg;
        ac.out_idx = q.agg[dst].idx;
        ac.out_w = q.agg[dst].w;
        ac.out_K = q.Kagg;
        ac.ncomm = ncomm;
        ac.err = &q.dsc->err;
        for (int b = 1; b < kBinHub; ++b) {
            const int64_t lo = ako[b], hi = ako[b + 1];
            if (hi == lo) continue;
            ac.prof = prof_begin(16 + b);
            CK(launch_aggregate(ac, b, q.list + lo, hi - lo, b <= 4 ? tile_blocks : big_blocks, s));
            prof_end();
            q.launches++;
        }
        // bin 6: one table per community, packed one after another; the
        // tables go in chunks of at most kAggTableBytes (a table larger than
        // that alone)
        const int64_t K6 = ako[kBinHub + 1] - ako[kBinHub];
        if (K6 > 0) {
            const int32_t *list6 = q.list + ako[kBinHub];
            int64_t *tsize = q.cnt, *toff = q.pos2;
            int32_t *tidx = q.cursor;
            CK(cudaMemsetAsync(tidx, 0xff, sizeof(int32_t) * ncomm, s));
            CK(launch_table_sizes(list6, K6, q.tdeg, q.coff, ncomm, det, tsize, tidx, q.tnm, q.Kagg, s));
            CK(launch_exclusive_scan(tsize, toff, K6, q.scan_tmp, s));
            CK(launch_exclusive_scan(q.tnm, q.tmoff, K6, q.scan_tmp, s));
            q.launches += 4;
            int64_t total = 0, M6 = 0;
            CK(cudaMemcpyAsync(&total, toff + K6, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&M6, q.tmoff + K6, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            // the flat member list of the tables and its entry scan (the
            // per-vertex schedule arrays are free during the aggregation)
            int32_t *fm = q.step, *ft = q.prop, *fd = q.scnt;
            CK(launch_table_members(list6, K6, q.tmoff, M6, q.coff, q.members, G.deg, fm, ft, fd, s));
            CK(launch_exclusive_scan_i32(fd, q.teoff, M6, q.scan_tmp, s));
            q.launches += 4;
            ac.fm = fm;
            ac.ft = ft;
            ac.moff = q.tmoff;
            ac.eoff = q.teoff;
            // slots: a 4-byte key and an 8-byte value (deterministic), or key
            // and fp32 value in one 8-byte word (asynchronous)
            const int64_t budget = kAggTableBytes / (det ? 12 : 8);
            std::vector<int64_t> hoff;
            if (total > budget) {
                hoff.resize((size_t)K6 + 1);
                CK(cudaMemcpyAsync(hoff.data(), toff, sizeof(int64_t) * (K6 + 1), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
            }
            ac.tab_off = toff;
            ac.tab_idx = tidx;
            for (int64_t k0 = 0; k0 < K6;) {
                int64_t k1 = K6;
                if (total > budget) {
                    k1 = k0 + 1;
                    while (k1 < K6 && hoff[k1 + 1] - hoff[k0] <= budget) ++k1;
                }
                const int64_t base = total > budget ? hoff[k0] : 0;
                const int64_t slots = total > budget ? hoff[k1] - base : total;
                if (slots > INT32_MAX) {
                    set_last_error("aggregation table of more than 2^31 slots");
                    return LEIDEN_ERR_OOM;
                }
                ST(q.ensure_hub(0, (int)slots, det));
                if (det) {
                    CK(cudaMemsetAsync(q.hub_keys, 0xff, sizeof(int32_t) * slots, s));
                    CK(cudaMemsetAsync(q.hub_vals, 0, 8 * slots, s));
                } else {
                    CK(launch_fill_u64(static_cast<unsigned long long *>(q.hub_vals), 0x00000000ffffffffULL, slots,
                                       s));
                    q.launches += 1;
                }
                ac.hub_keys = q.hub_keys;
                ac.hub_vals = q.hub_vals;
                ac.tab_k0 = k0;
                ac.tab_k1 = k1;
                ac.tab_base = base;
                ac.prof = prof_begin(16 + kBinHub);
                CK(launch_aggregate_tables(ac, list6, q.sm, s));
                prof_end();
                q.launches += 2;
                k0 = k1;
            }
        }
    }
    // deterministic mode: rows in ascending target order (reading R10)
    if (det && cap > 1) {
        void *stmp = nullptr;
        const size_t sb = sort_rows_tmp_bytes(cap);
        if (cudaMallocAsync(&stmp, sb, s) != cudaSuccess) {
            set_last_error("device allocation of " + std::to_string(sb) + " bytes for the row sort failed");
            return LEIDEN_ERR_OOM;
        }
        const cudaError_t e = launch_sort_rows(ncomm, q.agg[dst].off, q.agg[dst].deg, q.agg[dst].idx,
                                               static_cast<WInt *>(q.agg[dst].w), cap, stmp, s);
        cudaFreeAsync(stmp, s);
        CK(e);
        q.launches += 1;
    }
    // move-based labels of the super-vertices (reading R3), or each alone
    // (refine-based labels)
    if (prm.flags & LEIDEN_FLAG_REFINE_LABELS) {
        CK(launch_iota(q.label, ncomm, s));
        q.launches++;
    } else {
        CK(launch_bound_labels(q.Cd, q.CB, n, ncomm, q.bnd, q.rep, q.label, s));
        q.launches += 4;
    }
    if (batch) {  // graph of every super-vertex; segments of the next graph
        int32_t *nxt = cur_gid == q.gidA ? q.gidB : q.gidA;
        CK(launch_next_gid(q.Cd, cur_gid, n, nxt, s));
        cur_gid = nxt;
        q.launches++;
    }
    std::swap(q.vseg, q.vseg2);
    GraphView G2;
    G2.n = ncomm;
    G2.off = q.agg[dst].off;
    G2.deg = q.agg[dst].deg;
    G2.idx = q.agg[dst].idx;
    G2.w = q.agg[dst].w;
    G2.w_int = det;
    ST(q.sync_scalars());
    if (trace) {
        q.record(lp, 6, G2.off, ncomm + 1);
        q.record(lp, 7, G2.deg, ncomm);
        q.record(lp, 8, G2.idx, cap);
        // weights as fp64
        std::vector<char> raw((size_t)cap * (det ? sizeof(WInt) : sizeof(float)));
        if (cap) {
            CK(cudaMemcpyAsync(raw.data(), G2.w, raw.size(), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        std::vector<char> buf((size_t)cap * sizeof(double));
        double *d = reinterpret_cast<double *>(buf.data());
        for (int64_t e = 0; e < cap; ++e) {
            if (det) d[e] = (double)reinterpret_cast<const WInt *>(raw.data())[e];
            else d[e] = (double)reinterpret_cast<const float *>(raw.data())[e];
        }
        q.trace[{lp, 9}] = std::move(buf);
        q.trace_count[{lp, 9}] = cap;
    }
    G = G2;
    Gcap = cap;
    cur_agg = dst;
    tau /= prm.tolerance_drop;  // threshold scaling
    return LEIDEN_OK;
}

leiden_status Handle::trace_get(int pass, int what, void *dst, int64_t *count) const {
    auto it = p->trace.find({pass, what});
    if (it == p->trace.end() || !count) {
        set_last_error("trace item not recorded");
        return LEIDEN_ERR_INVALID;
    }
    const int64_t have = p->trace_count.at({pass, what});
    if (!dst) {
        *count = have;
        return LEIDEN_OK;
    }
    const int64_t k = *count < have ? *count : have;
    const size_t esz = have ? it->second.size() / (size_t)have : 0;
    std::memcpy(dst, it->second.data(), (size_t)k * esz);
    *count = k;
    return LEIDEN_OK;
}

leiden_status Handle::run(const leiden_params &prm, int32_t *membership, int where, double *modularity,
                          leiden_stats *stats) {
    Impl &q = *p;
    cudaStream_t s = q.s;
    const bool det = prm.mode == LEIDEN_DETERMINISTIC;
    const bool trace = (prm.flags & LEIDEN_FLAG_TRACE) != 0;
    const int32_t B = prm.schedule_buckets;
    const int32_t NG = q.G;
    const bool batch = NG > 1;
    // layer cap of every graph (reading S0): schedule_layers, or by the
    // graph's largest degree when it is 0; L is the largest
    int32_t L = prm.schedule_layers;
    std::vector<int32_t> hgL;
    if (L == 0) {
        if (batch) {
            hgL.resize((size_t)NG);
            for (int32_t g = 0; g < NG; ++g)
                hgL[g] = auto_layers(q.hgmaxdeg[g], q.hvseg0[g + 1] - q.hvseg0[g], q.hgnnz[g]);
            L = *std::max_element(hgL.begin(), hgL.end());
        } else {
            L = auto_layers(q.maxdeg0, q.n0, q.m0);
        }
    }
    if (prm.max_iterations < 1 || prm.max_passes < 0 || !(prm.tolerance_drop > 0) || L < 1 || B < 1 ||
        (prm.mode != LEIDEN_ASYNC && prm.mode != LEIDEN_DETERMINISTIC) || !(prm.resolution >= 0) ||
        !std::isfinite(prm.tolerance) || (q.n0 > 0 && !membership)) {
        set_last_error("invalid leiden_params or membership pointer");
        return LEIDEN_ERR_INVALID;
    }
    const int32_t nsteps = L - 1 + B;
    const int32_t nkeys = nsteps * kNumBins;
    if (nkeys + 1 > q.key_cap || L > 4096) {
        set_last_error("schedule_layers + schedule_buckets too large");
        return LEIDEN_ERR_INVALID;
    }
    ST(check_barrier_budget(prm.max_iterations, nsteps, det, q.sm));
    if (det && (prm.flags & LEIDEN_FLAG_RANDOM_REFINE)) {
        set_last_error("the randomized refinement has no deterministic mode");
        return LEIDEN_ERR_UNSUPPORTED;
    }
    if (batch && (trace || (prm.flags & LEIDEN_FLAG_STEP_LAUNCHES))) {
        set_last_error("a batch of graphs runs without trace and without per-step launches");
        return LEIDEN_ERR_UNSUPPORTED;
    }
    ST(q.ensure_phase(prm.max_iterations, NG));
    if (det) {
        if (prm.resolution != 1.0 || q.nonint) {
            set_last_error("deterministic mode needs integer weights and resolution 1");
            return LEIDEN_ERR_UNSUPPORTED;
        }
        double wmax = q.wsum;
        if (batch) {
            wmax = 0;
            for (double x : q.hgw) wmax = x > wmax ? x : wmax;
        }
        if (wmax >= kDetMaxTwoM) {
            set_last_error("deterministic mode needs 2m < 2^53 (in every graph of a batch)");
            return LEIDEN_ERR_OVERFLOW;
        }
    }
    // a failure of an earlier run (a barrier timeout, a full hash table)
    // must not outlive it: the error word starts clean
    CK(cudaMemsetAsync(&q.dsc->err, 0, sizeof(int), s));
    q.trace.clear();
    q.trace_count.clear();
    q.launches = 0;
    const bool profile = (prm.flags & LEIDEN_FLAG_PROFILE) != 0;
    q.prof_valid = false;
    q.prof_det = det;
    q.ev_used = 0;
    q.prof_spans.clear();
    q.prof_launches.assign(LEIDEN_PROFILE_CLASSES, 0);
    if (profile)
        CK(cudaMemsetAsync(q.prof_cnt, 0, sizeof(unsigned long long) * LEIDEN_PROFILE_CLASSES * kProfCounters, s));
    Run r;
    r.prm = &prm;
    r.det = det;
    r.trace = trace;
    r.profile = profile;
    r.batch = batch;
    r.L = L;
    r.B = B;
    r.NG = NG;
    if (batch) {  // per-graph caps (all L when schedule_layers is given)
        if (hgL.empty()) hgL.assign((size_t)NG, L);
        CK(cudaMemcpyAsync(q.gL, hgL.data(), sizeof(int32_t) * NG, cudaMemcpyHostToDevice, s));
        r.gL = q.gL;
    }
    cudaEvent_t &ev0 = r.ev0, &ev1 = r.ev1;  // destroyed with the run
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    CK(cudaEventRecord(ev0, s));
    std::vector<std::pair<cudaEvent_t, int>> &marks = r.marks;
    auto mark = [&](int phase) { return q.mark(r, phase); };
    leiden_stats &st = r.st;
    const int64_t n0 = q.n0;

    CK(launch_iota(q.C0, n0, s));
    q.launches++;
    // per-graph state: graphs with vertices start active
    {
        std::vector<int32_t> st0(NG);
        for (int32_t g = 0; g < NG; ++g)
            st0[g] = q.hvseg0[g + 1] > q.hvseg0[g] ? kGraphActive : kGraphFinished;
        CK(cudaMemcpyAsync(q.gstate, st0.data(), sizeof(int32_t) * NG, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(q.vseg, q.vseg0, sizeof(int64_t) * (NG + 1), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(q.gpasses, 0, sizeof(int32_t) * NG, s));
        CK(launch_fill_i32(q.gfresh, 1, NG, s));  // pass 0 begins from singletons
        CK(cudaStreamSynchronize(s));  // st0 is a local
    }
    r.n0 = n0;
    r.deg_bound = q.maxdeg0;
    r.cur_gid = batch ? q.gid0 : nullptr;  // graph of every vertex of G'
    r.G.n = n0;
    r.G.off = q.off0;
    r.G.deg = q.deg0;
    r.G.idx = q.idx0;
    r.G.w = q.w0;
    r.G.w_int = false;
    r.tau = prm.tolerance;
    r.cur_agg = 1;  // next pass writes agg[cur_agg ^ 1]
    r.Gcap = q.m0;  // entry capacity of G' (holey after aggregation)
    const bool &no_edges = r.no_edges;
    const int &passes = r.passes;

    for (int32_t lp = 0; lp < prm.max_passes; ++lp) {
        bool stop = false;
        ST(q.pass(r, lp, stop));
        if (stop) break;
    }
    ST(mark(3));
    // C <- lookup dendrogram using C to C' (reading R8): a graph without
    // edges ends on its singletons; graphs of a batch still running after
    // the last pass take ids of the last aggregated graph, moved into their
    // own range of the input
    if (no_edges) {
        CK(launch_lookup(q.C0, q.Cp, n0, s));
        q.launches++;
    }
    if (batch) {
        CK(launch_finalize_batch(q.C0, q.gid0, q.vseg0, q.vseg, q.gstate, n0, s));
        q.launches++;
    }
    // canonical labels: rank of each community's smallest vertex id (inside
    // its own graph)
    int32_t *outp = (where == LEIDEN_DEVICE) ? membership : q.out;
    CK(launch_min_vertex(q.C0, n0, q.minv, s));
    CK(launch_first_flags(q.C0, q.minv, n0, q.flag, s));
    CK(launch_exclusive_scan_i32(q.flag, q.pos, n0, q.scan_tmp, s));
    if (batch) CK(launch_canonical_batch(q.C0, q.minv, q.pos, q.gid0, q.vseg0, n0, outp, s));
    else CK(launch_canonical(q.C0, q.minv, q.pos, n0, outp, s));
    q.launches += 7;
    // modularity (Eq. 1) of the result on the input graph (each graph's own)
    CK(cudaMemsetAsync(q.sigtot, 0, sizeof(double) * n0, s));
    CK(cudaMemsetAsync(q.dsc->msum, 0, sizeof(double) * 4, s));
    if (batch) {
        CK(cudaMemsetAsync(q.gmsum, 0, sizeof(double) * 3 * NG, s));
        CK(launch_modularity_batch(n0, q.off0, q.idx0, q.w0, outp, q.gid0, q.vseg0, NG, prm.resolution, q.sigtot,
                                   q.gmsum, &q.dsc->msum[3], q.gq, s, q.maxdeg0 > kLongRow));
        CK(launch_graph_counts(q.pos, q.vseg0, NG, q.gcomm, s));
        q.launches += 4;
    } else {
        CK(launch_modularity_parts(n0, q.off0, q.idx0, q.w0, outp, q.sigtot, q.dsc->msum, s, q.maxdeg0 > kLongRow));
        CK(launch_sum_squares(q.sigtot, n0, &q.dsc->msum[2], s));
        q.launches += q.maxdeg0 > kLongRow ? 3 : 2;
    }
    int64_t ncomm_out = 0;
    CK(cudaMemcpyAsync(&ncomm_out, q.pos + n0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (where != LEIDEN_DEVICE && n0 > 0)
        CK(cudaMemcpyAsync(membership, q.out, sizeof(int32_t) * n0, cudaMemcpyDeviceToHost, s));
    std::vector<double> qg(batch ? NG : 0);
    q.hpasses.assign(NG, 0);
    q.hcomm.assign(NG, 0);
    if (batch) {
        CK(cudaMemcpyAsync(qg.data(), q.gq, sizeof(double) * NG, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(q.hpasses.data(), q.gpasses, sizeof(int32_t) * NG, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(q.hcomm.data(), q.gcomm, sizeof(int64_t) * NG, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(ev1, s));
    ST(q.sync_scalars());
    double Q;
    if (batch) {  // per-graph scores; the statistics carry their mean
        Q = 0;
        for (double x : qg) Q += x;
        Q /= NG;
        if (modularity) std::memcpy(modularity, qg.data(), sizeof(double) * NG);
    } else {
        const double two_m = q.hsc->msum[1];
        Q = two_m > 0 ? q.hsc->msum[0] / two_m - prm.resolution * q.hsc->msum[2] / (two_m * two_m) : 0.0;
        if (modularity) *modularity = Q;
        q.hpasses[0] = passes;
        q.hcomm[0] = ncomm_out;
    }
    if (stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        st.passes = passes;
        st.communities = ncomm_out;
        st.modularity = Q;
        st.ms_total = ms;
        double ph[4] = {0, 0, 0, 0};
        for (size_t i = 0; i < marks.size(); ++i) {
            cudaEvent_t end = (i + 1 < marks.size()) ? marks[i + 1].first : ev1;
            float t = 0;
            cudaEventElapsedTime(&t, marks[i].first, end);
            ph[marks[i].second] += t;
        }
        st.ms_move = ph[0];
        st.ms_refine = ph[1];
        st.ms_aggregate = ph[2];
        st.ms_other = ph[3];
        st.kernel_launches = q.launches;
        *stats = st;
    }
    if (profile) ST(q.finish_profile());
    return LEIDEN_OK;
}

int32_t Handle::num_graphs() const { return p->G; }

leiden_status Handle::graph_info(int32_t *passes, int64_t *communities) const {
    if (p->hpasses.size() != (size_t)p->G) {
        set_last_error("no run has finished on this handle");
        return LEIDEN_ERR_INVALID;
    }
    if (passes) std::memcpy(passes, p->hpasses.data(), sizeof(int32_t) * p->G);
    if (communities) std::memcpy(communities, p->hcomm.data(), sizeof(int64_t) * p->G);
    return LEIDEN_OK;
}

leiden_status Handle::set_tuning(const leiden_tuning &t) {
    if (!tuning_valid(t)) {
        set_last_error("leiden_tuning value outside its range");
        return LEIDEN_ERR_INVALID;
    }
    p->tune = t;
    return LEIDEN_OK;
}

leiden_status Handle::get_tuning(leiden_tuning *t) const {
    if (!t) {
        set_last_error("tuning is NULL");
        return LEIDEN_ERR_INVALID;
    }
    *t = p->tune;
    return LEIDEN_OK;
}

leiden_status Handle::profile_get(leiden_kernel_profile *out) const {
    if (!p->prof_valid || !out) {
        set_last_error("the last run was not profiled");
        return LEIDEN_ERR_INVALID;
    }
    std::memcpy(out, p->prof_out, sizeof(p->prof_out));
    return LEIDEN_OK;
}

// Communities of a membership that are not connected (Algorithm 5), on a
// CSR given as device pointers, with scratch from the stream-ordered
// allocator. Labels must lie in [0, n) (checked first).
leiden_status disconnected_device(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *memb,
                                  cudaStream_t s, int64_t *count) {
    if (n < 0 || !count || (n > 0 && (!off || !idx || !memb))) {
        set_last_error("invalid arguments to leiden_disconnected");
        return LEIDEN_ERR_INVALID;
    }
    *count = 0;
    if (n == 0) return LEIDEN_OK;
    int32_t *buf = nullptr;
    unsigned long long *flags = nullptr;
    if (cudaMallocAsync(&buf, sizeof(int32_t) * 2 * n, s) != cudaSuccess ||
        cudaMallocAsync(&flags, sizeof(unsigned long long) * 2, s) != cudaSuccess) {
        if (buf) cudaFreeAsync(buf, s);
        set_last_error("scratch allocation failed");
        return LEIDEN_ERR_OOM;
    }
    int32_t *parent = buf, *roots = buf + n;
    int *changed = reinterpret_cast<int *>(flags);
    unsigned long long *cnt = flags + 1;
    unsigned long long h[2] = {0, 0};
    leiden_status st = LEIDEN_OK;
    // labels out of range are an error
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long) * 2, s);
    if (e == cudaSuccess) e = launch_cc_labels(n, memb, changed, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (h[0] & 0xffffffffULL)) {
        set_last_error("leiden_disconnected: membership labels must lie in [0, n)");
        st = LEIDEN_ERR_INVALID;
    }
    if (e == cudaSuccess && st == LEIDEN_OK) {
        e = launch_cc_init(n, parent, roots, s);
        // a pass that finds an edge between two trees lowers some parent,
        // and on the graphs here components settle within a few passes; 64
        // is a safety bound, reported as a timeout
        int pass = 0;
        for (; e == cudaSuccess && pass < 64; ++pass) {
            e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long) * 2, s);
            if (e == cudaSuccess) e = launch_cc_pass(n, off, idx, memb, parent, changed, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess || !(h[0] & 0xffffffffULL)) break;
        }
        if (e == cudaSuccess && pass == 64) {
            set_last_error("leiden_disconnected: components did not settle");
            st = LEIDEN_ERR_TIMEOUT;
        }
        if (e == cudaSuccess && st == LEIDEN_OK) e = launch_cc_count(n, memb, parent, roots, cnt, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && st == LEIDEN_OK) *count = (int64_t)h[1];
    }
    cudaFreeAsync(buf, s);
    cudaFreeAsync(flags, s);
    if (e != cudaSuccess) {
        set_last_error(std::string("leiden_disconnected: ") + cudaGetErrorString(e));
        return LEIDEN_ERR_CUDA;
    }
    return st;
}

// Modularity (Eq. 1) of a membership on a CSR given as device pointers, with
// scratch from the stream-ordered allocator.
leiden_status modularity_device(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                const int32_t *memb, double gamma, cudaStream_t s, double *q_out) {
    if (n < 0 || !q_out || (n > 0 && (!off || !idx || !memb))) {
        set_last_error("invalid arguments to leiden_modularity");
        return LEIDEN_ERR_INVALID;
    }
    if (n == 0) {
        *q_out = 0.0;
        return LEIDEN_OK;
    }
    double *sig = nullptr, *sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sig, sizeof(double) * n, s);
    if (e != cudaSuccess) {
        set_last_error("scratch allocation failed");
        return LEIDEN_ERR_OOM;
    }
    e = cudaMallocAsync(&sums, sizeof(double) * 4, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(sig, s);
        set_last_error("scratch allocation failed");
        return LEIDEN_ERR_OOM;
    }
    double h[4] = {0, 0, 0, 0};
    cudaMemsetAsync(sig, 0, sizeof(double) * n, s);
    cudaMemsetAsync(sums, 0, sizeof(double) * 4, s);
    launch_modularity_parts(n, off, idx, w, memb, sig, sums, s);
    launch_sum_squares(sig, n, &sums[2], s);
    cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(sig, s);
    cudaFreeAsync(sums, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string("leiden_modularity: ") + cudaGetErrorString(e));
        return LEIDEN_ERR_CUDA;
    }
    if (h[3] != 0.0) {
        set_last_error("leiden_modularity: membership labels must lie in [0, n)");
        return LEIDEN_ERR_INVALID;
    }
    *q_out = h[1] > 0 ? h[0] / h[1] - gamma * h[2] / (h[1] * h[1]) : 0.0;
    return LEIDEN_OK;
}

}  // namespace lgb
