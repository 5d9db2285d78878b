// Serving with continuous batching.
//
// A serving handle keeps a union of graphs in flight, each at its own pass
// of Algorithm 1. A step first admits waiting graphs at the pass boundary
// (first come, first served) while a slot, the union's capacity and the
// device budget allow: each admitted graph's CSR is appended to the union's
// holey CSR and its vertices start as singletons. Then one pass runs over
// the whole union with the batch machinery (Handle::Impl::pass), every graph
// with its own 2m, schedule state (seed + its pass), tolerance (tau / drop^
// its pass), convergence and stop tests; a graph that stops -- or reaches
// MAX_PASSES -- leaves with its refined labels, the others continue as super-
// vertices of the aggregated union. Finished graphs get canonical labels and
// Eq. 1 on their own input. The dendrogram of every graph in flight lives in
// one arena, compacted after each step in union order.
#include <algorithm>
#include <chrono>

#include "engine_impl.h"

namespace lgb {

leiden_status Handle::server_init(const leiden_params &prm, int64_t max_vertices, int64_t max_entries,
                                  int32_t max_graphs, int64_t device_budget, void *stream, ServeShared *shared) {
    Impl &q = *p;
    if (max_vertices < 1 || max_vertices > 0x7fffffffLL || max_entries < 1 || max_graphs < 1 ||
        prm.max_iterations < 1 || prm.max_passes < 1 || !(prm.tolerance_drop > 0) || prm.schedule_layers < 0 ||
        prm.schedule_layers > 4096 || prm.schedule_buckets < 1 || !(prm.resolution >= 0) ||
        !std::isfinite(prm.tolerance) || (prm.mode != LEIDEN_ASYNC && prm.mode != LEIDEN_DETERMINISTIC)) {
        set_last_error("invalid server capacity or leiden_params");
        return LEIDEN_ERR_INVALID;
    }
    if (prm.mode == LEIDEN_DETERMINISTIC && (prm.flags & LEIDEN_FLAG_RANDOM_REFINE)) {
        set_last_error("the randomized refinement has no deterministic mode");
        return LEIDEN_ERR_UNSUPPORTED;
    }
    if (prm.mode == LEIDEN_DETERMINISTIC && prm.resolution != 1.0) {
        set_last_error("deterministic mode needs resolution 1");
        return LEIDEN_ERR_UNSUPPORTED;
    }
    // the largest layer cap a graph can take (reading S0)
    const int32_t nkeys = ((prm.schedule_layers > 0 ? prm.schedule_layers : kLayersHeavy) - 1 +
                           prm.schedule_buckets) * kNumBins;
    if (nkeys + 1 > 8192) {
        set_last_error("schedule_layers + schedule_buckets too large");
        return LEIDEN_ERR_INVALID;
    }
    q.s = static_cast<cudaStream_t>(stream);
    q.n0 = max_vertices;
    q.m0 = max_entries;
    q.G = max_graphs;
    q.hvseg0 = {0, 0};
    ST(q.init_device());
    ST(check_barrier_budget(prm.max_iterations, nkeys / kNumBins, prm.mode == LEIDEN_DETERMINISTIC, q.sm));
    ST(q.alloc_workspace(max_vertices, max_graphs));
    q.srv = new Serve;
    Serve &v = *q.srv;
    if (shared) v.sh = shared;
    v.prm = prm;
    v.prm.flags &= ~(uint32_t)(LEIDEN_FLAG_TRACE | LEIDEN_FLAG_PROFILE |
                               LEIDEN_FLAG_STEP_LAUNCHES);
    v.cap_v = max_vertices;
    v.cap_e = max_entries;
    v.cap_g = max_graphs;
    ST(q.ensure_agg(0, max_entries, prm.mode == LEIDEN_DETERMINISTIC));
    ST(q.ensure_agg(1, max_entries, prm.mode == LEIDEN_DETERMINISTIC));
    ST(q.ensure_part_tmp(partition_tmp_bytes(max_vertices, nkeys + 1)));
    ST(q.ensure_phase(prm.max_iterations, max_graphs));
    v.arena[0] = q.C0;
    ST(q.alloc(&v.arena[1], max_vertices));
    for (int32_t **a : {&q.gid0, &q.gidA, &q.gidB}) ST(q.alloc(a, max_vertices));
    ST(q.alloc(&v.gpass, max_graphs));
    ST(q.alloc(&v.gtau, max_graphs));
    ST(q.alloc(&v.gL, max_graphs));
    CK(cudaStreamSynchronize(q.s));
    if (v.sh->budget <= 0) {  // the first lane of a server sets the budget
        if (device_budget <= 0) {
            size_t fr = 0, tot = 0;
            CK(cudaMemGetInfo(&fr, &tot));
            device_budget = (int64_t)(fr / 2);
        }
        v.sh->budget = device_budget;
    }
    return LEIDEN_OK;
}

namespace {

// device bytes of a graph's own buffers: CSR copy and result
int64_t graph_bytes(int64_t n, int64_t m) {
    return (int64_t)sizeof(int64_t) * (n + 1) + (int64_t)(sizeof(int32_t) + sizeof(float)) * m +
           (int64_t)sizeof(int32_t) * n;
}
int64_t request_bytes(const Request &r) { return graph_bytes(r.n, r.m); }

}  // namespace

// Copy a request to device memory and check it as validation would: offsets
// monotone within [0, m], indices in range, weights finite and >= 0,
// w_ij == w_ji; weight sum and integrality for the deterministic mode.
static leiden_status upload(Handle::Impl &q, Request &r, const int64_t *off, const int32_t *idx, const float *w,
                            cudaMemcpyKind kind) {
    cudaStream_t s = q.s;
    const int64_t n = r.n, m = r.m;
    auto get = [&](void **dst, size_t bytes) -> leiden_status {
        if (cudaMallocAsync(dst, bytes ? bytes : 1, s) != cudaSuccess) {
            set_last_error("device allocation for a served graph failed");
            return LEIDEN_ERR_OOM;
        }
        return LEIDEN_OK;
    };
    r.bytes = request_bytes(r);  // charged first: free_request() gives back exactly this
    q.srv->sh->used += r.bytes;
    ST(get((void **)&r.off, sizeof(int64_t) * (n + 1)));
    ST(get((void **)&r.idx, sizeof(int32_t) * m));
    ST(get((void **)&r.w, sizeof(float) * m));
    ST(get((void **)&r.memb, sizeof(int32_t) * n));
    r.on_device = true;
    CK(cudaMemcpyAsync(r.off, off, sizeof(int64_t) * (n + 1), kind, s));
    if (m > 0) {
        CK(cudaMemcpyAsync(r.idx, idx, sizeof(int32_t) * m, kind, s));
        if (w) CK(cudaMemcpyAsync(r.w, w, sizeof(float) * m, kind, s));
        else CK(launch_fill_i32(reinterpret_cast<int32_t *>(r.w), 0x3f800000, m, s));  // unit weights: 1.0f
    }
    CK(cudaMemsetAsync(q.dsc, 0, sizeof(Scalars), s));
    CK(launch_degrees(r.off, q.scnt, n, &q.dsc->err, s));
    CK(launch_max_i32(q.scnt, n, &q.dsc->maxdeg, s));
    CK(launch_validate(n, r.off, r.idx, r.w, &q.dsc->err, s));
    CK(launch_weight_props(r.w, m, &q.dsc->nonint, &q.dsc->wsum, s));
    CK(cudaMemcpyAsync(q.hsc, q.dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (q.hsc->err) {
        const int e = q.hsc->err;
        set_last_error(e == 2 ? "CSR is not symmetric (w_ij != w_ji)" : "malformed CSR (offsets, indices or weights)");
        return e == 2 ? LEIDEN_ERR_NOT_SYMMETRIC : LEIDEN_ERR_INVALID;
    }
    const int32_t pl = q.srv->prm.schedule_layers;
    r.L = pl > 0 ? pl : auto_layers(q.hsc->maxdeg, n, m);
    if (q.srv->prm.mode == LEIDEN_DETERMINISTIC) {
        if (q.hsc->nonint) {
            set_last_error("deterministic mode needs integer weights");
            return LEIDEN_ERR_UNSUPPORTED;
        }
        if (q.hsc->wsum >= kDetMaxTwoM) {
            set_last_error("deterministic mode needs 2m < 2^53");
            return LEIDEN_ERR_OVERFLOW;
        }
    }
    return LEIDEN_OK;
}

// free the input copies of a request; its result buffer stays until read
static void release_input(Handle::Impl &q, Request &r) {
    for (void **b : {(void **)&r.off, (void **)&r.idx, (void **)&r.w}) {
        if (*b) cudaFreeAsync(*b, q.s);
        *b = nullptr;
    }
    const int64_t keep = r.memb ? (int64_t)sizeof(int32_t) * r.n : 0;
    q.srv->sh->used -= r.bytes - keep;
    r.bytes = keep;
    std::vector<int64_t>().swap(r.hoff);
    std::vector<int32_t>().swap(r.hidx);
    std::vector<float>().swap(r.hw);
}
// free everything a request holds on the device
static void free_request(Handle::Impl &q, Request &r) {
    release_input(q, r);
    if (r.memb) cudaFreeAsync(r.memb, q.s);
    r.memb = nullptr;
    q.srv->sh->used -= r.bytes;
    r.bytes = 0;
}

leiden_status Handle::server_submit(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const float *w,
                                    int where, int64_t *id) {
    Impl &q = *p;
    if (!q.srv) {
        set_last_error("not a serving handle");
        return LEIDEN_ERR_INVALID;
    }
    Serve &v = *q.srv;
    if (!id || n < 0 || nnz < 0 || !off || (nnz > 0 && !idx) || (where != LEIDEN_HOST && where != LEIDEN_DEVICE)) {
        set_last_error("invalid CSR arguments");
        return LEIDEN_ERR_INVALID;
    }
    if (n > v.cap_v || nnz > v.cap_e) {
        set_last_error("graph larger than the server's capacity");
        return LEIDEN_ERR_INVALID;
    }
    if (graph_bytes(n, nnz) > v.sh->budget) {  // could never be admitted, and would hold up every later graph
        set_last_error("graph needs " + std::to_string(graph_bytes(n, nnz)) + " device bytes, more than the " +
                       "server's device budget of " + std::to_string(v.sh->budget));
        return LEIDEN_ERR_OOM;
    }
    if (where == LEIDEN_HOST && (off[0] != 0 || off[n] != nnz)) {
        set_last_error("offsets[0] must be 0 and offsets[n] must equal nnz");
        return LEIDEN_ERR_INVALID;
    }
    Request r;
    const int64_t rid = v.sh->next_id++;
    r.id = rid;
    r.n = n;
    r.m = nnz;
    if (n == 0) {  // nothing to cluster: finished at once
        r.fin_seq = v.sh->fin_seq++;
        v.reqs[rid] = std::move(r);
        v.finished.push_back(rid);
        *id = rid;
        return LEIDEN_OK;
    }
    const cudaMemcpyKind kind = where == LEIDEN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // copied to the device at once unless the budget is spent or an earlier
    // graph still waits on the host (uploads keep the order of arrival)
    if (v.sh->used + request_bytes(r) <= v.sh->budget && v.on_host == 0) {
        leiden_status st = upload(q, r, off, idx, w, kind);
        if (st != LEIDEN_OK) {
            free_request(q, r);
            return st;
        }
    } else {  // keep a host copy until the budget allows
        r.hoff.resize((size_t)n + 1);
        r.hidx.resize((size_t)nnz);
        r.hw.assign((size_t)nnz, 1.0f);
        const cudaMemcpyKind back = where == LEIDEN_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        CK(cudaMemcpyAsync(r.hoff.data(), off, sizeof(int64_t) * (n + 1), back, q.s));
        if (nnz > 0) {
            CK(cudaMemcpyAsync(r.hidx.data(), idx, sizeof(int32_t) * nnz, back, q.s));
            if (w) CK(cudaMemcpyAsync(r.hw.data(), w, sizeof(float) * nnz, back, q.s));
        }
        CK(cudaStreamSynchronize(q.s));
        v.on_host++;
    }
    *id = rid;
    v.waiting.push_back(rid);
    v.reqs[rid] = std::move(r);
    return LEIDEN_OK;
}

leiden_status Handle::server_step(int32_t *finished_out) {
    Impl &q = *p;
    if (!q.srv) {
        set_last_error("not a serving handle");
        return LEIDEN_ERR_INVALID;
    }
    Serve &v = *q.srv;
    cudaStream_t s = q.s;
    const leiden_params &prm = v.prm;
    const bool det = prm.mode == LEIDEN_DETERMINISTIC;
    int32_t nfin = 0;
    if (finished_out) *finished_out = 0;
    // ---- admission at the pass boundary (first come, first served)
    int64_t sum_m = 0;
    for (int64_t id : v.inflight) sum_m += v.reqs[id].m;
    while (!v.waiting.empty()) {
        Request &r = v.reqs[v.waiting.front()];
        if (!r.on_device) {
            if (v.sh->used + request_bytes(r) > v.sh->budget) break;
            v.on_host--;
            leiden_status st = upload(q, r, r.hoff.data(), r.hidx.data(), r.hw.data(), cudaMemcpyHostToDevice);
            if (st != LEIDEN_OK) {  // the graph fails; its error is its result
                r.status = st;
                release_input(q, r);
                r.fin_seq = v.sh->fin_seq++;
                v.finished.push_back(r.id);
                v.waiting.pop_front();
                nfin++;
                continue;
            }
        }
        if ((int32_t)v.inflight.size() >= v.cap_g || v.arena_n + r.n > v.cap_v || v.n_union + r.n > v.cap_v ||
            v.e_union + r.m > v.cap_e || sum_m + r.m > v.cap_e)
            break;
        const Impl::Agg &u = q.agg[v.cur];
        CK(launch_append_graph(r.n, r.off, r.idx, r.w, v.n_union, v.e_union, det, (int32_t)v.inflight.size(), u.off,
                               u.deg, u.idx, u.w, q.gidA, v.arena[v.arena_cur], v.arena_n, s));
        r.pass = 0;
        r.fresh = 1;
        r.n_cur = r.n;
        r.arena = v.arena_n;
        v.n_union += r.n;
        v.e_union += r.m;
        v.arena_n += r.n;
        sum_m += r.m;
        v.inflight.push_back(r.id);
        v.waiting.pop_front();
    }
    if (v.inflight.empty()) {
        if (finished_out) *finished_out = nfin;
        return LEIDEN_OK;
    }
    // ---- per-graph arrays of this step, in union order; the error word
    // starts clean (an earlier step's failure must not outlive it)
    CK(cudaMemsetAsync(&q.dsc->err, 0, sizeof(int), s));
    const int32_t K = (int32_t)v.inflight.size();
    v.hvseg.assign(K + 1, 0);
    v.hvseg0.assign(K + 1, 0);
    v.hpass.assign(K, 0);
    v.hfresh.assign(K, 1);
    v.hstate.assign(K, kGraphActive);
    v.htau.assign(K, 0.0);
    v.hL.assign(K, 0);
    int32_t Lmax = 1;
    for (int32_t k = 0; k < K; ++k) {
        const Request &r = v.reqs[v.inflight[k]];
        v.hL[k] = r.L;
        Lmax = std::max(Lmax, r.L);
        v.hvseg[k + 1] = v.hvseg[k] + r.n_cur;
        v.hvseg0[k + 1] = v.hvseg0[k] + r.n;
        v.hpass[k] = r.pass;
        v.hfresh[k] = r.fresh;
        v.htau[k] = prm.tolerance / std::pow(prm.tolerance_drop, (double)r.pass);  // threshold scaling
    }
    CK(cudaMemcpyAsync(q.vseg, v.hvseg.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(q.vseg0, v.hvseg0.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(v.gpass, v.hpass.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(q.gstate, v.hstate.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(q.gfresh, v.hfresh.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(v.gtau, v.htau.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(v.gL, v.hL.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CK(launch_graph_ids(q.vseg, K, v.n_union, q.gidA, s));
    CK(launch_graph_ids(q.vseg0, K, v.arena_n, q.gid0, s));
    q.C0 = v.arena[v.arena_cur];
    // ---- one pass of every graph in flight
    Run r;
    r.prm = &prm;
    r.det = det;
    r.batch = true;
    r.L = Lmax;
    r.gL = v.gL;
    r.B = prm.schedule_buckets;
    r.NG = K;
    const Impl::Agg &u = q.agg[v.cur];
    r.G.n = v.n_union;
    r.G.off = u.off;
    r.G.deg = u.deg;
    r.G.idx = u.idx;
    r.G.w = u.w;
    r.G.w_int = det;
    r.Gcap = v.e_union;
    r.cur_agg = v.cur;
    r.cur_gid = q.gidA;
    r.tau = prm.tolerance;
    r.n0 = v.arena_n;
    r.n_cont = v.n_cont;
    r.gpass = v.gpass;
    r.gtau = v.gtau;
    r.graph_max_passes = prm.max_passes;
    bool stop = false;
    ST(q.pass(r, 0, stop));
    v.steps++;
    // ---- graphs that stopped leave with their results
    CK(cudaMemcpyAsync(v.hstate.data(), q.gstate, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(v.hfresh.data(), q.gfresh, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s));
    if (!stop) CK(cudaMemcpyAsync(v.hvseg.data(), q.vseg, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int64_t> next;
    int64_t arena_next = 0;
    int32_t *dst_arena = v.arena[v.arena_cur ^ 1];
    for (int32_t k = 0; k < K; ++k) {
        Request &rq = v.reqs[v.inflight[k]];
        if (!stop && v.hstate[k] == kGraphActive) {  // goes on: pack its dendrogram
            rq.n_cur = v.hvseg[k + 1] - v.hvseg[k];
            rq.pass++;
            rq.fresh = v.hfresh[k];
            CK(cudaMemcpyAsync(dst_arena + arena_next, q.C0 + rq.arena, sizeof(int32_t) * rq.n,
                               cudaMemcpyDeviceToDevice, s));
            rq.arena = arena_next;
            arena_next += rq.n;
            next.push_back(rq.id);
            continue;
        }
        // finished: its refined labels, as ids in its own range, to canonical labels; Eq. 1 on its input
        const int64_t n = rq.n;
        CK(launch_shift_labels(q.C0 + rq.arena, n, rq.arena, q.Cd, s));
        CK(launch_min_vertex(q.Cd, n, q.minv, s));
        CK(launch_first_flags(q.Cd, q.minv, n, q.flag, s));
        CK(launch_exclusive_scan_i32(q.flag, q.pos, n, q.scan_tmp, s));
        CK(launch_canonical(q.Cd, q.minv, q.pos, n, rq.memb, s));
        CK(cudaMemsetAsync(q.sigtot, 0, sizeof(double) * n, s));
        CK(cudaMemsetAsync(q.dsc->msum, 0, sizeof(double) * 4, s));
        CK(launch_modularity_parts(n, rq.off, rq.idx, rq.w, rq.memb, q.sigtot, q.dsc->msum, s));
        CK(launch_sum_squares(q.sigtot, n, &q.dsc->msum[2], s));
        int64_t ncomm = 0;
        CK(cudaMemcpyAsync(&ncomm, q.pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        ST(q.sync_scalars());
        const double tm = q.hsc->msum[1];
        rq.q = tm > 0 ? q.hsc->msum[0] / tm - prm.resolution * q.hsc->msum[2] / (tm * tm) : 0.0;
        rq.communities = ncomm;
        rq.passes = rq.pass + 1;
        rq.status = LEIDEN_OK;
        release_input(q, rq);
        rq.fin_seq = v.sh->fin_seq++;
        v.finished.push_back(rq.id);
        nfin++;
    }
    v.inflight.swap(next);
    v.arena_cur ^= 1;
    v.arena_n = arena_next;
    q.C0 = v.arena[v.arena_cur];
    if (stop || v.inflight.empty()) {
        v.n_union = v.e_union = v.n_cont = 0;
        v.cur = r.cur_agg;
    } else {  // the aggregated union carries the graphs that go on
        v.n_union = r.G.n;
        v.e_union = r.Gcap;
        v.n_cont = r.G.n;
        v.cur = r.cur_agg;
    }
    CK(cudaStreamSynchronize(s));
    if (finished_out) *finished_out = nfin;
    return LEIDEN_OK;
}

leiden_status Handle::server_next(int64_t *id) {
    Impl &q = *p;
    if (!q.srv || !id) {
        set_last_error("not a serving handle");
        return LEIDEN_ERR_INVALID;
    }
    *id = q.srv->finished.empty() ? -1 : q.srv->finished.front();
    return LEIDEN_OK;
}

leiden_status Handle::server_result(int64_t id, int32_t *membership, int where, double *qout, int32_t *passes,
                                    int64_t *communities) {
    Impl &q = *p;
    if (!q.srv) {
        set_last_error("not a serving handle");
        return LEIDEN_ERR_INVALID;
    }
    Serve &v = *q.srv;
    auto it = v.reqs.find(id);
    bool done = false;
    for (int64_t f : v.finished) done |= f == id;
    if (it == v.reqs.end() || !done) {
        set_last_error("unknown or unfinished request id");
        return LEIDEN_ERR_INVALID;
    }
    Request &r = it->second;
    leiden_status st = r.status;
    if (st == LEIDEN_OK && r.n > 0) {
        if (!membership) {
            set_last_error("membership is NULL");
            return LEIDEN_ERR_INVALID;
        }
        CK(cudaMemcpyAsync(membership, r.memb, sizeof(int32_t) * r.n,
                           where == LEIDEN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, q.s));
        CK(cudaStreamSynchronize(q.s));
    }
    if (qout) *qout = r.q;
    if (passes) *passes = r.passes;
    if (communities) *communities = r.communities;
    free_request(q, r);
    for (auto f = v.finished.begin(); f != v.finished.end(); ++f)
        if (*f == id) {
            v.finished.erase(f);
            break;
        }
    v.reqs.erase(it);
    if (st != LEIDEN_OK) set_last_error("the graph failed when it was copied to the device");
    return st;
}

leiden_status Handle::server_info(leiden_server_state *out) const {
    const Impl &q = *p;
    if (!q.srv || !out) {
        set_last_error("not a serving handle");
        return LEIDEN_ERR_INVALID;
    }
    const Serve &v = *q.srv;
    out->waiting = (int32_t)v.waiting.size();
    out->in_flight = (int32_t)v.inflight.size();
    out->finished = (int32_t)v.finished.size();
    out->reserved = 0;
    out->union_vertices = v.n_union;
    out->union_entries = v.e_union;
    out->device_bytes = v.sh->used;
    out->steps = v.steps;
    return LEIDEN_OK;
}

bool Handle::server_busy() const {
    const Serve *v = p->srv;
    return v && (!v->inflight.empty() || !v->waiting.empty());
}

bool Handle::server_has(int64_t id) const { return p->srv && p->srv->reqs.count(id) > 0; }

int64_t Handle::server_oldest(int64_t *id) const {
    const Serve *v = p->srv;
    if (!v || v->finished.empty()) return -1;
    *id = v->finished.front();
    return v->reqs.at(*id).fin_seq;
}

// ---------------------------------------------------------------- two lanes

namespace {

// largest row length of a device CSR (offsets only)
__global__ void k_max_row_len(const int64_t *__restrict__ off, int64_t n, unsigned long long *out) {
    unsigned long long mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = off[i + 1] - off[i];
        if (d > 0 && (unsigned long long)d > mx) mx = (unsigned long long)d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

}  // namespace

struct Server::State {
    leiden_params prm{};
    int64_t cap_v = 0, cap_e = 0, budget_arg = 0;
    int32_t cap_g = 0;
    cudaStream_t s = nullptr;
    ServeShared sh;
    Handle lane[2];
    bool ready[2] = {false, false};
    double vtime[2] = {0.0, 0.0};  // device time (ms) each lane's steps have taken
    std::map<int64_t, int> lane_of;  // unread request ids -> lane
    unsigned long long *dmax = nullptr;
    int64_t steps = 0;
};

Server::Server() : st(new State) {}

Server::~Server() {
    if (st->dmax) cudaFreeAsync(st->dmax, st->s);
    delete st;  // the lanes free their own state
}

leiden_status Server::init(const leiden_params &prm, int64_t max_vertices, int64_t max_entries, int32_t max_graphs,
                           int64_t device_budget, void *stream) {
    State &v = *st;
    v.prm = prm;
    v.cap_v = max_vertices;
    v.cap_e = max_entries;
    v.cap_g = max_graphs;
    v.budget_arg = device_budget;
    v.s = static_cast<cudaStream_t>(stream);
    // lane 0 now (it checks the parameters and fixes the budget), lane 1 when
    // its first graph comes
    ST(v.lane[0].server_init(prm, max_vertices, max_entries, max_graphs, device_budget, stream, &v.sh));
    v.ready[0] = true;
    if (cudaMallocAsync((void **)&v.dmax, sizeof(unsigned long long), v.s) != cudaSuccess) {
        set_last_error("device allocation for the server failed");
        return LEIDEN_ERR_OOM;
    }
    return LEIDEN_OK;
}

leiden_status Server::submit(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const float *w,
                             int where, int64_t *id) {
    State &v = *st;
    int k = 0;
    // the lane of a graph: its schedule's layer cap (reading S0); with a fixed
    // cap every graph shares lane 0. Malformed arguments are left to the
    // lane's own checks.
    if (v.prm.schedule_layers == 0 && n > 0 && nnz > 0 && off && (where == LEIDEN_HOST || where == LEIDEN_DEVICE) &&
        n <= v.cap_v && nnz <= v.cap_e) {
        int64_t maxdeg = 0;
        if (where == LEIDEN_HOST) {
            for (int64_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, off[i + 1] - off[i]);
        } else {
            unsigned long long h = 0;
            CK(cudaMemsetAsync(v.dmax, 0, sizeof(unsigned long long), v.s));
            const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
            k_max_row_len<<<(unsigned)blocks, 256, 0, v.s>>>(off, n, v.dmax);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&h, v.dmax, sizeof(h), cudaMemcpyDeviceToHost, v.s));
            CK(cudaStreamSynchronize(v.s));
            maxdeg = (int64_t)std::min<unsigned long long>(h, (unsigned long long)nnz);
        }
        k = auto_layers(maxdeg, n, nnz) == kLayersHeavy ? 1 : 0;
    }
    if (!v.ready[k]) {
        ST(v.lane[k].server_init(v.prm, v.cap_v, v.cap_e, v.cap_g, v.budget_arg, v.s, &v.sh));
        v.ready[k] = true;
    }
    const bool was_busy = v.lane[k].server_busy();
    ST(v.lane[k].server_submit(n, nnz, off, idx, w, where, id));
    v.lane_of[*id] = k;
    const int o = k ^ 1;
    if (!was_busy && v.ready[o] && v.lane[o].server_busy())  // starts level: no burst to catch up
        v.vtime[k] = std::max(v.vtime[k], v.vtime[o]);
    return LEIDEN_OK;
}

leiden_status Server::step(int32_t *finished) {
    State &v = *st;
    if (finished) *finished = 0;
    const int first = v.vtime[0] <= v.vtime[1] ? 0 : 1;
    // the busy lane with less device time first; if it runs no pass (its
    // waiting graphs do not fit the budget the other lane holds), the other
    int32_t total = 0;
    for (int k : {first, first ^ 1}) {
        if (!v.ready[k] || !v.lane[k].server_busy()) continue;
        leiden_server_state a{}, b{};
        ST(v.lane[k].server_info(&a));
        int32_t f = 0;
        const auto t0 = std::chrono::steady_clock::now();
        ST(v.lane[k].server_step(&f));  // returns after the step's work is done
        v.vtime[k] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        ST(v.lane[k].server_info(&b));
        total += f;
        if (b.steps > a.steps) {
            v.steps++;
            break;
        }
    }
    if (finished) *finished = total;
    return LEIDEN_OK;
}

leiden_status Server::next(int64_t *id) {
    State &v = *st;
    if (!id) {
        set_last_error("request_id is NULL");
        return LEIDEN_ERR_INVALID;
    }
    *id = -1;
    int64_t best = -1;
    for (int k = 0; k < 2; ++k) {
        if (!v.ready[k]) continue;
        int64_t rid = -1;
        const int64_t seq = v.lane[k].server_oldest(&rid);
        if (seq >= 0 && (best < 0 || seq < best)) {
            best = seq;
            *id = rid;
        }
    }
    return LEIDEN_OK;
}

leiden_status Server::result(int64_t id, int32_t *membership, int where, double *q, int32_t *passes,
                             int64_t *communities) {
    State &v = *st;
    auto it = v.lane_of.find(id);
    if (it == v.lane_of.end()) {
        set_last_error("unknown or unfinished request id");
        return LEIDEN_ERR_INVALID;
    }
    const int k = it->second;
    const leiden_status s = v.lane[k].server_result(id, membership, where, q, passes, communities);
    if (!v.lane[k].server_has(id)) v.lane_of.erase(it);  // released by the read
    return s;
}

leiden_status Server::info(leiden_server_state *out) const {
    const State &v = *st;
    if (!out) {
        set_last_error("out is NULL");
        return LEIDEN_ERR_INVALID;
    }
    leiden_server_state t{};
    *out = leiden_server_state{};
    for (int k = 0; k < 2; ++k) {
        if (!v.ready[k]) continue;
        ST(v.lane[k].server_info(&t));
        out->waiting += t.waiting;
        out->in_flight += t.in_flight;
        out->finished += t.finished;
        out->union_vertices += t.union_vertices;
        out->union_entries += t.union_entries;
        out->device_bytes = t.device_bytes;  // shared
    }
    out->steps = v.steps;
    return LEIDEN_OK;
}

}  // namespace lgb
