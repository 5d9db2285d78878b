// extern "C" entry points declared in include/leiden.h.
#include <new>

#include "engine_impl.h"

struct leiden_graph_s {
    lgb::Handle h;
};
struct leiden_server_s {
    lgb::Server h;
};

extern "C" {

void leiden_tuning_default(leiden_tuning *t) {
    if (t) lgb::tuning_default(*t);
}

leiden_status leiden_set_tuning(leiden_graph_t g, const leiden_tuning *t) {
    if (!g || !t) {
        lgb::set_last_error("NULL handle or tuning");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.set_tuning(*t);
}

leiden_status leiden_get_tuning(leiden_graph_t g, leiden_tuning *t) {
    if (!g) {
        lgb::set_last_error("NULL handle");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.get_tuning(t);
}

leiden_status leiden_tuning_lookup(const char *cache_path, const char *gpu_name, int64_t n, int64_t nnz,
                                   int64_t max_degree, leiden_tuning *out) {
    if (!cache_path || !gpu_name || !out || n < 0 || nnz < 0 || max_degree < 0) {
        lgb::set_last_error("invalid arguments to leiden_tuning_lookup");
        return LEIDEN_ERR_INVALID;
    }
    return lgb::tuning_lookup(cache_path, gpu_name, n, nnz, max_degree, *out);
}

leiden_status leiden_test_fail_allocation(int64_t after) {
    lgb::g_fail_alloc_after.store(after < 0 ? -1 : after);
    return LEIDEN_OK;
}

void leiden_params_default(leiden_params *p) {
    if (!p) return;
    p->resolution = 1.0;
    p->tolerance = 0.01;
    p->aggregation_tolerance = 0.8;
    p->tolerance_drop = 10.0;
    p->max_iterations = 20;
    p->max_passes = 10;
    p->mode = LEIDEN_ASYNC;
    p->flags = 0;
    p->schedule_layers = 0;
    p->schedule_buckets = 16;
    p->seed = 0;
}

leiden_status leiden_create(leiden_graph_t *out, int64_t n, int64_t nnz, const int64_t *offsets,
                            const int32_t *indices, const float *weights, int32_t where, int32_t validate,
                            void *stream) {
    if (!out) {
        lgb::set_last_error("out is NULL");
        return LEIDEN_ERR_INVALID;
    }
    *out = nullptr;
    if (n < 0 || n > 0x7fffffffLL || nnz < 0 || !offsets || (nnz > 0 && !indices) ||
        (where != LEIDEN_HOST && where != LEIDEN_DEVICE)) {
        lgb::set_last_error("invalid CSR arguments");
        return LEIDEN_ERR_INVALID;
    }
    if (where == LEIDEN_HOST) {  // host arrays are checked here, device arrays by validate
        if (offsets[0] != 0 || offsets[n] != nnz) {
            lgb::set_last_error("offsets[0] must be 0 and offsets[n] must equal nnz");
            return LEIDEN_ERR_INVALID;
        }
    }
    leiden_graph_s *g = new (std::nothrow) leiden_graph_s;
    if (!g) {
        lgb::set_last_error("host allocation failed");
        return LEIDEN_ERR_OOM;
    }
    leiden_status st = g->h.create(n, nnz, offsets, indices, weights, where, validate, stream);
    if (st != LEIDEN_OK) {
        delete g;
        return st;
    }
    *out = g;
    return LEIDEN_OK;
}

leiden_status leiden_run(leiden_graph_t g, const leiden_params *p, int32_t *membership, int32_t where,
                         double *modularity, leiden_stats *stats) {
    if (!g || !p) {
        lgb::set_last_error("NULL handle or params");
        return LEIDEN_ERR_INVALID;
    }
    if (where != LEIDEN_HOST && where != LEIDEN_DEVICE) {
        lgb::set_last_error("invalid where");
        return LEIDEN_ERR_INVALID;
    }
    if (g->h.num_graphs() != 1) {
        lgb::set_last_error("leiden_run takes a single graph; use leiden_batch_run for a batch");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.run(*p, membership, where, modularity, stats);
}

leiden_status leiden_batch_create(leiden_graph_t *out, int32_t num_graphs, const int64_t *vtx_seg, int64_t nnz,
                                  const int64_t *offsets, const int32_t *indices, const float *weights, int32_t where,
                                  int32_t validate, void *stream) {
    if (!out) {
        lgb::set_last_error("out is NULL");
        return LEIDEN_ERR_INVALID;
    }
    *out = nullptr;
    if (num_graphs < 1 || !vtx_seg || vtx_seg[0] != 0) {
        lgb::set_last_error("a batch needs num_graphs >= 1 and vtx_seg[0] == 0");
        return LEIDEN_ERR_INVALID;
    }
    for (int32_t g = 0; g < num_graphs; ++g)
        if (vtx_seg[g + 1] < vtx_seg[g]) {
            lgb::set_last_error("vtx_seg must be non-decreasing");
            return LEIDEN_ERR_INVALID;
        }
    const int64_t n = vtx_seg[num_graphs];
    if (n > 0x7fffffffLL || nnz < 0 || !offsets || (nnz > 0 && !indices) ||
        (where != LEIDEN_HOST && where != LEIDEN_DEVICE)) {
        lgb::set_last_error("invalid CSR arguments");
        return LEIDEN_ERR_INVALID;
    }
    if (where == LEIDEN_HOST && (offsets[0] != 0 || offsets[n] != nnz)) {
        lgb::set_last_error("offsets[0] must be 0 and offsets[n] must equal nnz");
        return LEIDEN_ERR_INVALID;
    }
    leiden_graph_s *g = new (std::nothrow) leiden_graph_s;
    if (!g) {
        lgb::set_last_error("host allocation failed");
        return LEIDEN_ERR_OOM;
    }
    leiden_status st = g->h.create(n, nnz, offsets, indices, weights, where, validate, stream, num_graphs, vtx_seg);
    if (st != LEIDEN_OK) {
        delete g;
        return st;
    }
    *out = g;
    return LEIDEN_OK;
}

leiden_status leiden_batch_run(leiden_graph_t g, const leiden_params *p, int32_t *membership, int32_t where,
                               double *modularity, leiden_stats *stats) {
    if (!g || !p) {
        lgb::set_last_error("NULL handle or params");
        return LEIDEN_ERR_INVALID;
    }
    if (where != LEIDEN_HOST && where != LEIDEN_DEVICE) {
        lgb::set_last_error("invalid where");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.run(*p, membership, where, modularity, stats);
}

leiden_status leiden_batch_info(leiden_graph_t g, int32_t *num_graphs, int32_t *passes, int64_t *communities) {
    if (!g) {
        lgb::set_last_error("NULL handle");
        return LEIDEN_ERR_INVALID;
    }
    if (num_graphs) *num_graphs = g->h.num_graphs();
    if (!passes && !communities) return LEIDEN_OK;
    return g->h.graph_info(passes, communities);
}

leiden_status leiden_server_create(leiden_server_t *out, const leiden_params *p, int64_t max_vertices,
                                   int64_t max_entries, int32_t max_graphs, int64_t device_budget, void *stream) {
    if (!out || !p) {
        lgb::set_last_error("out or params is NULL");
        return LEIDEN_ERR_INVALID;
    }
    *out = nullptr;
    leiden_server_s *sv = new (std::nothrow) leiden_server_s;
    if (!sv) {
        lgb::set_last_error("host allocation failed");
        return LEIDEN_ERR_OOM;
    }
    leiden_status st = sv->h.init(*p, max_vertices, max_entries, max_graphs, device_budget, stream);
    if (st != LEIDEN_OK) {
        delete sv;
        return st;
    }
    *out = sv;
    return LEIDEN_OK;
}

leiden_status leiden_server_submit(leiden_server_t s, int64_t n, int64_t nnz, const int64_t *offsets,
                                   const int32_t *indices, const float *weights, int32_t where, int64_t *request_id) {
    if (!s) {
        lgb::set_last_error("NULL server");
        return LEIDEN_ERR_INVALID;
    }
    return s->h.submit(n, nnz, offsets, indices, weights, where, request_id);
}

leiden_status leiden_server_step(leiden_server_t s, int32_t *finished) {
    if (!s) {
        lgb::set_last_error("NULL server");
        return LEIDEN_ERR_INVALID;
    }
    return s->h.step(finished);
}

leiden_status leiden_server_next(leiden_server_t s, int64_t *request_id) {
    if (!s) {
        lgb::set_last_error("NULL server");
        return LEIDEN_ERR_INVALID;
    }
    return s->h.next(request_id);
}

leiden_status leiden_server_result(leiden_server_t s, int64_t request_id, int32_t *membership, int32_t where,
                                   double *modularity, int32_t *passes, int64_t *communities) {
    if (!s) {
        lgb::set_last_error("NULL server");
        return LEIDEN_ERR_INVALID;
    }
    if (where != LEIDEN_HOST && where != LEIDEN_DEVICE) {
        lgb::set_last_error("invalid where");
        return LEIDEN_ERR_INVALID;
    }
    return s->h.result(request_id, membership, where, modularity, passes, communities);
}

leiden_status leiden_server_info(leiden_server_t s, leiden_server_state *out) {
    if (!s) {
        lgb::set_last_error("NULL server");
        return LEIDEN_ERR_INVALID;
    }
    return s->h.info(out);
}

leiden_status leiden_server_destroy(leiden_server_t s) {
    delete s;
    return LEIDEN_OK;
}

leiden_status leiden_destroy(leiden_graph_t g) {
    delete g;
    return LEIDEN_OK;
}

leiden_status leiden_modularity(int64_t n, const int64_t *offsets, const int32_t *indices, const float *weights,
                                const int32_t *membership, double gamma, void *stream, double *q_out) {
    return lgb::modularity_device(n, offsets, indices, weights, membership, gamma,
                                  static_cast<cudaStream_t>(stream), q_out);
}

leiden_status leiden_disconnected(int64_t n, const int64_t *offsets, const int32_t *indices, const int32_t *membership,
                                  void *stream, int64_t *count) {
    return lgb::disconnected_device(n, offsets, indices, membership, static_cast<cudaStream_t>(stream), count);
}

leiden_status leiden_csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                                    int32_t where, int32_t drop_self_loops, int32_t combine, int64_t *offsets,
                                    int32_t *indices, float *weights, int64_t *nnz, void *stream) {
    return lgb::csr_from_edges(n, m, src, dst, w, where, drop_self_loops, combine, offsets, indices, weights, nnz,
                               static_cast<cudaStream_t>(stream));
}

leiden_status leiden_trace_get(leiden_graph_t g, int32_t pass, int32_t what, void *dst, int64_t *count) {
    if (!g) {
        lgb::set_last_error("NULL handle");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.trace_get(pass, what, dst, count);
}

leiden_status leiden_profile_get(leiden_graph_t g, leiden_kernel_profile *out) {
    if (!g) {
        lgb::set_last_error("NULL handle");
        return LEIDEN_ERR_INVALID;
    }
    return g->h.profile_get(out);
}

const char *leiden_status_string(int32_t s) {
    switch (s) {
        case LEIDEN_OK: return "LEIDEN_OK";
        case LEIDEN_ERR_INVALID: return "LEIDEN_ERR_INVALID";
        case LEIDEN_ERR_NOT_SYMMETRIC: return "LEIDEN_ERR_NOT_SYMMETRIC";
        case LEIDEN_ERR_OOM: return "LEIDEN_ERR_OOM";
        case LEIDEN_ERR_CUDA: return "LEIDEN_ERR_CUDA";
        case LEIDEN_ERR_TIMEOUT: return "LEIDEN_ERR_TIMEOUT";
        case LEIDEN_ERR_UNSUPPORTED: return "LEIDEN_ERR_UNSUPPORTED";
        case LEIDEN_ERR_OVERFLOW: return "LEIDEN_ERR_OVERFLOW";
        default: return "LEIDEN_ERR_UNKNOWN";
    }
}

const char *leiden_last_error(void) { return lgb::last_error(); }

}  // extern "C"
