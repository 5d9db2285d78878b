// Host engine behind the C ABI (include/leiden.h).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/leiden.h"

namespace lgb {

void set_last_error(const std::string &s);
const char *last_error();

struct ServeShared;

class Handle {
  public:
    Handle();
    ~Handle();
    Handle(const Handle &) = delete;
    Handle &operator=(const Handle &) = delete;
    // one graph (num_graphs = 1, vtx_seg null) or a batch: graph g owns
    // vertices [vtx_seg[g], vtx_seg[g+1]) and its indices are local to it
    leiden_status create(int64_t n, int64_t nnz, const int64_t *offsets, const int32_t *indices, const float *weights,
                         int where, int validate, void *stream, int32_t num_graphs = 1,
                         const int64_t *vtx_seg = nullptr);
    // modularity: one value, or num_graphs values for a batch (host)
    leiden_status run(const leiden_params &p, int32_t *membership, int where, double *modularity, leiden_stats *stats);
    int32_t num_graphs() const;
    // per-graph passes and communities of the last run (host arrays)
    leiden_status graph_info(int32_t *passes, int64_t *communities) const;
    // serving (continuous batching): capacity for the graphs in flight; a
    // step admits waiting graphs at the pass boundary and runs one pass of
    // every graph in flight
    leiden_status server_init(const leiden_params &p, int64_t max_vertices, int64_t max_entries, int32_t max_graphs,
                              int64_t device_budget, void *stream, ServeShared *shared = nullptr);
    leiden_status server_submit(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const float *w,
                                int where, int64_t *id);
    leiden_status server_step(int32_t *finished);
    leiden_status server_next(int64_t *id);
    leiden_status server_result(int64_t id, int32_t *membership, int where, double *q, int32_t *passes,
                                int64_t *communities);
    leiden_status server_info(leiden_server_state *out) const;
    bool server_busy() const;  // graphs in flight or waiting
    bool server_has(int64_t id) const;  // a request the lane still holds
    // finishing order (ServeShared::fin_seq) of the oldest unread result and
    // its id, or -1 when no result is unread
    int64_t server_oldest(int64_t *id) const;
    leiden_status trace_get(int pass, int what, void *dst, int64_t *count) const;
    // launch shape of later runs (leiden_tuning)
    leiden_status set_tuning(const leiden_tuning &t);
    leiden_status get_tuning(leiden_tuning *t) const;
    leiden_status profile_get(leiden_kernel_profile *out) const;

    struct Impl;  // device state (engine_impl.h)

  private:
    Impl *p;
};

// A serving handle of two lanes. Each lane is a union of its own
// (Handle::server_*): graphs whose schedule takes the light layer cap go to
// lane 0, heavy-tailed ones (reading S0) to lane 1, so that no graph's sweeps
// are paced by another's thousand-layer schedule. A step runs one pass of
// one lane: of the busy lanes, the one that has had the least device time
// (a lane that becomes busy starts level with the other), so each lane holds
// at least half the GPU while both have work. Ids, the finishing order and
// the device budget are shared; results come out in finishing order.
class Server {
  public:
    Server();
    ~Server();
    Server(const Server &) = delete;
    Server &operator=(const Server &) = delete;
    leiden_status init(const leiden_params &p, int64_t max_vertices, int64_t max_entries, int32_t max_graphs,
                       int64_t device_budget, void *stream);
    leiden_status submit(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const float *w, int where,
                         int64_t *id);
    leiden_status step(int32_t *finished);
    leiden_status next(int64_t *id);
    leiden_status result(int64_t id, int32_t *membership, int where, double *q, int32_t *passes,
                         int64_t *communities);
    leiden_status info(leiden_server_state *out) const;

    struct State;

  private:
    State *st;
};

leiden_status disconnected_device(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *memb,
                                  cudaStream_t s, int64_t *count);
leiden_status csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w, int where,
                             int drop_self, int combine, int64_t *offsets, int32_t *indices, float *weights,
                             int64_t *nnz_io, cudaStream_t s);
// launch-shape defaults, range check and the autotuner cache (tuning.cu)
void tuning_default(leiden_tuning &t);
bool tuning_valid(const leiden_tuning &t);
leiden_status tuning_lookup(const char *path, const char *gpu, int64_t n, int64_t nnz, int64_t maxdeg,
                            leiden_tuning &out);
leiden_status modularity_device(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                const int32_t *memb, double gamma, cudaStream_t s, double *q_out);
// refuses an iteration limit under which one persistent phase of a schedule
// of nsteps steps could count more grid-barrier arrivals than 32 bits hold
leiden_status check_barrier_budget(int32_t max_iterations, int32_t nsteps, bool det, int sm);

}  // namespace lgb
