/*
 * leiden.h -- C ABI of the GB300 (sm_103a) Leiden community-detection library.
 *
 * The library runs the parallel Leiden method of "GVE-Leiden: Fast Leiden
 * Algorithm for Community Detection in Shared Memory Setting" (Sahu, arXiv
 * 2312.13936) on one GPU: the pass loop of Algorithm 1 with local-moving
 * (Algorithm 2), refinement (Algorithm 3) and aggregation (Algorithm 4),
 * threshold scaling and the aggregation-tolerance stop. Every step runs in
 * the library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a leiden_status and never aborts the process.
 *     leiden_last_error() gives a one-line description of the last failure
 *     on the calling thread.
 *   - Graphs are undirected and weighted (paper, Section 3 "Preliminaries":
 *     w_ij = w_ji). They are passed as a symmetric CSR: offsets[n+1] (int64,
 *     offsets[0] = 0, non-decreasing), indices[nnz] (int32 in [0, n)),
 *     weights[nnz] (float32, finite, >= 0; NULL means unit weights). Each
 *     undirected edge appears once in each direction; a self-loop is one
 *     entry and counts once in K_i and in 2m.
 *   - `where` tells where a pointer lives: LEIDEN_HOST or LEIDEN_DEVICE (a
 *     pointer into memory of the current CUDA device, e.g.
 *     torch.Tensor.data_ptr()).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All work of a call is ordered on that stream.
 *   - Inputs are borrowed for the duration of the call; outputs are owned by
 *     the caller; a leiden_graph_t owns its device copies and workspace.
 *   - A handle is not thread-safe; different handles may run concurrently on
 *     different streams.
 */
#ifndef LEIDEN_GB300_H
#define LEIDEN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LEIDEN_OK = 0,
    LEIDEN_ERR_INVALID = -1,       /* bad argument or malformed CSR */
    LEIDEN_ERR_NOT_SYMMETRIC = -2, /* validation found w_ij != w_ji */
    LEIDEN_ERR_OOM = -3,           /* device allocation failed */
    LEIDEN_ERR_CUDA = -4,          /* a CUDA runtime call or kernel failed */
    LEIDEN_ERR_TIMEOUT = -5,       /* a bounded device loop gave up */
    LEIDEN_ERR_UNSUPPORTED = -6,   /* mode/parameter combination not supported */
    LEIDEN_ERR_OVERFLOW = -7       /* exact arithmetic would overflow */
} leiden_status;

enum { LEIDEN_HOST = 0, LEIDEN_DEVICE = 1 };

/* mode: LEIDEN_ASYNC applies local-moving moves inside the kernels as soon
 * as they are decided (the paper's asynchronous execution, Section 4.1);
 * LEIDEN_DETERMINISTIC evaluates each schedule step against the state at
 * the start of the step and decides in exact integer arithmetic (int64
 * sums, 128-bit move keys), so results are reproducible bit for bit
 * (requires integer weights, resolution 1 and 2m < 2^53). */
enum { LEIDEN_ASYNC = 0, LEIDEN_DETERMINISTIC = 1 };

/* flags */
enum {
    LEIDEN_FLAG_VALIDATE = 1u,            /* check symmetry and weights on device */
    LEIDEN_FLAG_REFINE_SINGLE_SWEEP = 2u, /* one refinement sweep, as Algorithm 3 prints it */
    LEIDEN_FLAG_TRACE = 4u,               /* keep per-pass intermediate results (leiden_trace_get) */
    LEIDEN_FLAG_PROFILE = 8u,             /* time every sweep/aggregation launch (leiden_profile_get) */
    LEIDEN_FLAG_STEP_LAUNCHES = 16u,      /* one launch per schedule step and degree bin instead of one
                                             persistent launch per sweep (same results; for testing) */
    LEIDEN_FLAG_REFINE_LABELS = 64u,      /* refine-based super-vertex labels (Section 4.1): every
                                             super-vertex starts the next pass in its own community
                                             instead of its move-based one */
    LEIDEN_FLAG_LOUVAIN = 128u,           /* the Louvain method of the paper's comparison (Section 5):
                                             no refinement phase; each pass aggregates its local-moving
                                             communities, which need not be connected */
    LEIDEN_FLAG_RANDOM_REFINE = 256u,     /* asynchronous mode: randomized refinement (Sections 3.4, 4.1):
                                             an isolated vertex joins a community of positive gain within
                                             its bound with probability proportional to the gain, drawn
                                             from the seed, pass, sweep, vertex and community; the
                                             deterministic mode refuses it (LEIDEN_ERR_UNSUPPORTED) */
    LEIDEN_FLAG_TEST_STALL_BARRIER = 512u /* testing aid for the timeout path: block 1 of every persistent
                                             sweep launch of more than one block ends without arriving at
                                             the grid barrier, and the other blocks wait about a
                                             millisecond instead of about a second before they give up;
                                             the run then returns LEIDEN_ERR_TIMEOUT and the handle stays
                                             usable. Not for production use. */
};

typedef struct {
    double resolution;            /* gamma: multiplies the null-model term of Eq. 1 and Eq. 2; default 1 */
    double tolerance;             /* tau: initial per-iteration tolerance (Algorithm 2); default 0.01 */
    double aggregation_tolerance; /* tau_agg: stop when |Gamma|/|V'| exceeds it (Algorithm 1); default 0.8 */
    double tolerance_drop;        /* TOLERANCE_DROP: tau /= drop after each pass (Algorithm 1); default 10 */
    int32_t max_iterations;       /* MAX_ITERATIONS per phase (Algorithm 2); default 20. The persistent
                                     sweep's grid barrier counts arrivals in 32 bits, so a limit with
                                     max_iterations * (8 steps + 4) * resident blocks > 2^32 - 1
                                     (steps = layers - 1 + buckets) is LEIDEN_ERR_INVALID: on a GB300 (608
                                     blocks) above 869 with the 1000-layer schedule, 18,589 with 32 */
    int32_t max_passes;           /* MAX_PASSES (Algorithm 1; not given in the paper); default 10 */
    int32_t mode;                 /* LEIDEN_ASYNC or LEIDEN_DETERMINISTIC */
    uint32_t flags;               /* LEIDEN_FLAG_* */
    int32_t schedule_layers;      /* L: priority layers of the sweep schedule (L - 1 + B at most
                                     1023); 0 (default): 1000 for a heavy-tailed graph (largest
                                     degree above 64 times the mean degree nnz/n), else 32, graph
                                     by graph in a batch or server */
    int32_t schedule_buckets;     /* B: priority buckets after the last layer; default 16 */
    uint64_t seed;                /* seed of the schedule's vertex priorities; default 0 */
} leiden_params;

typedef struct {
    int32_t passes;               /* passes executed */
    int32_t move_iterations;      /* local-moving sweeps, all passes */
    int32_t refine_iterations;    /* refinement sweeps, all passes */
    int32_t reserved;
    int64_t communities;          /* communities in the returned membership */
    double modularity;            /* Eq. 1 of the result on the input graph */
    double ms_total;              /* device time of leiden_run (CUDA events) */
    double ms_move, ms_refine, ms_aggregate, ms_other; /* per-phase device time */
    int64_t kernel_launches;      /* kernels launched by the call */
} leiden_stats;

/* Per-kernel-class profile of the last leiden_run made with
 * LEIDEN_FLAG_PROFILE. Class index = phase * 8 + bin, with phase 0 the
 * local-moving sweep (Algorithm 2), 1 the refinement sweep (Algorithm 3), 2
 * the aggregation (Algorithm 4), and bin 1..6 the degree bin (degree <= 8:
 * a thread per vertex, or a tile of 8 lanes per community; <= 16 and <= 32:
 * a tile of 16/32 lanes; <= 256: warp table; <= 2048: block table; larger:
 * global-memory table, in the aggregation one packed table per community
 * that every member vertex inserts into); bin 7 is unused; bin 0 is the
 * persistent kernel that runs a whole sweep (all bins) in one launch. bytes counts the
 * algorithmic bytes of the launches (each array element the method reads or
 * writes counted once at its own size; random gathers count their element,
 * not the memory sector), from work counters the kernels accumulate. */
typedef struct {
    int64_t launches;  /* kernel launches of this class */
    double ms;         /* device time of those launches (CUDA events on the run's stream) */
    double bytes;      /* algorithmic bytes */
    int64_t items;     /* vertices (communities) evaluated */
    int64_t skipped;   /* listed vertices skipped (pruned or not isolated) */
    int64_t edges;     /* CSR entries scanned */
    int64_t distinct;  /* distinct neighbour communities accumulated */
    int64_t moved;     /* moves made or proposed (entries written, aggregation) */
} leiden_kernel_profile;
enum { LEIDEN_PROFILE_CLASSES = 24 };

typedef struct leiden_graph_s *leiden_graph_t;
typedef struct leiden_server_s *leiden_server_t;

/* State of a serving handle (filled by leiden_server_info). */
typedef struct {
    int32_t waiting;          /* submitted graphs not yet in flight */
    int32_t in_flight;        /* graphs in the lanes' unions */
    int32_t finished;         /* finished graphs whose results are unread */
    int32_t reserved;
    int64_t union_vertices;   /* vertices of the unions' current graphs */
    int64_t union_entries;    /* CSR entries of the unions' current graphs */
    int64_t device_bytes;     /* device bytes held by the requests' own buffers */
    int64_t steps;            /* steps that ran a pass */
} leiden_server_state;

/* Fill *p with the defaults listed above. */
void leiden_params_default(leiden_params *p);

/* Create a handle from a symmetric CSR (Section 3 graph model). The arrays
 * are copied into device memory owned by the handle (from host or device
 * memory, per `where`) and a workspace sized for the graph is reserved.
 * n >= 0, nnz = offsets[n]; weights may be NULL (unit weights). With
 * `validate` != 0 the CSR is checked on the device (offsets monotone,
 * indices in range, weights finite and >= 0, w_ij == w_ji); failures return
 * LEIDEN_ERR_INVALID or LEIDEN_ERR_NOT_SYMMETRIC and *out stays NULL. */
leiden_status leiden_create(leiden_graph_t *out, int64_t n, int64_t nnz, const int64_t *offsets,
                            const int32_t *indices, const float *weights, int32_t where, int32_t validate,
                            void *stream);

/* Run Algorithm 1 on the handle's graph (a handle from leiden_create;
 * batch handles of more than one graph return LEIDEN_ERR_INVALID). membership (n int32, host or device
 * per `where`) receives canonical labels: community ids are ranks of each
 * community's smallest vertex id. *modularity (nullable) receives Eq. 1 of
 * the result on the input graph; *stats (nullable) the run statistics. The
 * call returns after the results are written (it synchronises `stream`). */
leiden_status leiden_run(leiden_graph_t g, const leiden_params *p, int32_t *membership, int32_t where,
                         double *modularity, leiden_stats *stats);

/* Release the handle and its device memory. NULL is accepted. */
leiden_status leiden_destroy(leiden_graph_t g);

/* Batches: many independent graphs, each run through Algorithm 1 exactly as
 * leiden_run would run it alone, solved together by one set of launches per
 * pass (the paper runs one graph at a time; the batch is a disjoint union
 * whose graphs keep their own 2m, their own convergence and stop tests and
 * their own pass count, and leave the union when they stop).
 *
 * Create a batch handle from num_graphs >= 1 graphs packed one after the
 * other: graph g owns vertices [vtx_seg[g], vtx_seg[g+1]) of the packed CSR
 * (vtx_seg: num_graphs+1 int64 in HOST memory, vtx_seg[0] = 0,
 * non-decreasing; empty graphs allowed), offsets has vtx_seg[num_graphs]+1
 * entries indexing the packed indices/weights (nnz = offsets[n]), and the
 * indices of graph g are LOCAL to it (in [0, n_g)): each graph's CSR is
 * appended unchanged but for the shift of its offsets. Other arguments and
 * checks as for leiden_create; a local index outside its graph returns
 * LEIDEN_ERR_INVALID. In deterministic mode the 2m < 2^53 rule holds per
 * graph. */
leiden_status leiden_batch_create(leiden_graph_t *out, int32_t num_graphs, const int64_t *vtx_seg, int64_t nnz,
                                  const int64_t *offsets, const int32_t *indices, const float *weights, int32_t where,
                                  int32_t validate, void *stream);

/* Run Algorithm 1 on every graph of a batch handle. membership (n int32,
 * host or device per `where`) receives every graph's canonical labels, local
 * to the graph (ranks of each community's smallest vertex inside it);
 * modularity (nullable, num_graphs doubles in HOST memory) receives Eq. 1 of
 * every graph's result on its input; stats (nullable) describes the whole
 * batch (passes of the union, total communities, mean modularity). Trace and
 * per-step launches are single-graph features (LEIDEN_ERR_UNSUPPORTED). A
 * handle from leiden_create is a batch of one graph. */
leiden_status leiden_batch_run(leiden_graph_t g, const leiden_params *p, int32_t *membership, int32_t where,
                               double *modularity, leiden_stats *stats);

/* Serving with continuous batching. A server holds graphs in flight, each
 * at its own pass of Algorithm 1, in two lanes: graphs whose schedule takes
 * the light layer cap in lane 0, heavy-tailed graphs (largest degree times n
 * above 64 nnz, the 1000-layer schedule of schedule_layers = 0) in lane 1;
 * with a fixed schedule_layers every graph is in lane 0. Each lane is a
 * union of its graphs. leiden_server_step runs one pass of one lane -- of
 * the lanes with graphs in flight or waiting, the one whose steps have taken
 * the least time so far (a lane that becomes busy starts level with the
 * other), so that light graphs are not paced by a heavy graph's schedule and
 * each lane holds at least half the GPU while both have work. The step
 * admits that lane's waiting graphs at the pass boundary (first come, first
 * served, while a slot, union capacity and the device budget allow), then
 * runs one pass of every graph in it with one set of launches; graphs that
 * stop leave with their results. Every graph's result is the one leiden_run
 * gives alone (bit for bit in deterministic mode). The caller drives the
 * loop: submit graphs as they arrive, call step, read finished results.
 * Capacities and max_graphs hold per lane; lane 1 reserves its workspace
 * when its first graph is submitted. The device budget is shared.
 *
 * Create a server for graphs of up to max_vertices vertices and max_entries
 * CSR entries in flight together (one graph may not exceed either), at most
 * max_graphs graphs in flight, and device_budget bytes for the submitted
 * graphs' own buffers (CSR copy and result; <= 0: half the free device
 * memory after the server's workspace). p fixes the parameters of every run
 * (LEIDEN_FLAG_TRACE, _PROFILE and _STEP_LAUNCHES are ignored). */
leiden_status leiden_server_create(leiden_server_t *out, const leiden_params *p, int64_t max_vertices,
                                   int64_t max_entries, int32_t max_graphs, int64_t device_budget, void *stream);

/* Submit one graph (a symmetric CSR with indices in [0, n), as for
 * leiden_create; it is checked as with validate). The arrays are copied at
 * once: to device memory when the budget allows, else to host memory until
 * it does. *request_id receives the graph's id. Graphs without vertices are
 * finished at once. Returns LEIDEN_ERR_INVALID for a graph larger than the
 * server's capacity, LEIDEN_ERR_OOM for a graph whose own buffers
 * (8 (n + 1) + 4 n + 8 nnz bytes) exceed the device budget, since it could
 * never be admitted; in deterministic mode LEIDEN_ERR_UNSUPPORTED or
 * LEIDEN_ERR_OVERFLOW as leiden_run would. */
leiden_status leiden_server_submit(leiden_server_t s, int64_t n, int64_t nnz, const int64_t *offsets,
                                   const int32_t *indices, const float *weights, int32_t where, int64_t *request_id);

/* One step of one lane: admit, run one pass of every graph in flight in
 * the lane, finish the graphs that stop. *finished (nullable) receives the number of graphs finished by
 * the step. Returns at once when nothing is in flight or waiting. */
leiden_status leiden_server_step(leiden_server_t s, int32_t *finished);

/* Id of the earliest finished graph whose result is unread, or -1. */
leiden_status leiden_server_next(leiden_server_t s, int64_t *request_id);

/* Read and release the result of a finished graph: membership (n int32,
 * host or device per `where`; canonical labels as leiden_run gives them),
 * and (nullable) modularity, passes and communities. Returns
 * LEIDEN_ERR_INVALID for an unknown or unfinished id, or the graph's own
 * error status if it failed when it was copied to the device. */
leiden_status leiden_server_result(leiden_server_t s, int64_t request_id, int32_t *membership, int32_t where,
                                   double *modularity, int32_t *passes, int64_t *communities);

/* Current state of the server (host struct). */
leiden_status leiden_server_info(leiden_server_t s, leiden_server_state *out);

/* Release the server, its workspace and every graph it holds. NULL is accepted. */
leiden_status leiden_server_destroy(leiden_server_t s);

/* Per-graph results of the last run on the handle: passes executed and
 * communities found (host arrays of num_graphs entries; either may be
 * NULL). *num_graphs (nullable) receives the handle's graph count. */
leiden_status leiden_batch_info(leiden_graph_t g, int32_t *num_graphs, int32_t *passes, int64_t *communities);

/* Modularity (Eq. 1 with resolution gamma) of `membership` (n labels in
 * [0, n)) on a symmetric CSR. All pointers are device pointers; the result
 * is written to *q_out (host). Device scratch of 16 bytes per vertex is
 * taken from the stream-ordered allocator for the duration of the call. */
leiden_status leiden_modularity(int64_t n, const int64_t *offsets, const int32_t *indices, const float *weights,
                                const int32_t *membership, double gamma, void *stream, double *q_out);

/* Number of communities of `membership` (n labels in [0, n)) whose vertices
 * do not form one connected subgraph of the symmetric CSR (Appendix A.1,
 * Algorithm 5; the paper runs a BFS per community, this computes the
 * components of the intra-community subgraph for all communities at once).
 * All pointers are device pointers; the result is written to *count (host).
 * Device scratch of 8 bytes per vertex comes from the stream-ordered
 * allocator. LEIDEN_ERR_INVALID for labels outside [0, n). */
leiden_status leiden_disconnected(int64_t n, const int64_t *offsets, const int32_t *indices, const int32_t *membership,
                                  void *stream, int64_t *count);

/* Modularity as leiden_modularity computes it, without allocating any
 * device memory. The paper has no counterpart: this entry point is for
 * callers that cannot allocate device memory when they need the score (a
 * host framework that owns all device memory through its own pool, a
 * process at its memory cap, a path that must not call an allocator). Its
 * scratch is a fixed static device array (8 MiB + 32 bytes) that every GPU
 * loading the library keeps until the process exits, so n is limited to
 * 1,048,576 vertices (larger n returns LEIDEN_ERR_INVALID). The first call
 * on a device looks up the array's address there and keeps it; make that
 * call before any stream capture, and do not call this entry point again
 * after a reset of the device (cudaDeviceReset) in the same process. All calls on a device share the array: calls whose work
 * overlaps on the GPU race and must be serialised by the caller. Arguments
 * and result as for leiden_modularity. */
leiden_status leiden_modularity_noalloc(int64_t n, const int64_t *offsets, const int32_t *indices,
                                        const float *weights, const int32_t *membership, double gamma, void *stream,
                                        double *q_out);

/* Edge list to symmetric CSR on the GPU: the input preparation of the
 * paper's experiments (edges undirected, reverse edges added, weight 1 by
 * default; Section 5.1 and Table 2, |E| counting both directions). The n
 * vertices are 0..n-1; edge e is (src[e], dst[e]) with weight w[e] (w NULL:
 * 1.0), m edges in host (where = LEIDEN_HOST) or device memory (LEIDEN_DEVICE,
 * on stream). An edge u != v gives the entries (u, v) and (v, u); a
 * self-loop gives the single entry (u, u) (one CSR entry, counted once in K
 * and 2m), or none when drop_self_loops != 0. Entries with the same
 * (row, target) are merged: weights summed in fp64 and rounded once to fp32
 * (combine = 0) or the largest kept (combine = 1). Rows list their targets
 * in ascending order. m may exceed 2^31 (positions are 64-bit; rows are
 * sorted in chunks of at most 2^30 entries).
 * Outputs, in the same kind of memory as the input: offsets[n+1], and
 * indices/weights with room for *nnz entries as passed in (2m always
 * suffices); *nnz receives the entry count. Returns LEIDEN_ERR_INVALID for an
 * endpoint outside [0, n), a negative or non-finite weight, a row of more
 * than 2^30 entries before merging, or too small a capacity (*nnz then holds
 * the count needed). Device scratch, allocated and freed on stream: 8 bytes
 * per entry before merging (12 with weights), about 32 bytes per entry of the
 * largest chunk, 32 bytes per vertex, and a device copy of a host edge list. */
leiden_status leiden_csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const float *w,
                                    int32_t where, int32_t drop_self_loops, int32_t combine, int64_t *offsets,
                                    int32_t *indices, float *weights, int64_t *nnz, void *stream);

/* Per-pass trace of the last leiden_run made with LEIDEN_FLAG_TRACE. what:
 * 1 C' at the start of local-moving (int32[n']), 2 C' after local-moving
 * (int32[n']), 3 C' after refinement (int32[n']), 4 counts (int64[4]: n',
 * l_i, l_j, |Gamma|), 5 renumbered C' (int32[n']), 6/7/8/9 the aggregated
 * holey CSR (offsets int64[|Gamma|+1], fill int32[|Gamma|], targets
 * int32[cap], weights float64[cap]; entries past a row's fill are
 * undefined), 10 dendrogram C after the lookup (int32[n0]). With dst NULL,
 * *count receives the element count; otherwise up to *count elements are
 * copied to host memory dst. Returns LEIDEN_ERR_INVALID if the pass or item
 * was not recorded. */
leiden_status leiden_trace_get(leiden_graph_t g, int32_t pass, int32_t what, void *dst, int64_t *count);

/* Copy the LEIDEN_PROFILE_CLASSES entries of the last profiled run into
 * out (host memory). Returns LEIDEN_ERR_INVALID if the last run was not
 * profiled. */
leiden_status leiden_profile_get(leiden_graph_t g, leiden_kernel_profile *out);

/* Launch shape of a handle's kernels: degree-bin bounds and the persistent
 * sweep's grid. None of them changes a result of the deterministic mode (the
 * bins only choose how a vertex's or community's neighbour weights are
 * gathered; every decision is exact), and in the asynchronous mode they
 * change only the order of concurrent updates. The paper's counterpart is
 * the OpenMP dynamic schedule and its chunk size (Section 4.1), which it
 * tuned by measurement; here an autotuner measures the candidates per GPU
 * and graph class and stores the best in a cache (leiden_tuning_lookup). */
typedef struct {
    int32_t thread_max_deg;      /* sweeps: rows up to this many entries take one thread each (1..8); default 8 */
    int32_t warp_max_deg;        /* rows (community entries) up to this many take one warp and a shared-memory
                                    table (32..256); default 256 */
    int32_t block_max_deg;       /* rows up to this many take one block and a shared-memory table (128..2048,
                                    >= warp_max_deg); longer rows take the whole grid (sweeps) or a global
                                    table (aggregation); default 2048 */
    int32_t coop_blocks_per_sm;  /* blocks per SM of the persistent sweep (0: as many as fit); default 0 */
    int32_t vertices_per_block;  /* persistent sweep: vertices per block below a full grid (256..65536);
                                    default 2048 */
    int32_t list_order_min_vertices; /* a pass whose graph has at least this many vertices, no row longer than
                                    block_max_deg and one graph gives its sweeps a copy of its rows and
                                    vertex weights in the order of the schedule's (step, bin) lists, so
                                    that each step reads them contiguously (0: never); default 1048576 */
    int32_t reserved[2];
} leiden_tuning;

/* Fill *t with the defaults listed above. */
void leiden_tuning_default(leiden_tuning *t);

/* Set (or read) the launch shape of a handle (single graph or batch); it
 * holds for its later runs. LEIDEN_ERR_INVALID for a value outside the
 * ranges above. leiden_create and leiden_batch_create start from the
 * defaults, or, when the environment variable LEIDEN_TUNING_CACHE names a
 * cache file, from leiden_tuning_lookup of that cache for the current GPU
 * and the input graph (the defaults when nothing matches). */
leiden_status leiden_set_tuning(leiden_graph_t g, const leiden_tuning *t);
leiden_status leiden_get_tuning(leiden_graph_t g, leiden_tuning *t);

/* Autotuner cache lookup (host only). The cache is a JSON file
 * {"format": 1, "entries": [{"gpu": <name>, "heavy_tailed": 0|1,
 * "log2_vertices": <int>, "log2_mean_degree": <int>, "thread_max_deg": ...,
 * "warp_max_deg": ..., "block_max_deg": ..., "coop_blocks_per_sm": ...,
 * "vertices_per_block": ..., "list_order_min_vertices": ... (optional),
 * other keys ignored}, ...]}; a field an entry leaves out keeps its default. A graph of n
 * vertices, nnz CSR entries and largest degree max_degree has the class
 * (heavy_tailed = max_degree > 64 nnz / n, log2_vertices = round(log2 n),
 * log2_mean_degree = round(log2(nnz / n))); among the entries of gpu_name
 * with the same heavy_tailed, the one nearest in |d log2_vertices| +
 * |d log2_mean_degree| (ties: the first in the file) fills *out.
 * LEIDEN_ERR_INVALID (and *out untouched) if the file cannot be read or
 * parsed or no entry matches. */
leiden_status leiden_tuning_lookup(const char *cache_path, const char *gpu_name, int64_t n, int64_t nnz,
                                   int64_t max_degree, leiden_tuning *out);

/* Testing aid for the out-of-memory paths. The paper has no counterpart.
 * After `after` more successful device allocations made by handles
 * (leiden_create, leiden_batch_create, leiden_run, leiden_batch_run and the
 * server's workspace), the next one fails as if the device were out of
 * memory (LEIDEN_ERR_OOM); the calls made after that allocate normally
 * again. A negative value switches the injection off (the default). The
 * counter is process-wide. Not for production use. */
leiden_status leiden_test_fail_allocation(int64_t after);

/* Human-readable name of a status code. */
const char *leiden_status_string(int32_t status);

/* Description of the last error on the calling thread ("" if none). */
const char *leiden_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LEIDEN_GB300_H */
