// Host-side launchers of the Leiden kernels. Every launcher enqueues work on
// the given stream and returns the launch status; none synchronises.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lgb {

// Degree bins of the sweep and aggregation kernels: a vertex (or community)
// of degree d goes to the first bin whose bound holds it. Bin 0 (no edges)
// is never listed; bin 7 is unused. The bounds of bins 1, 4 and 5 are the
// handle's launch shape (leiden_tuning); the defaults and their largest
// values are:
//   bin 1  d <= 8      one thread per vertex (sweeps), a tile of 8 lanes (aggregation)
//   bin 2  d <= 16     a tile of 16 lanes
//   bin 3  d <= 32     a tile of 32 lanes
//   bin 4  d <= 256    one warp, shared-memory table
//   bin 5  d <= 2048   one block, shared-memory table
//   bin 6  larger      the whole grid (persistent sweep) or one block with a
//                      global-memory table; aggregation: one packed table
//                      per community, filled by all vertices
constexpr int kNumBins = 8;
constexpr int kThreadMaxDeg = 8;
constexpr int kWarpMaxDeg = 256;
constexpr int kBlockMaxDeg = 2048;
constexpr int kWarpSlots = 512;     // 8 warp tables fill the same 48 KB as one block table
constexpr int kBlockSlots = 4096;
constexpr int kBinHub = 6;
// the packed bin-6 tables of the aggregation are cleared and filled in
// chunks of at most this many bytes (12 per slot; 8 in the asynchronous
// mode, whose slot holds key and fp32 value in one word)
constexpr int64_t kAggTableBytes = (int64_t)8 << 30;
// rows longer than this are walked by a whole warp in the schedule kernel
// (its long-row variant, chosen when a graph's degree bound exceeds it) and
// shared by the warps their entries span in the vertex-weight and
// modularity kernels
constexpr int32_t kLongRow = 64;
// the bounds of bins 1, 4 and 5 (at most kThreadMaxDeg, kWarpMaxDeg and
// kBlockMaxDeg, which the kernels' registers and shared-memory tables hold)
struct BinBounds {
    int32_t thread_max = kThreadMaxDeg, warp_max = kWarpMaxDeg, block_max = kBlockMaxDeg;
};
__host__ __device__ inline int degree_bin(int64_t d, const BinBounds &b) {
    return d <= 0 ? 0 : d <= b.thread_max ? 1 : d <= 16 ? 2 : d <= 32 ? 3 : d <= b.warp_max ? 4 : d <= b.block_max ? 5 : 6;
}

// Weights of aggregated graphs in the deterministic mode: exact integers
// up to 2m (below 2^53), held in int64.
using WInt = long long;

// A 128-bit unsigned sum held as two words as a double: (double)hi * 2^64 +
// (double)lo, each conversion and the sum rounded to nearest (the
// deterministic mode's sweep delta-modularity takes exactly these
// roundings, reading S4).
__host__ __device__ inline double u128_words_to_double(unsigned long long lo, unsigned long long hi) {
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// The current graph G' (a holey CSR, paper Fig. 5): row i is
// idx/w[off[i] .. off[i]+deg[i]). Weights are float, or WInt (int64) in
// deterministic mode after the first aggregation.
struct GraphView {
    int64_t n = 0;
    const int64_t *off = nullptr;
    const int32_t *deg = nullptr;
    const int32_t *idx = nullptr;
    const void *w = nullptr;
    bool w_int = false;
};

// State of one local-moving or refinement sweep step.
struct SweepCtx {
    GraphView g;
    bool det = false;         // Det (int64) or Async (fp64) policy
    bool refine = false;      // Algorithm 3 (bounded scan, isolated vertices) vs Algorithm 2
    int32_t *C = nullptr;     // C' (membership of G' vertices)
    const int32_t *CB = nullptr;  // C'_B, community bound (refinement)
    const void *K = nullptr;  // K' (acc type)
    void *Sig = nullptr;      // Sigma' (acc type)
    int32_t *size = nullptr;  // members per community
    uint8_t *unproc = nullptr;    // Algorithm 2 pruning flags (1 = unprocessed)
    int32_t *prop = nullptr;      // proposed target (-1 none)
    long long *gain = nullptr;    // key gain of a proposal: two words per vertex (det, 128 bits) or fp32
    const int32_t *step = nullptr;  // schedule step of every vertex
    // the rows and vertex weights in the order of the (step, bin) lists, or
    // null (read by vertex): list position t's row is lidx/lw[loff[t] ..
    // loff[t+1]) and its weight lK[t] (values as in g and K)
    const int64_t *loff = nullptr;
    const int32_t *lidx = nullptr;
    const void *lw = nullptr;
    const void *lK = nullptr;
    double two_m_f = 0;
    long long two_m_i = 0;
    double gamma = 1;
    int32_t cur_step = 0, cap_step = 0;  // steps >= cap_step may hold adjacent vertices
    int32_t nsteps = 0;                  // persistent sweep: steps and their (step, bin) offsets
    const int64_t *key_off = nullptr;    // device, nsteps*kNumBins+1 entries (step-major)
    // persistent phase: at most max_it sweeps, convergence tested on the device
    int32_t max_it = 1, single_sweep = 0;
    double tau = 0;
    void *dq_arr = nullptr;                 // max_it x G gain sums, zeroed (det: two words each)
    unsigned long long *moved_arr = nullptr;  // max_it move counts, zeroed
    int32_t *iters_out = nullptr;           // sweeps executed
    void *dq_acc = nullptr;       // sweep delta-modularity numerator (det: two words, lo and hi)
    unsigned long long *moved = nullptr;  // refinement: accepted moves
    int32_t *hub_keys = nullptr;  // global tables for bin 6 (one region per block)
    void *hub_vals = nullptr;
    int hub_bits = 0, hub_regions = 0;
    // persistent sweep: bin 6 evaluated by the whole grid (launch_hub_prep
    // fills hubs; hub_keys/hub_vals then hold one step's tables); per hub:
    // hd, hcand, hmv, hkey, hkvd (8 bytes); per eligible hub of a step: hj,
    // htoff, heoff (+1); hinfo: 3 words
    bool grid_hubs = false;
    int32_t *act = nullptr;  // persistent sweep: per-step marks (1024 entries; null: no step skipped)
    bool rand_refine = false;  // randomized refinement (asynchronous mode)
    uint64_t rseed = 0;        // its draws: seed + 0xD1B54A32D192ED03 * 64 * pass
    int32_t sweep = 0;         // sweep index of a per-step launch
    const int32_t *hubs = nullptr;
    int32_t *hj = nullptr;
    int64_t *htoff = nullptr, *heoff = nullptr, *hinfo = nullptr;
    int32_t *hd = nullptr, *hcand = nullptr, *hmv = nullptr;
    unsigned long long *hkey = nullptr;
    void *hkvd = nullptr;
    unsigned *bar = nullptr;      // grid barrier state (2 words, zeroed before every launch)
    int *err = nullptr;
    unsigned long long *prof = nullptr;  // 8 work counters of this launch's class, or null
    int32_t block_max = kBlockMaxDeg;    // rows longer than this are bin 6 (the hubs)
    // testing aid for the timeout path: block stall_block (-1: none) of a
    // persistent launch ends without arriving at the barrier; the others
    // poll at most spin_limit times
    int32_t stall_block = -1;
    unsigned long long spin_limit = 1ULL << 24;
    // A batch of G independent graphs swept as one (a disjoint union): every
    // vertex uses its own graph's 2m, and every graph converges on its own.
    // gid == null means one graph (index 0) and the scalars above.
    const int32_t *gid = nullptr;  // graph of every vertex (sweep space)
    const void *gks = nullptr;     // per-graph key scale (acc type): 2m (det) or 1/2m (async)
    const double *g2m = nullptr;   // per-graph 2m, for the convergence test
    int32_t *gdone = nullptr;      // per-graph "phase converged" flags (1 = skip its vertices)
    int32_t *giters = nullptr;     // per-graph sweeps executed in the phase
    const double *gtau = nullptr;  // per-graph tolerance (graphs at different passes), or tau for all
    unsigned *gactive = nullptr;   // per sweep: graphs still running after it (max_it, zeroed)
    int32_t G = 1;                 // dq_arr and moved_arr hold max_it x G sums
};

// Work counters (kernels add to them when profiling): sweep kernels
// {evaluated, skipped, edges, distinct, moved, moved_edges}; aggregation
// {communities, members, edges, written}.
constexpr int kProfCounters = 8;

// evaluate one (step, bin) vertex list
cudaError_t launch_sweep_eval(const SweepCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                              cudaStream_t s);
// deterministic local-moving: apply a step's proposals (list covers all bins)
cudaError_t launch_move_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s);
// refinement: accept (rule S5) and apply a step's proposals
cudaError_t launch_refine_apply(const SweepCtx &c, const int32_t *list, int64_t count, cudaStream_t s);
// one whole phase (sweeps of every step, grid barriers between steps, the
// convergence test on the device) in one cooperative launch
cudaError_t launch_sweep_coop(const SweepCtx &c, const int32_t *list, int grid, cudaStream_t s);
int sweep_coop_blocks_per_sm(bool det, bool w_int, bool refine);

// Aggregation (Algorithm 4) of G' by dense labels Cd into the holey CSR G''.
struct AggCtx {
    GraphView g;
    bool det = false;
    const int32_t *Cd = nullptr;      // renumbered refined membership, [0, ncomm)
    const int64_t *coff = nullptr;    // community-vertex CSR offsets
    const int32_t *members = nullptr;
    const int64_t *out_off = nullptr; // offsets of G'' (scan of community total degree)
    int32_t *out_deg = nullptr;
    int32_t *out_idx = nullptr;
    void *out_w = nullptr;            // float (async) or WInt (det)
    void *out_K = nullptr;            // K'' (acc type): row sums of G''
    int64_t ncomm = 0;
    // bin 6 (communities of more than kBlockMaxDeg member entries): one
    // global table per community, packed: table k (community list[k]) owns
    // slots [tab_off[k], tab_off[k+1]) (a power of two); tab_idx[c] = k or -1.
    // A launch takes tables [tab_k0, tab_k1), whose slots start at tab_base
    // within hub_keys/hub_vals.
    int32_t *hub_keys = nullptr;
    void *hub_vals = nullptr;
    const int64_t *tab_off = nullptr;
    const int32_t *tab_idx = nullptr;
    int64_t tab_k0 = 0, tab_k1 = 0, tab_base = 0;
    // the members of the bin-6 communities as one flat list in table order:
    // member t of table k is at moff[k] + t, its vertex fm[t], its table
    // ft[t]; eoff: the scan of their degrees (the flat entry range)
    const int32_t *fm = nullptr, *ft = nullptr;
    const int64_t *moff = nullptr, *eoff = nullptr;
    int *err = nullptr;
    unsigned long long *prof = nullptr;
};
// bins 1-5 of the aggregation: one community per tile, warp or block
cudaError_t launch_aggregate(const AggCtx &c, int bin, const int32_t *list, int64_t count, int max_blocks,
                             cudaStream_t s);
// bin 6 sizes: tab_size[k] = 2^max(6, ceil log2(2 min(tdeg, ncomm))) of
// community list[k], tab_idx[list[k]] = k, tab_nm[k] its member count
// (coff: the community-vertex CSR), out_K[list[k]] = 0 (acc type)
cudaError_t launch_table_sizes(const int32_t *list, int64_t count, const int64_t *tdeg, const int64_t *coff,
                               int64_t ncomm, bool det, int64_t *tab_size, int32_t *tab_idx, int64_t *tab_nm,
                               void *out_K, cudaStream_t s);
// the flat member list of the K6 bin-6 tables (moff: the scan of tab_nm, M6
// members): fm[t] = vertex, ft[t] = table, fd[t] = degree
cudaError_t launch_table_members(const int32_t *list, int64_t K6, const int64_t *moff, int64_t M6, const int64_t *coff,
                                 const int32_t *members, const int32_t *deg, int32_t *fm, int32_t *ft, int32_t *fd,
                                 cudaStream_t s);
// bin 6, tables [tab_k0, tab_k1) (cleared by the caller): the flat entry
// range of their members goes into their tables, 32 entries per warp, then
// the whole grid writes the tables' distinct entries as the communities'
// rows, 32 slots per warp
cudaError_t launch_aggregate_tables(const AggCtx &c, const int32_t *list, int sms, cudaStream_t s);

// Rows of a holey CSR (n rows, cap = offsets[n] slots, weights WInt)
// sorted by target in place, each row's unused slots kept after its fill
// (reading R10, the deterministic mode); tmp >= sort_rows_tmp_bytes(cap)
// bytes of device scratch. Synchronises the stream when cap > 2^30 (the row
// offsets are then read on the host to cut the rows into chunks).
size_t sort_rows_tmp_bytes(int64_t cap);
cudaError_t launch_sort_rows(int64_t n, const int64_t *off, const int32_t *deg, int32_t *idx, WInt *w, int64_t cap,
                             void *tmp, cudaStream_t s);

// ---- utilities (k_util.cu)
cudaError_t launch_iota(int32_t *a, int64_t n, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *a, int32_t v, int64_t n, cudaStream_t s);
// rows of the sweeps' list in list order: len[t] = deg[list[t]] (then the
// caller scans len into loff), and the copy of list position t's row and
// vertex weight to lidx/lw[loff[t] ..) and lK[t] (weights WInt or fp32,
// vertex weights int64 (det) or fp32)
cudaError_t launch_list_lens(const int32_t *list, int64_t nl, const int32_t *deg, int32_t *len, cudaStream_t s);
cudaError_t launch_list_rows(const int32_t *list, int64_t nl, const GraphView &g, const void *K, bool det,
                             const int64_t *loff, int32_t *lidx, void *lw, void *lK, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long *a, unsigned long long v, int64_t n, cudaStream_t s);
cudaError_t launch_degrees(const int64_t *off, int32_t *deg, int64_t n, int *err, cudaStream_t s);
// K[i] = sum of row i (acc type), *two_m += sum of K (acc type)
cudaError_t launch_vertex_weights(const GraphView &g, bool det, void *K, void *two_m, cudaStream_t s);
// exclusive scan of n int64 counts into out[0..n] (out[n] = total); tmp >= scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
cudaError_t launch_exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t s);
// stable partition of the items 0..n-1 by key[i] in [0, nkeys) (-1: dropped):
// list holds the items grouped by key, ascending within a key; key_off has
// nkeys+1 entries; tmp >= partition_tmp_bytes(n, nkeys)
size_t partition_tmp_bytes(int64_t n, int32_t nkeys);
cudaError_t launch_partition(const int32_t *key, int64_t n, int32_t nkeys, int64_t *key_off, int32_t *list, void *tmp,
                             cudaStream_t s);
cudaError_t launch_max_i32(const int32_t *a, int64_t n, int32_t *out, cudaStream_t s);
cudaError_t launch_validate(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int *err,
                            cudaStream_t s);

// ---- schedule (k_schedule.cu): step of every vertex (reading S0)
struct SchedWork {
    int32_t *cnt, *layer, *ord, *lord;  // n each
    int32_t *scratch;                   // 11 words; after the launch scratch[9] = layers
                                        // produced, scratch[10] = vertices in bucket steps
    int *err;                    // kErrTimeout if a grid barrier gave up
};
// (gid, vseg: a batch of graphs, priorities drawn at indices inside each
// graph; gpass: graphs at different passes, state + gpass[g] for graph g)
// long_rows: some row may exceed kLongRow entries
// gL: the layer cap of every graph of a batch (L is then the largest; a
// graph's buckets follow step L-1, so its order of steps is its own)
cudaError_t launch_schedule(const GraphView &g, uint64_t state, int32_t L, int32_t B, const SchedWork &w,
                            int32_t *step, cudaStream_t s, const int32_t *gid = nullptr,
                            const int64_t *vseg = nullptr, const int32_t *gpass = nullptr, bool long_rows = true,
                            const int32_t *gL = nullptr);
// layer cap of a graph of n vertices and nnz entries whose largest degree
// is maxdeg, when schedule_layers is 0 (reading S0): 1000 for a heavy-tailed
// graph, whose largest degree exceeds 64 times its mean degree nnz / n,
// else 32
constexpr int32_t kLayersHeavy = 1000, kLayersLight = 32;
inline int32_t auto_layers(int64_t maxdeg, int64_t n, int64_t nnz) {
    return (__int128)maxdeg * n > (__int128)64 * nnz ? kLayersHeavy : kLayersLight;
}
// key[i] = step*kNumBins + bin (step-major: one list per step and bin), or
// bin*nsteps + step (bin-major: one step-ordered list per bin); vertices
// without edges get key nsteps*kNumBins (a trailing bucket)
// Hubs of a pass for the whole-grid bin 6 of the persistent sweep: the
// bin-6 lists of the steps (key_off step-major, nsteps steps) compacted in
// list order into hubs[]; *max_span (device) = the largest sum of one
// step's table sizes (2^max(6, ceil log2 2 deg) slots each).
cudaError_t launch_hub_prep(const int64_t *key_off, int32_t nsteps, const int32_t *list, const int32_t *deg,
                            int32_t *hubs, unsigned long long *max_span, cudaStream_t s);
cudaError_t launch_step_bin_keys(const int32_t *step, const int32_t *deg, int64_t n, int32_t nsteps, bool bin_major,
                                 const BinBounds &bb, int32_t *key, cudaStream_t s);

// ---- batches of graphs (k_batch.cu). vseg has G+1 vertex offsets (graph g
// owns vertices [vseg[g], vseg[g+1])); gid maps a vertex to its graph.
enum : int32_t { kGraphActive = 0, kGraphFinishing = 1, kGraphFinished = 2 };
// gid[v] = the g with vseg[g] <= v < vseg[g+1] (binary search)
cudaError_t launch_graph_ids(const int64_t *vseg, int32_t G, int64_t n, int32_t *gid, cudaStream_t s);
// local row indices to global ids: idx[e] += vseg[gid[v]] for the edges of v
// (m entries in all); *err = 1 if a local index is outside [0, n_g) or a row
// lies outside [0, m)
cudaError_t launch_globalize_indices(const int64_t *vseg, const int32_t *gid, int64_t n, const int64_t *off,
                                     int64_t m, int32_t *idx, int *err, cudaStream_t s);
// out[gid[i]] += x[i] (acc type of K: float -> double sums, int64 -> int64)
cudaError_t launch_graph_sums(const void *K, bool det, const int32_t *gid, int64_t n, void *out, cudaStream_t s);
// out[gid[v]] = max(out[gid[v]], deg[v]) (out cleared by the caller)
cudaError_t launch_graph_max_deg(const int32_t *deg, const int32_t *gid, int64_t n, int32_t *out, cudaStream_t s);
// per-graph key scale and 2m from the per-graph sums of K
cudaError_t launch_graph_scales(const void *sums, bool det, int32_t G, void *gks, double *g2m, cudaStream_t s);
// phase start: gdone[g] = (state[g] != active); giters[g] = 0
cudaError_t launch_phase_init(const int32_t *state, int32_t G, int32_t *gdone, int32_t *giters, cudaStream_t s);
// stop tests of Algorithm 1 per graph (readings R4, R5', R12): from the scans
// pos (refined labels) and pos2 (bound labels), li and the aggregation
// tolerance; active graphs that stop become finishing; keep[g] = refined
// communities of the graphs that go on (0 otherwise); passes[g]++ for active
// graphs. With gpass (graphs at different passes) a graph also stops when
// gpass[g] + 1 reaches max_passes. fresh[g] = 1 when the graph's pass began
// with every super-vertex in its own community (R5' stops only such a
// pass); it is set for the next pass of the graphs that go on.
// (deg, gid, n: the current graph; reading R4 leaves each graph's vertices
// without edges out of its ratio, counted into gz, G entries of scratch)
cudaError_t launch_graph_stop(const int64_t *vseg, const int64_t *pos, const int64_t *pos2, const int32_t *li,
                              const double *g2m, double agg_tol, int32_t G, int32_t *state, int64_t *keep,
                              int32_t *passes, cudaStream_t s, const int32_t *gpass, int32_t max_passes,
                              const int32_t *deg, const int32_t *gid, int64_t n, unsigned long long *gz,
                              int32_t *fresh, bool refine_labels);
// C' at the start of local-moving: the first n_cont vertices continue with
// their move-based labels, the others start as singletons
cudaError_t launch_init_labels(const int32_t *label, int64_t n_cont, int64_t n, int32_t *Cp, cudaStream_t s);
// append graph g (n rows of a CSR with local indices and fp32 weights) to the
// holey CSR of a union at row v0 and entry e0: out_off/out_deg/out_idx (ids
// + v0)/out_w (fp32, or WInt when w_int), gid[v0+i] = g, and the
// dendrogram of its vertices C0[a0+i] = v0+i
cudaError_t launch_append_graph(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int64_t v0,
                                int64_t e0, bool w_int, int32_t g, int64_t *out_off, int32_t *out_deg,
                                int32_t *out_idx, void *out_w, int32_t *gid, int32_t *C0, int64_t a0,
                                cudaStream_t s);
// dense ids of the next graph: Cd[i] = vseg2[g] + pos[C[i]] - pos[vseg[g]]
// for graphs that go on, -1 for graphs that stop
cudaError_t launch_renumber_batch(const int32_t *C, const int64_t *pos, const int32_t *gid, const int64_t *vseg,
                                  const int64_t *vseg2, const int32_t *state, int32_t *Cd, int64_t n, cudaStream_t s);
// dendrogram: active graphs C0[v] = Cd[C0[v]]; finishing graphs end on their
// refined label, stored as vseg0[g] + (Cp[C0[v]] - vseg[g]) (an id in the
// input graph's range of g)
cudaError_t launch_lookup_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                                const int32_t *state, const int32_t *Cd, const int32_t *Cp, int64_t n0,
                                cudaStream_t s);
// graphs still active when the pass loop ends: C0[v] = vseg0[g] + (C0[v] - vseg[g])
cudaError_t launch_finalize_batch(int32_t *C0, const int32_t *gid0, const int64_t *vseg0, const int64_t *vseg,
                                  const int32_t *state, int64_t n0, cudaStream_t s);
// finishing -> finished
cudaError_t launch_commit_states(int32_t *state, int32_t G, cudaStream_t s);
// dst[v] = src[v] - off (a graph's dendrogram ids into its own range)
cudaError_t launch_shift_labels(const int32_t *src, int64_t n, int64_t off, int32_t *dst, cudaStream_t s);
// out[g] = pos[vseg[g+1]] - pos[vseg[g]]
cudaError_t launch_graph_counts(const int64_t *pos, const int64_t *vseg, int32_t G, int64_t *out, cudaStream_t s);
// graph of every super-vertex: gid2[Cd[i]] = gid[i] (Cd >= 0)
cudaError_t launch_next_gid(const int32_t *Cd, const int32_t *gid, int64_t n, int32_t *gid2, cudaStream_t s);
// canonical labels inside each graph: out[v] = rank[minv[C0[v]]] - rank[vseg0[gid0[v]]]
cudaError_t launch_canonical_batch(const int32_t *C0, const int32_t *minv, const int64_t *rank, const int32_t *gid0,
                                   const int64_t *vseg0, int64_t n0, int32_t *out, cudaStream_t s);
// Eq. 1 per graph on the input batch with labels local to each graph:
// gsum[3g+0] += intra weight, gsum[3g+1] += 2m, sigtot[vseg0[g] + label] += K_i,
// then gsum[3g+2] += sum of squares over the graph's range; *bad counts labels
// outside [0, n_g); q[g] from the sums
cudaError_t launch_modularity_batch(int64_t n0, const int64_t *off, const int32_t *idx, const float *w,
                                    const int32_t *C, const int32_t *gid0, const int64_t *vseg0, int32_t G,
                                    double gamma, double *sigtot, double *gsum, double *bad, double *q,
                                    cudaStream_t s, bool long_rows = true);

// ---- disconnected communities (k_check.cu, Algorithm 5): components of the
// intra-community subgraph by hooking and pointer jumping
// *bad = 1 if a label lies outside [0, n)
cudaError_t launch_cc_labels(int64_t n, const int32_t *C, int *bad, cudaStream_t s);
cudaError_t launch_cc_init(int64_t n, int32_t *parent, int32_t *roots, cudaStream_t s);
// one hooking pass and one jump; *changed = 1 if anything was hooked
cudaError_t launch_cc_pass(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *C, int32_t *parent,
                           int *changed, cudaStream_t s);
// *count += communities with more than one component (labels C in [0, n))
cudaError_t launch_cc_count(int64_t n, const int32_t *C, const int32_t *parent, int32_t *roots,
                            unsigned long long *count, cudaStream_t s);

// ---- pass bookkeeping (k_pass.cu)
// Sigma[c] += K[i], size[c] += 1 over C (acc type)
cudaError_t launch_community_totals(const int32_t *C, const void *K, bool det, int64_t n, void *Sig, int32_t *size,
                                    cudaStream_t s);
// flag[c] = (size[c] > 0)
cudaError_t launch_nonempty_flags(const int32_t *size, int64_t n, int32_t *flag, cudaStream_t s);
// flag[CB[i]] = 1
cudaError_t launch_mark_labels(const int32_t *lab, int64_t n, int32_t *flag, cudaStream_t s);
// out[i] = map[in[i]] (in-place allowed when out == in)
cudaError_t launch_gather_map(const int32_t *map_pos, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
// dense id of community c = (int32)pos[c] where pos is the exclusive scan of flags
cudaError_t launch_renumber(const int32_t *C, const int64_t *pos, int32_t *Cd, int64_t n, cudaStream_t s);
// C0[v] = map[C0[v]] for the dendrogram
cudaError_t launch_lookup(int32_t *C0, const int32_t *map, int64_t n0, cudaStream_t s);
// community-vertex CSR: cnt[Cd[i]]++, tdeg[Cd[i]] += deg[i] (Cd < 0: skipped)
cudaError_t launch_comm_counts(const int32_t *Cd, const int32_t *deg, int64_t n, int64_t *cnt, int64_t *tdeg,
                               cudaStream_t s);
cudaError_t launch_comm_fill(const int32_t *Cd, int64_t n, const int64_t *coff, int32_t *cursor, int32_t *members,
                             cudaStream_t s);
// bins of communities by total degree
cudaError_t launch_comm_bin_keys(const int64_t *tdeg, int64_t ncomm, const BinBounds &bb, int32_t *key,
                                 cudaStream_t s);
// move-based labels: bnd[Cd[i]] = CB[i]; rep[b] = min s; label[s] = rep[bnd[s]] (Cd < 0: skipped)
cudaError_t launch_bound_labels(const int32_t *Cd, const int32_t *CB, int64_t n, int64_t ncomm, int32_t *bnd,
                                int32_t *rep, int32_t *label, cudaStream_t s);
// canonical labels: rank of the smallest vertex of each community
cudaError_t launch_min_vertex(const int32_t *C0, int64_t n0, int32_t *minv, cudaStream_t s);
cudaError_t launch_first_flags(const int32_t *C0, const int32_t *minv, int64_t n0, int32_t *first, cudaStream_t s);
cudaError_t launch_canonical(const int32_t *C0, const int32_t *minv, const int64_t *rank, int64_t n0, int32_t *out,
                             cudaStream_t s);
// modularity (Eq. 1) of labels C (in [0,n)) on a plain CSR: sums[0] += intra
// weight, sums[1] += 2m, sigtot[c] += K_i, sums[3] += labels out of range;
// then sums[2] += sum_c sigtot[c]^2
cudaError_t launch_modularity_parts(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                                    const int32_t *C, double *sigtot, double *sums, cudaStream_t s,
                                    bool long_rows = true);
cudaError_t launch_sum_squares(const double *x, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_max_i64(const int64_t *a, int64_t n, unsigned long long *out, cudaStream_t s);
// nonint = 1 if some weight is not an integer; sum += sum of weights (fp64)
cudaError_t launch_weight_props(const float *w, int64_t m, int *nonint, double *sum, cudaStream_t s);

}  // namespace lgb
