/*
 * Leiden oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential, single-threaded CPU restatement of the parallel Leiden
 * method of "GVE-Leiden: Fast Leiden Algorithm for Community Detection in
 * Shared Memory Setting" (arXiv 2312.13936): the main loop (Algorithm 1), the
 * local-moving phase (Algorithm 2), the refinement phase (Algorithm 3), the
 * aggregation phase (Algorithm 4), modularity (Eq. 1) and delta-modularity
 * (Eq. 2), plus the disconnected-community check (Algorithm 5, appendix).
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline may load this file's library. It shares no code, header, table or
 * helper with the CUDA implementation, and nothing in the product calls it.
 *
 * Two modes:
 *   OG_SEQ  -- vertices are visited in id order and every move is applied at
 *              once (the sequential reading of Algorithms 2 and 3); float
 *              arithmetic in fp64. The quality reference for the GPU's
 *              asynchronous mode.
 *   OG_SYNC -- layered synchronous sweeps (S0-S5 below): the vertices are
 *              visited step by step in a hashed priority order; inside a
 *              step every vertex is evaluated against the state at the start
 *              of the step, then all accepted moves are applied. Integer
 *              weights, exact int64 move decisions. The bit-exact reference
 *              for the GPU's deterministic mode.
 *
 * Readings of points the paper leaves open, numbered R1-R14, S0-S5 and V1-V3:
 *   R1  MAX_PASSES is not given; it is a parameter (default 10).
 *   R2  Candidates are the communities in the scan table other than the
 *       vertex's own; the best one is taken (ties: lowest community id) and
 *       the vertex moves only if its delta-modularity is strictly positive.
 *   R3  Pass 0 starts from singletons; pass p > 0 starts each super-vertex in
 *       its move-based community (Algorithm 1, "Map C' to C'_B"), labelled by
 *       the smallest super-vertex id of that community; Sigma' is the sum of
 *       K' over each label.
 *   R4  |Gamma| is the number of non-empty refined communities and
 *       |Gamma_old| the vertex count of the current graph, both without the
 *       z vertices that have no edges (each is its own community in every
 *       pass and can take part in no aggregation, Section 4.1's purpose of
 *       the tolerance): stop if (|Gamma| - z) / (|Gamma_old| - z) exceeds
 *       the aggregation tolerance.
 *   R5  l_i is the number of local-moving sweeps executed and l_j the
 *       number of refinement sweeps; see R5' for the stop test.
 *   R6  Refinement repeats sweeps over the still-isolated vertices until a
 *       sweep moves nobody or MAX_ITERATIONS sweeps ran (flag
 *       OG_REFINE_SINGLE_SWEEP gives the literal single sweep).
 *   R7  A vertex is isolated when its community has exactly one member (the
 *       exact form of the Sigma' == K' test of Algorithm 3).
 *   R8  The output composes the dendrogram through the refined partition of
 *       the last pass executed.
 *   R9  Renumbering keeps ascending order of the old ids.
 *   R10 Rows of the aggregated graph are written in ascending target order.
 *   R11 A self-loop is one CSR entry, counted once in K_i and in 2m; the
 *       aggregated self-loop of a community carries the sum of all CSR entries
 *       inside it (scanCommunities with self = true).
 *   R12 If m = 0 the result is the singleton partition and Q = 0.
 *   R13 The resolution gamma multiplies the null-model term of Eq. 1 and the
 *       second term of Eq. 2 (gamma = 1 is the paper's modularity).
 *   R14 The tolerance test compares the sum of the delta-modularity of the
 *       moves made in a sweep with tau; tau is divided by TOLERANCE_DROP
 *       after every aggregated pass.
 *   SYNC-only:
 *   S0  Sweep order: priority steps. h(v) is output number v+1 of
 *       SplitMix64 (Steele, Lea & Flood 2014) from state seed + pass, and
 *       prio(v) = deg(v) * 2^32 + (h(v) >> 32): the row length first, so
 *       vertices of higher degree go first (an importance ordering, one of
 *       the Louvain optimisations the paper carries over, Section 3), the
 *       hash breaking ties at random; u precedes v when prio(u) > prio(v),
 *       ties by smaller id. layer(v) =
 *       1 + max layer of v's preceding neighbours (0 if none) -- the rounds
 *       of Jones & Plassmann's parallel colouring. A vertex with
 *       layer(v) < L-1 takes step layer(v); every other vertex takes step
 *       L-1 + ((h(v) >> 32) mod B) (B = schedule_buckets). L is
 *       schedule_layers, or, when that is 0 (the default), 1000 for a
 *       heavy-tailed input -- one whose largest degree exceeds 64 times its
 *       mean degree nnz/n (edgeless vertices counted) -- and 32 otherwise:
 *       on heavy-tailed graphs the hubs must be handled one layer after
 *       another (vertices past the cap share bucket steps with their
 *       neighbours, and on R-MAT graphs the refinement of the last pass then
 *       splits large communities), elsewhere a short schedule is as good and
 *       cheaper. (Lattices, block models and G(n, p) graphs have ratios
 *       below 4; R-MAT graphs from scale 13 up have ratios above 90.) Steps
 *       are processed in increasing order. A step
 *       below L-1 holds no two adjacent vertices, so on those edges the two
 *       ends are handled in priority order as in a sequential sweep. Inside a
 *       step every vertex is evaluated against the state at the start of the
 *       step, then all accepted moves are applied.
 *   S1  Move decisions use key(c) = 2m*K_{i->c} - K_i*Sigma_c (Eq. 2 times
 *       2m^2 up to a term common to all c); the vertex moves iff
 *       key(c*) > 2m*K_{i->d} - K_i*(Sigma_d - K_i). Weights, K, Sigma and
 *       2m are int64, keys and their differences 128-bit integers (every
 *       product is below (2m)^2). Requires integer weights, gamma = 1 and
 *       2m < 2^53 (the weight sum is then exact in fp64 and every key
 *       difference, and a sweep's sum of them, fits in 128 bits).
 *   S2  In steps >= L-1 only (where neighbours can move together), a
 *       vertex alone in its community does not move into another
 *       single-vertex community with a larger id (no endless label swaps).
 *   S3  Pruning as in Algorithm 2: a vertex is marked processed when it is
 *       evaluated; the CSR neighbours (self-loop included) of a vertex that
 *       moved are marked unprocessed when its layer's moves are applied.
 *   S4  Sweep delta-modularity = 2*num / (2m)^2 in fp64, num the sweep's
 *       sum of key gains (an unsigned 128-bit integer, every gain being
 *       positive) converted as (double)(num >> 64) * 2^64 + (double)(num
 *       mod 2^64), each conversion and the sum rounded to nearest.
 *   S5  Refinement accepts a proposal i -> t unless t is a single-vertex
 *       community whose vertex proposes in the same step; of two vertices
 *       proposing to each other, the one with the larger id moves. Below
 *       step L-1 this never rejects (a proposer's target vertex is a
 *       neighbour, hence in another step); in later steps it keeps every
 *       accepted vertex joined to a community that keeps the neighbour it
 *       saw.
 *   Variants (flags, both modes):
 *   V1  OG_REFINE_LABELS: refine-based super-vertex labels (Section 4.1):
 *       every super-vertex starts a pass in its own community instead of
 *       the move-based one of R3.
 *   V2  OG_LOUVAIN: the Louvain method the paper compares with (Section 5):
 *       no refinement; the refined partition of a pass is its local-moving
 *       partition (so l_j = 0 and R5' reduces to l_i <= 1), and aggregation
 *       merges the local-moving communities. Communities need not be
 *       connected.
 *   V3  OG_RANDOM_REFINE (SEQ mode only): the randomized refinement of the
 *       original Leiden method (Sections 3.4 and 4.1): an isolated vertex
 *       joins one of the communities of positive gain within its bound with
 *       probability proportional to the gain, instead of the best one. The
 *       draw: the candidates in ascending community id, u = ((x >> 11) +
 *       0.5) / 2^53 with x = SplitMix64 output number i+1 from state
 *       seed + 0xD1B54A32D192ED03 * (64 pass + sweep + 1), the first
 *       candidate whose running gain sum exceeds u times the total.
 *   Both modes:
 *   R5' The passes stop (global convergence) when the local-moving phase
 *       converged in its first sweep (l_i <= 1), the refinement split no
 *       local-moving community (as many refined communities as local-moving
 *       ones), and the pass began with every super-vertex in its own
 *       community (pass 0; a pass after one whose refinement split nothing;
 *       every pass under V1): another pass could then change nothing. A pass
 *       that began from move-based labels (R3) grouping several
 *       super-vertices cannot merge two communities by moving single
 *       super-vertices, but the next pass, whose super-vertices are those
 *       communities, can.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 og_i128;            /* S1 keys (a GCC extension on 64-bit targets) */
typedef unsigned __int128 og_u128;   /* S4 sweep sums */

/* S4: a sweep's gain sum as a double, in a fixed order of roundings */
static double u128_to_double(og_u128 x) {
    return (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x;
}

enum { OG_OK = 0, OG_ERR_INVALID = -1, OG_ERR_OOM = -3, OG_ERR_UNSUPPORTED = -6, OG_ERR_OVERFLOW = -7 };
enum { OG_SEQ = 0, OG_SYNC = 1 };
enum { OG_REFINE_SINGLE_SWEEP = 1, OG_NO_PRUNE = 2, OG_REFINE_LABELS = 4, OG_LOUVAIN = 8, OG_RANDOM_REFINE = 16 };

/* what-codes passed to the trace callback */
enum {
    OG_T_INIT_LABELS = 1,  /* int32[n']: C' at the start of local-moving      */
    OG_T_MOVE = 2,         /* int32[n']: C' after local-moving (= C'_B)       */
    OG_T_REFINE = 3,       /* int32[n']: C' after refinement                  */
    OG_T_COUNTS = 4,       /* int64[4]: n', l_i, l_j, |Gamma|                 */
    OG_T_RENUMBER = 5,     /* int32[n']: renumbered refined C'                */
    OG_T_AGG_OFF = 6,      /* int64[|Gamma|+1]: holey CSR offsets             */
    OG_T_AGG_DEG = 7,      /* int32[|Gamma|]: holey CSR row fill              */
    OG_T_AGG_IDX = 8,      /* int32[cap]: holey CSR targets (gaps are -1)     */
    OG_T_AGG_W = 9,        /* double[cap]: holey CSR weights (gaps are 0)     */
    OG_T_DENDRO = 10       /* int32[n0]: C after the dendrogram lookup        */
};

typedef struct {
    double resolution;            /* gamma (R13), default 1 */
    double tolerance;             /* tau_0, default 0.01 */
    double aggregation_tolerance; /* tau_agg, default 0.8 */
    double tolerance_drop;        /* TOLERANCE_DROP, default 10 */
    int32_t max_iterations;       /* MAX_ITERATIONS, default 20 */
    int32_t max_passes;           /* MAX_PASSES (R1), default 10 */
    int32_t mode;                 /* OG_SEQ or OG_SYNC */
    int32_t flags;                /* OG_REFINE_SINGLE_SWEEP, OG_NO_PRUNE (SEQ, tests only),
                                     OG_REFINE_LABELS, OG_LOUVAIN (V1, V2),
                                     OG_RANDOM_REFINE (V3, SEQ only) */
    int32_t schedule_layers;      /* SYNC: L, priority layers (S0); 0 (default): by the graph, S0 */
    int32_t schedule_buckets;     /* SYNC: B, buckets after the last layer (S0), default 16 */
    uint64_t seed;                /* SYNC: priority seed (S0), default 0 */
} og_params;

typedef void (*og_trace_fn)(void *ctx, int32_t pass, int32_t what, const void *data, int64_t count);

/* A (possibly holey) weighted CSR: row i holds entries [off[i], off[i]+deg[i]).
 * This is the "Weighted Holey CSR with degree" of the paper's Fig. 5. */
typedef struct {
    int64_t n;
    int64_t *off;
    int32_t *deg;
    int32_t *idx;
    double *w;
} og_graph;

static void graph_free(og_graph *g) {
    free(g->off); free(g->deg); free(g->idx); free(g->w);
    memset(g, 0, sizeof(*g));
}

/* -------------------------------------------------------------------------
 * Scan table: the collision-free table H of Algorithms 2-4 (a dense value
 * array indexed by community id plus the list of keys present).
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t cap;
    double *val;      /* fp64 values (SEQ) */
    int64_t *ival;    /* exact int64 values (SYNC) */
    uint8_t *has;
    int32_t *keys;
    int64_t nkeys;
} og_table;

static int table_init(og_table *t, int64_t cap) {
    t->cap = cap;
    t->val = (double *)calloc((size_t)(cap ? cap : 1), sizeof(double));
    t->ival = (int64_t *)calloc((size_t)(cap ? cap : 1), sizeof(int64_t));
    t->has = (uint8_t *)calloc((size_t)(cap ? cap : 1), 1);
    t->keys = (int32_t *)malloc((size_t)(cap ? cap : 1) * sizeof(int32_t));
    t->nkeys = 0;
    return (t->val && t->ival && t->has && t->keys) ? 0 : -1;
}
static void table_free(og_table *t) { free(t->val); free(t->ival); free(t->has); free(t->keys); }
static void table_clear(og_table *t) {
    for (int64_t k = 0; k < t->nkeys; ++k) {
        int32_t c = t->keys[k];
        t->has[c] = 0; t->val[c] = 0.0; t->ival[c] = 0;
    }
    t->nkeys = 0;
}
static void table_add(og_table *t, int32_t c, double w) {
    if (!t->has[c]) { t->has[c] = 1; t->keys[t->nkeys++] = c; }
    t->val[c] += w;
    t->ival[c] += (int64_t)w;
}

/* scanCommunities (Algorithm 2): H[C[j]] += w over the edges (j, w) of i,
 * skipping j == i unless self. */
static void scan_communities(og_table *t, const og_graph *g, const int32_t *C, int64_t i, int self) {
    for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) {
        int32_t j = g->idx[e];
        if (!self && j == i) continue;
        table_add(t, C[j], g->w[e]);
    }
}

/* scanBounded (Algorithm 3): as scanCommunities, but only neighbours j with
 * the same community bound as i (C_B[i] == C_B[j]). */
static void scan_bounded(og_table *t, const og_graph *g, const int32_t *CB, const int32_t *C, int64_t i,
                         int self) {
    for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) {
        int32_t j = g->idx[e];
        if (!self && j == i) continue;
        if (CB[i] != CB[j]) continue;
        table_add(t, C[j], g->w[e]);
    }
}

/* Eq. 2 with resolution (R13): delta-modularity of moving i from d to c.
 *   dQ = (K_{i->c} - K_{i->d}) / m - gamma * K_i (K_i + Sigma_c - Sigma_d) / (2 m^2) */
static double delta_q(double Kic, double Kid, double Ki, double Sc, double Sd, double m, double gamma) {
    return (Kic - Kid) / m - gamma * Ki * (Ki + Sc - Sd) / (2.0 * m * m);
}

/* vertexWeights (Algorithm 1): K_i = sum of the weights of i's CSR entries. */
static void vertex_weights(const og_graph *g, double *K) {
    for (int64_t i = 0; i < g->n; ++i) {
        double s = 0.0;
        for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) s += g->w[e];
        K[i] = s;
    }
}

/* ------------------------------------------------------------------------
 * SEQ mode
 * --------------------------------------------------------------------- */

/* leidenMove (Algorithm 2), sequential: returns l_i, the sweeps executed. */
static int move_seq(const og_graph *g, int32_t *C, const double *K, double *Sig, double tau, double gamma,
                    double two_m, int32_t max_it, int no_prune, og_table *H) {
    int64_t n = g->n;
    double m = two_m / 2.0;
    uint8_t *unprocessed = (uint8_t *)malloc((size_t)(n ? n : 1));
    if (!unprocessed) return -1;
    memset(unprocessed, 1, (size_t)n); /* mark all vertices unprocessed */
    int sweeps = 0;
    for (int32_t it = 0; it < max_it; ++it) {
        sweeps++;
        double dQ = 0.0;
        if (no_prune) memset(unprocessed, 1, (size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            if (!unprocessed[i]) continue;
            unprocessed[i] = 0; /* prune */
            table_clear(H);
            scan_communities(H, g, C, i, 0);
            int32_t d = C[i];
            double Kid = H->has[d] ? H->val[d] : 0.0;
            int32_t best = -1;
            double best_dq = 0.0;
            for (int64_t k = 0; k < H->nkeys; ++k) {
                int32_t c = H->keys[k];
                if (c == d) continue;
                double q = delta_q(H->val[c], Kid, K[i], Sig[c], Sig[d], m, gamma);
                if (best < 0 || q > best_dq || (q == best_dq && c < best)) { best = c; best_dq = q; }
            }
            if (best < 0 || !(best_dq > 0.0)) continue;
            Sig[d] -= K[i];
            Sig[best] += K[i];
            C[i] = best;
            dQ += best_dq;
            for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) unprocessed[g->idx[e]] = 1;
        }
        if (dQ <= tau) break; /* locally converged */
    }
    free(unprocessed);
    return sweeps;
}

/* leidenRefine (Algorithm 3), sequential, with R6/R7: returns l_j. */
uint64_t og_splitmix64_at(uint64_t s, uint64_t i);
static int cmp_cand(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* rnd: NULL for the greedy refinement (Algorithm 3); else the state of V3's
 * draws for this pass (seed + 0xD1B54A32D192ED03 * (64 pass + sweep + 1) is
 * formed per sweep) and a scratch array of n candidate ids. */
static int refine_seq(const og_graph *g, const int32_t *CB, int32_t *C, const double *K, double *Sig,
                      int32_t *size, double gamma, double two_m, int32_t max_it, int single_sweep,
                      og_table *H, const uint64_t *rnd, int32_t *cand) {
    int64_t n = g->n;
    double m = two_m / 2.0;
    int sweeps = 0;
    for (int32_t it = 0; it < max_it; ++it) {
        sweeps++;
        int64_t moved = 0;
        for (int64_t i = 0; i < n; ++i) {
            int32_t c = C[i];
            if (size[c] != 1) continue; /* only isolated vertices move */
            table_clear(H);
            scan_bounded(H, g, CB, C, i, 0);
            double Kic_own = H->has[c] ? H->val[c] : 0.0;
            int32_t best = -1;
            double best_dq = 0.0;
            if (rnd) { /* V3: a candidate of positive gain, with probability proportional to it */
                int64_t nc = 0;
                for (int64_t k = 0; k < H->nkeys; ++k)
                    if (H->keys[k] != c) cand[nc++] = H->keys[k];
                qsort(cand, (size_t)nc, sizeof(int32_t), cmp_cand);
                double total = 0.0;
                for (int64_t k = 0; k < nc; ++k) {
                    double q = delta_q(H->val[cand[k]], Kic_own, K[i], Sig[cand[k]], Sig[c], m, gamma);
                    if (q > 0.0) total += q;
                }
                if (!(total > 0.0)) continue;
                uint64_t x = og_splitmix64_at(*rnd + 0xD1B54A32D192ED03ULL * (uint64_t)(it + 1), (uint64_t)i);
                double u = ((double)(x >> 11) + 0.5) / 9007199254740992.0;
                double t = u * total, run = 0.0;
                for (int64_t k = 0; k < nc; ++k) {
                    double q = delta_q(H->val[cand[k]], Kic_own, K[i], Sig[cand[k]], Sig[c], m, gamma);
                    if (!(q > 0.0)) continue;
                    run += q;
                    best = cand[k];
                    best_dq = q;
                    if (run > t) break;
                }
            } else {
                for (int64_t k = 0; k < H->nkeys; ++k) {
                    int32_t cc = H->keys[k];
                    if (cc == c) continue;
                    double q = delta_q(H->val[cc], Kic_own, K[i], Sig[cc], Sig[c], m, gamma);
                    if (best < 0 || q > best_dq || (q == best_dq && cc < best)) { best = cc; best_dq = q; }
                }
            }
            if (best < 0 || !(best_dq > 0.0)) continue;
            Sig[c] -= K[i];
            Sig[best] += K[i];
            size[c]--;
            size[best]++;
            C[i] = best;
            moved++;
        }
        if (moved == 0 || single_sweep) break;
    }
    return sweeps;
}

/* ------------------------------------------------------------------------
 * SYNC mode (S1-S5)
 * --------------------------------------------------------------------- */

/* S0: SplitMix64 output number i+1 from state s (Steele, Lea & Flood 2014). */
uint64_t og_splitmix64_at(uint64_t s, uint64_t i) {
    uint64_t z = s + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static const uint64_t *g_sort_prio; /* qsort context (single-threaded) */
static int cmp_by_priority(const void *a, const void *b) {
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    if (g_sort_prio[u] != g_sort_prio[v]) return g_sort_prio[u] > g_sort_prio[v] ? -1 : 1;
    return (u > v) - (u < v);
}

/* S0: step of every vertex; returns the number of steps (max step + 1). The
 * layers are computed by visiting the vertices in priority order. */
int32_t og_schedule(int64_t n, const int64_t *off, const int32_t *deg, const int32_t *idx, uint64_t state,
                    int32_t cap, int32_t buckets, int32_t *layer) {
    uint64_t *prio = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    int32_t *order = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint8_t *done = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    if (!prio || !order || !done || cap < 1 || buckets < 1) { free(prio); free(order); free(done); return -1; }
    for (int64_t v = 0; v < n; ++v) {
        prio[v] = ((uint64_t)deg[v] << 32) | (og_splitmix64_at(state, (uint64_t)v) >> 32);
        order[v] = (int32_t)v;
    }
    g_sort_prio = prio;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_by_priority);
    int32_t used = 0;
    for (int64_t k = 0; k < n; ++k) {
        int32_t v = order[k];
        int32_t L = 0;
        for (int64_t e = off[v]; e < off[v] + deg[v]; ++e) {
            int32_t u = idx[e];
            if (u != v && done[u] && layer[u] + 1 > L) L = layer[u] + 1; /* done[u]: u precedes v */
        }
        layer[v] = L < cap - 1 ? L : cap - 1;
        done[v] = 1;
    }
    for (int64_t v = 0; v < n; ++v) {
        if (layer[v] == cap - 1)
            layer[v] = cap - 1 + (int32_t)((og_splitmix64_at(state, (uint64_t)v) >> 32) % (uint64_t)buckets);
        if (layer[v] + 1 > used) used = layer[v] + 1;
    }
    free(prio); free(order); free(done);
    return used;
}

/* vertices grouped by layer: lst[lo[k]..lo[k+1]) holds layer k, ascending id */
static int layer_lists(int64_t n, const int32_t *layer, int32_t nl, int64_t **lo_out, int32_t **lst_out) {
    int64_t *lo = (int64_t *)calloc((size_t)nl + 1, sizeof(int64_t));
    int32_t *lst = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t *cur = (int64_t *)malloc(((size_t)nl + 1) * sizeof(int64_t));
    if (!lo || !lst || !cur) { free(lo); free(lst); free(cur); return -1; }
    for (int64_t v = 0; v < n; ++v) lo[layer[v] + 1]++;
    for (int32_t k = 0; k < nl; ++k) lo[k + 1] += lo[k];
    memcpy(cur, lo, ((size_t)nl + 1) * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) lst[cur[layer[v]]++] = (int32_t)v;
    free(cur);
    *lo_out = lo; *lst_out = lst;
    return 0;
}

/* leidenMove (Algorithm 2), layered synchronous sweeps with exact keys. */
static int move_sync(const og_graph *g, int32_t *C, const int64_t *K, int64_t *Sig, int32_t *size, double tau,
                     int64_t two_m, int32_t max_it, int32_t cap, const int32_t *layer, int32_t nl,
                     og_table *H) {
    int64_t n = g->n;
    uint8_t *unprocessed = (uint8_t *)malloc((size_t)(n ? n : 1));
    int32_t *prop = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    og_i128 *gain = (og_i128 *)malloc((size_t)(n ? n : 1) * sizeof(og_i128));
    int64_t *lo = NULL;
    int32_t *lst = NULL;
    if (!unprocessed || !prop || !gain || layer_lists(n, layer, nl, &lo, &lst)) {
        free(unprocessed); free(prop); free(gain); return -1;
    }
    memset(unprocessed, 1, (size_t)n); /* mark all vertices unprocessed */
    int sweeps = 0;
    for (int32_t it = 0; it < max_it; ++it) {
        sweeps++;
        og_u128 num = 0;
        for (int32_t k = 0; k < nl; ++k) {
            /* evaluate the layer against the state at its start */
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) {
                int32_t i = lst[q];
                prop[i] = -1;
                if (!unprocessed[i]) continue;
                unprocessed[i] = 0; /* prune */
                table_clear(H);
                scan_communities(H, g, C, i, 0);
                int32_t d = C[i];
                int64_t Kid = H->has[d] ? H->ival[d] : 0;
                og_i128 key_d = (og_i128)two_m * Kid - (og_i128)K[i] * (Sig[d] - K[i]);
                int32_t best = -1;
                og_i128 best_key = 0;
                for (int64_t t = 0; t < H->nkeys; ++t) {
                    int32_t c = H->keys[t];
                    if (c == d) continue;
                    og_i128 key = (og_i128)two_m * H->ival[c] - (og_i128)K[i] * Sig[c];
                    if (best < 0 || key > best_key || (key == best_key && c < best)) { best = c; best_key = key; }
                }
                if (best < 0 || best_key <= key_d) continue;
                if (k >= cap - 1 && size[d] == 1 && size[best] == 1 && best > d) continue; /* S2 */
                prop[i] = best;
                gain[i] = best_key - key_d;
            }
            /* apply the layer's moves; mark neighbours of movers unprocessed */
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) {
                int32_t i = lst[q];
                if (prop[i] < 0) continue;
                int32_t d = C[i], c = prop[i];
                Sig[d] -= K[i];
                Sig[c] += K[i];
                size[d]--;
                size[c]++;
                C[i] = c;
                num += (og_u128)gain[i];
                for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) unprocessed[g->idx[e]] = 1;
            }
        }
        double dQ = 2.0 * u128_to_double(num) / ((double)two_m * (double)two_m); /* S4 */
        if (dQ <= tau) break;
    }
    free(unprocessed); free(prop); free(gain); free(lo); free(lst);
    return sweeps;
}

/* leidenRefine (Algorithm 3), layered synchronous sweeps, exact keys, S5. */
static int refine_sync(const og_graph *g, const int32_t *CB, int32_t *C, const int64_t *K, int64_t *Sig,
                       int32_t *size, int64_t two_m, int32_t max_it, int single_sweep, const int32_t *layer,
                       int32_t nl, og_table *H) {
    int64_t n = g->n;
    int32_t *prop = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint8_t *accept = (uint8_t *)malloc((size_t)(n ? n : 1));
    int64_t *lo = NULL;
    int32_t *lst = NULL;
    if (!prop || !accept || layer_lists(n, layer, nl, &lo, &lst)) { free(prop); free(accept); return -1; }
    for (int64_t i = 0; i < n; ++i) prop[i] = -1;
    int sweeps = 0;
    for (int32_t it = 0; it < max_it; ++it) {
        sweeps++;
        int64_t moved = 0;
        for (int32_t k = 0; k < nl; ++k) {
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) {
                int32_t i = lst[q];
                int32_t c = C[i];
                if (size[c] != 1) continue; /* isolated vertices only (R7) */
                table_clear(H);
                scan_bounded(H, g, CB, C, i, 0);
                int64_t Kic_own = H->has[c] ? H->ival[c] : 0;
                og_i128 key_c = (og_i128)two_m * Kic_own - (og_i128)K[i] * (Sig[c] - K[i]);
                int32_t best = -1;
                og_i128 best_key = 0;
                for (int64_t t = 0; t < H->nkeys; ++t) {
                    int32_t cc = H->keys[t];
                    if (cc == c) continue;
                    og_i128 key = (og_i128)two_m * H->ival[cc] - (og_i128)K[i] * Sig[cc];
                    if (best < 0 || key > best_key || (key == best_key && cc < best)) { best = cc; best_key = key; }
                }
                if (best >= 0 && best_key > key_c) prop[i] = best;
            }
            /* S5: an isolated vertex i has C[i] == i, and a non-empty refined
             * community t always contains vertex t */
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) {
                int32_t i = lst[q];
                int32_t t = prop[i];
                accept[i] = 0;
                if (t < 0) continue;
                if (prop[t] < 0 || (prop[t] == i && i > t)) accept[i] = 1;
            }
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) {
                int32_t i = lst[q];
                if (accept[i]) {
                    int32_t c = C[i], t = prop[i];
                    Sig[c] -= K[i];
                    Sig[t] += K[i];
                    size[c]--;
                    size[t]++;
                    C[i] = t;
                    moved++;
                }
            }
            for (int64_t q = lo[k]; q < lo[k + 1]; ++q) prop[lst[q]] = -1;
        }
        if (moved == 0 || single_sweep) break;
    }
    free(prop); free(accept); free(lo); free(lst);
    return sweeps;
}

/* ------------------------------------------------------------------------
 * Aggregation (Algorithm 4)
 * --------------------------------------------------------------------- */

/* countCommunityVertices + exclusiveScan + fill: the community-vertex CSR
 * G'_{C'} (members of each community, ascending vertex id within a row). */
int og_community_vertices(int64_t n, const int32_t *C, int64_t ncomm, int64_t *coff, int32_t *members) {
    for (int64_t c = 0; c <= ncomm; ++c) coff[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (C[i] < 0 || C[i] >= ncomm) return OG_ERR_INVALID;
        coff[C[i] + 1]++;
    }
    for (int64_t c = 0; c < ncomm; ++c) coff[c + 1] += coff[c];
    int64_t *cur = (int64_t *)malloc((size_t)(ncomm ? ncomm : 1) * sizeof(int64_t));
    if (!cur) return OG_ERR_OOM;
    memcpy(cur, coff, (size_t)ncomm * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) members[cur[C[i]]++] = (int32_t)i;
    free(cur);
    return OG_OK;
}

static int cmp_int32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* leidenAggregate (Algorithm 4): super-vertex graph G'' as a holey CSR whose
 * row c has capacity communityTotalDegree(c) (sum of member degrees). */
static int aggregate(const og_graph *g, const int32_t *C, int64_t ncomm, og_graph *out) {
    int64_t n = g->n;
    int rc = OG_ERR_OOM;
    int64_t *coff = (int64_t *)malloc((size_t)(ncomm + 1) * sizeof(int64_t));
    int32_t *members = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    og_table H;
    memset(out, 0, sizeof(*out));
    if (table_init(&H, ncomm) || !coff || !members) goto done;
    if ((rc = og_community_vertices(n, C, ncomm, coff, members)) != OG_OK) goto done;
    rc = OG_ERR_OOM;
    out->n = ncomm;
    out->off = (int64_t *)calloc((size_t)ncomm + 1, sizeof(int64_t));
    out->deg = (int32_t *)calloc((size_t)(ncomm ? ncomm : 1), sizeof(int32_t));
    if (!out->off || !out->deg) goto done;
    /* communityTotalDegree + exclusiveScan */
    for (int64_t i = 0; i < n; ++i) out->off[C[i] + 1] += g->deg[i];
    for (int64_t c = 0; c < ncomm; ++c) out->off[c + 1] += out->off[c];
    int64_t cap = out->off[ncomm];
    out->idx = (int32_t *)malloc((size_t)(cap ? cap : 1) * sizeof(int32_t));
    out->w = (double *)malloc((size_t)(cap ? cap : 1) * sizeof(double));
    if (!out->idx || !out->w) goto done;
    for (int64_t e = 0; e < cap; ++e) { out->idx[e] = -1; out->w[e] = 0.0; }
    for (int64_t c = 0; c < ncomm; ++c) {
        table_clear(&H);
        for (int64_t k = coff[c]; k < coff[c + 1]; ++k) scan_communities(&H, g, C, members[k], 1);
        qsort(H.keys, (size_t)H.nkeys, sizeof(int32_t), cmp_int32); /* R10 */
        for (int64_t k = 0; k < H.nkeys; ++k) {
            int32_t d = H.keys[k];
            out->idx[out->off[c] + k] = d;
            out->w[out->off[c] + k] = H.val[d];
        }
        out->deg[c] = (int32_t)H.nkeys;
    }
    rc = OG_OK;
done:
    free(coff); free(members); table_free(&H);
    if (rc != OG_OK) graph_free(out);
    return rc;
}

/* exported wrapper of leidenAggregate for tests; out arrays are sized by the
 * caller: out_off[ncomm+1], out_deg[ncomm], out_idx/out_w[sum of deg]. */
int og_aggregate(int64_t n, const int64_t *off, const int32_t *deg, const int32_t *idx, const double *w,
                 const int32_t *C, int64_t ncomm, int64_t *out_off, int32_t *out_deg, int32_t *out_idx,
                 double *out_w) {
    og_graph g = {n, (int64_t *)off, (int32_t *)deg, (int32_t *)idx, (double *)w};
    og_graph r;
    int rc = aggregate(&g, C, ncomm, &r);
    if (rc != OG_OK) return rc;
    memcpy(out_off, r.off, (size_t)(ncomm + 1) * sizeof(int64_t));
    memcpy(out_deg, r.deg, (size_t)ncomm * sizeof(int32_t));
    memcpy(out_idx, r.idx, (size_t)r.off[ncomm] * sizeof(int32_t));
    memcpy(out_w, r.w, (size_t)r.off[ncomm] * sizeof(double));
    graph_free(&r);
    return OG_OK;
}

/* ------------------------------------------------------------------------
 * Modularity (Eq. 1, community form), delta-modularity (Eq. 2)
 * --------------------------------------------------------------------- */

/* Q = sum_c [ sigma_c / 2m - gamma (Sigma_c / 2m)^2 ], sigma_c = weight of the
 * CSR entries with both ends in c, Sigma_c = total weight of entries leaving
 * vertices of c. Labels must lie in [0, n). */
static double modularity_g(const og_graph *g, const int32_t *C, double gamma) {
    int64_t n = g->n;
    double *sig_in = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *sig_tot = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    if (!sig_in || !sig_tot) { free(sig_in); free(sig_tot); return NAN; }
    double two_m = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = g->off[i]; e < g->off[i] + g->deg[i]; ++e) {
            two_m += g->w[e];
            sig_tot[C[i]] += g->w[e];
            if (C[g->idx[e]] == C[i]) sig_in[C[i]] += g->w[e];
        }
    double q = 0.0;
    if (two_m > 0.0)
        for (int64_t c = 0; c < n; ++c) {
            double a = sig_tot[c] / two_m;
            q += sig_in[c] / two_m - gamma * a * a;
        }
    free(sig_in); free(sig_tot);
    return q;
}

static int to_graph(int64_t n, const int64_t *off, const int32_t *idx, const float *wf, og_graph *g) {
    g->n = n;
    int64_t nnz = off[n];
    g->off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    g->deg = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    g->idx = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    g->w = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    if (!g->off || !g->deg || !g->idx || !g->w) { graph_free(g); return OG_ERR_OOM; }
    memcpy(g->off, off, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(g->idx, idx, (size_t)nnz * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) g->deg[i] = (int32_t)(off[i + 1] - off[i]);
    for (int64_t e = 0; e < nnz; ++e) g->w[e] = wf ? (double)wf[e] : 1.0;
    return OG_OK;
}

/* Eq. 1 on a plain CSR with float weights (NULL weights = unit). */
double og_modularity(int64_t n, const int64_t *off, const int32_t *idx, const float *w, const int32_t *C,
                     double gamma) {
    og_graph g;
    if (to_graph(n, off, idx, w, &g) != OG_OK) return NAN;
    for (int64_t i = 0; i < n; ++i)
        if (C[i] < 0 || C[i] >= n) { graph_free(&g); return NAN; }
    double q = modularity_g(&g, C, gamma);
    graph_free(&g);
    return q;
}

/* Eq. 1 on a holey CSR with fp64 weights. */
double og_modularity_holey(int64_t n, const int64_t *off, const int32_t *deg, const int32_t *idx,
                           const double *w, const int32_t *C, double gamma) {
    og_graph g = {n, (int64_t *)off, (int32_t *)deg, (int32_t *)idx, (double *)w};
    for (int64_t i = 0; i < n; ++i)
        if (C[i] < 0 || C[i] >= n) return NAN;
    return modularity_g(&g, C, gamma);
}

/* Eq. 2 for moving vertex i from its community C[i] to community c, with K
 * and Sigma recomputed from scratch from C. */
double og_delta_modularity(int64_t n, const int64_t *off, const int32_t *deg, const int32_t *idx,
                           const double *w, const int32_t *C, int64_t i, int32_t c, double gamma) {
    og_graph g = {n, (int64_t *)off, (int32_t *)deg, (int32_t *)idx, (double *)w};
    double *K = (double *)calloc((size_t)n, sizeof(double));
    double *Sig = (double *)calloc((size_t)n, sizeof(double));
    if (!K || !Sig) { free(K); free(Sig); return NAN; }
    vertex_weights(&g, K);
    double two_m = 0.0;
    for (int64_t v = 0; v < n; ++v) { two_m += K[v]; Sig[C[v]] += K[v]; }
    double Kic = 0.0, Kid = 0.0;
    int32_t d = C[i];
    for (int64_t e = off[i]; e < off[i] + deg[i]; ++e) {
        if (idx[e] == i) continue;
        if (C[idx[e]] == c) Kic += w[e];
        if (C[idx[e]] == d) Kid += w[e];
    }
    double r = delta_q(Kic, Kid, K[i], Sig[c], Sig[d], two_m / 2.0, gamma);
    free(K); free(Sig);
    return r;
}

/* S1 key difference key(c) - key_d for moving i from C[i] to c (integer
 * weights): equals dQ * 2m^2 exactly. */
int64_t og_delta_key(int64_t n, const int64_t *off, const int32_t *deg, const int32_t *idx, const double *w,
                     const int32_t *C, int64_t i, int32_t c) {
    int64_t two_m = 0, Ki = 0, Sc = 0, Sd = 0, Kic = 0, Kid = 0;
    int32_t d = C[i];
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = off[v]; e < off[v] + deg[v]; ++e) {
            int64_t x = (int64_t)w[e];
            two_m += x;
            if (C[v] == c) Sc += x;
            if (C[v] == d) Sd += x;
            if (v == i) {
                Ki += x;
                if (idx[e] != i && C[idx[e]] == c) Kic += x;
                if (idx[e] != i && C[idx[e]] == d) Kid += x;
            }
        }
    int64_t key_c = two_m * Kic - Ki * Sc;
    int64_t key_d = two_m * Kid - Ki * (Sd - Ki);
    return key_c - key_d;
}

/* ------------------------------------------------------------------------
 * Disconnected communities (Algorithm 5): BFS inside each community from
 * its first vertex; a community is disconnected if the BFS reaches fewer
 * vertices than its size. flags[c] (n entries) is set per community.
 * Returns the number of disconnected communities, or -1 on error.
 * --------------------------------------------------------------------- */
int64_t og_disconnected(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *C, uint8_t *flags) {
    if (n < 0) return -1;
    int64_t *S = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    uint8_t *vis = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    int32_t *queue = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!S || !vis || !queue) { free(S); free(vis); free(queue); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        if (C[i] < 0 || C[i] >= n) { free(S); free(vis); free(queue); return -1; }
        S[C[i]]++;
    }
    if (flags) memset(flags, 0, (size_t)n);
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = C[i];
        if (S[c] == 0) continue;
        int64_t head = 0, tail = 0, reached = 0;
        queue[tail++] = (int32_t)i;
        vis[i] = 1;
        while (head < tail) {
            int32_t u = queue[head++];
            reached++;
            for (int64_t e = off[u]; e < off[u + 1]; ++e) {
                int32_t v = idx[e];
                if (C[v] != c || vis[v]) continue;
                vis[v] = 1;
                queue[tail++] = v;
            }
        }
        if (reached < S[c]) { if (flags) flags[c] = 1; count++; }
        S[c] = 0;
    }
    free(S); free(vis); free(queue);
    return count;
}

/* ------------------------------------------------------------------------
 * Brute force: the maximum of Eq. 1 over all set partitions of n <= 12
 * vertices, enumerated as restricted growth strings.
 * --------------------------------------------------------------------- */
double og_brute_force(int64_t n, const int64_t *off, const int32_t *idx, const float *w, double gamma,
                      int32_t *best_C) {
    if (n < 0 || n > 12) return NAN;
    if (n == 0) return 0.0;
    og_graph g;
    if (to_graph(n, off, idx, w, &g) != OG_OK) return NAN;
    int32_t a[12], mx[12];
    double best = -INFINITY;
    for (int64_t i = 0; i < n; ++i) { a[i] = 0; mx[i] = 0; }
    for (;;) {
        double q = modularity_g(&g, a, gamma);
        if (q > best) {
            best = q;
            if (best_C) for (int64_t i = 0; i < n; ++i) best_C[i] = a[i];
        }
        /* next restricted growth string: a[0] = 0, a[i] <= 1 + max(a[0..i-1]) */
        int64_t i = n - 1;
        while (i > 0 && a[i] == mx[i - 1] + 1) --i;
        if (i == 0) break;
        a[i]++;
        mx[i] = a[i] > mx[i - 1] ? a[i] : mx[i - 1];
        for (int64_t k = i + 1; k < n; ++k) { a[k] = 0; mx[k] = mx[i]; }
    }
    graph_free(&g);
    return best;
}

/* ------------------------------------------------------------------------
 * leiden (Algorithm 1)
 * --------------------------------------------------------------------- */
void og_params_default(og_params *p) {
    p->resolution = 1.0;
    p->tolerance = 0.01;
    p->aggregation_tolerance = 0.8;
    p->tolerance_drop = 10.0;
    p->max_iterations = 20;
    p->max_passes = 10;
    p->mode = OG_SEQ;
    p->flags = 0;
    p->schedule_layers = 0;
    p->schedule_buckets = 16;
    p->seed = 0;
}

static void trace_graph(og_trace_fn cb, void *ctx, int32_t pass, const og_graph *g) {
    if (!cb) return;
    int64_t cap = g->off[g->n];
    cb(ctx, pass, OG_T_AGG_OFF, g->off, g->n + 1);
    cb(ctx, pass, OG_T_AGG_DEG, g->deg, g->n);
    cb(ctx, pass, OG_T_AGG_IDX, g->idx, cap);
    cb(ctx, pass, OG_T_AGG_W, g->w, cap);
}

/* Runs Algorithm 1 on the symmetric CSR (offsets, indices, weights; NULL
 * weights = unit). membership[n] receives the canonical labels (the rank of
 * each community's smallest vertex id); *q_out the modularity (Eq. 1) of the
 * result on the input graph; *passes_out the passes executed. */
int og_leiden(int64_t n0, const int64_t *off0, const int32_t *idx0, const float *w0, const og_params *p,
              int32_t *membership, double *q_out, int32_t *passes_out, og_trace_fn cb, void *ctx) {
    if (n0 < 0 || !off0 || (n0 > 0 && !membership) || !p) return OG_ERR_INVALID;
    if (off0[0] != 0) return OG_ERR_INVALID;
    for (int64_t i = 0; i < n0; ++i)
        if (off0[i + 1] < off0[i] || off0[i + 1] - off0[i] > INT32_MAX) return OG_ERR_INVALID;
    int64_t nnz = off0[n0];
    for (int64_t e = 0; e < nnz; ++e) {
        if (idx0[e] < 0 || idx0[e] >= n0) return OG_ERR_INVALID;
        if (w0 && (!isfinite(w0[e]) || w0[e] < 0.0f)) return OG_ERR_INVALID;
    }
    if (p->max_iterations < 1 || p->max_passes < 0 || !(p->tolerance_drop > 0)) return OG_ERR_INVALID;
    if (p->mode == OG_SYNC && (p->schedule_layers < 0 || p->schedule_buckets < 1)) return OG_ERR_INVALID;
    if (p->mode == OG_SYNC && (p->flags & OG_RANDOM_REFINE)) return OG_ERR_UNSUPPORTED; /* V3: SEQ only */
    /* S0: L of the run (0: 1000 for a heavy-tailed input, largest degree
     * above 64 times the mean degree nnz/n; else 32) */
    int32_t Ls = p->schedule_layers;
    if (Ls == 0) {
        int64_t maxdeg = 0;
        for (int64_t i = 0; i < n0; ++i)
            if (off0[i + 1] - off0[i] > maxdeg) maxdeg = off0[i + 1] - off0[i];
        Ls = (og_i128)maxdeg * n0 > (og_i128)64 * nnz ? 1000 : 32;
    }
    int sync = (p->mode == OG_SYNC);
    if (sync) {
        if (p->resolution != 1.0) return OG_ERR_UNSUPPORTED;
        double s = 0.0;
        for (int64_t e = 0; e < nnz; ++e) {
            double x = w0 ? (double)w0[e] : 1.0;
            if (x != floor(x)) return OG_ERR_UNSUPPORTED;
            s += x;
        }
        if (s >= 9007199254740992.0) return OG_ERR_OVERFLOW; /* S1: 2m < 2^53 */
    }
    if (passes_out) *passes_out = 0;
    if (q_out) *q_out = 0.0;
    if (n0 == 0) return OG_OK;

    int rc = OG_ERR_OOM;
    og_graph G;  /* G' of the current pass */
    memset(&G, 0, sizeof(G));
    int32_t *C = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));   /* dendrogram */
    int32_t *Cp = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));  /* C' */
    int32_t *CB = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));  /* C'_B */
    int32_t *init = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));
    int32_t *size = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));
    int32_t *newid = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));
    int32_t *layer = (int32_t *)malloc((size_t)n0 * sizeof(int32_t));
    double *K = (double *)malloc((size_t)n0 * sizeof(double));
    double *Sig = (double *)malloc((size_t)n0 * sizeof(double));
    int64_t *Ki = (int64_t *)malloc((size_t)n0 * sizeof(int64_t));
    int64_t *Si = (int64_t *)malloc((size_t)n0 * sizeof(int64_t));
    og_table H;
    memset(&H, 0, sizeof(H));
    if (!C || !Cp || !CB || !init || !size || !newid || !layer || !K || !Sig || !Ki || !Si) goto done;
    if (table_init(&H, n0)) goto done;
    if (to_graph(n0, off0, idx0, w0, &G) != OG_OK) goto done;

    for (int64_t v = 0; v < n0; ++v) C[v] = (int32_t)v; /* C <- [0..|V|) */
    int fresh = 1; /* R5': the pass begins with every super-vertex in its own community */
    double tau = p->tolerance;
    double gamma = p->resolution;
    int broke = 0, passes = 0;
    for (int32_t lp = 0; lp < p->max_passes; ++lp) {
        int64_t n = G.n;
        /* Sigma' <- K' <- vertexWeights(G'); C' <- initial labels (R3) */
        vertex_weights(&G, K);
        double two_m = 0.0;
        for (int64_t i = 0; i < n; ++i) two_m += K[i];
        if (lp == 0)
            for (int64_t i = 0; i < n; ++i) init[i] = (int32_t)i;
        if (!(two_m > 0.0)) { /* R12 */
            for (int64_t i = 0; i < n; ++i) Cp[i] = (int32_t)i;
            broke = 1;
            passes++;
            break;
        }
        passes++;
        for (int64_t i = 0; i < n; ++i) {
            Cp[i] = init[i];
            Sig[i] = 0.0; Si[i] = 0; size[i] = 0;
            Ki[i] = (int64_t)K[i];
        }
        for (int64_t i = 0; i < n; ++i) { Sig[Cp[i]] += K[i]; Si[Cp[i]] += Ki[i]; size[Cp[i]]++; }
        if (cb) cb(ctx, lp, OG_T_INIT_LABELS, Cp, n);

        /* S0: priority steps of this pass's graph */
        int32_t nl = 0;
        if (sync) {
            nl = og_schedule(n, G.off, G.deg, G.idx, p->seed + (uint64_t)lp, Ls, p->schedule_buckets, layer);
            if (nl < 0) goto done;
        }
        /* local-moving phase (Algorithm 2) */
        int li = sync ? move_sync(&G, Cp, Ki, Si, size, tau, (int64_t)two_m, p->max_iterations,
                                  Ls, layer, nl, &H)
                      : move_seq(&G, Cp, K, Sig, tau, gamma, two_m, p->max_iterations,
                                 (p->flags & OG_NO_PRUNE) != 0, &H);
        if (li < 0) goto done;
        if (cb) cb(ctx, lp, OG_T_MOVE, Cp, n);

        int lj = 0;
        if (p->flags & OG_LOUVAIN) { /* V2: the local-moving partition is the refined one */
            for (int64_t i = 0; i < n; ++i) CB[i] = Cp[i];
        } else {
            /* C'_B <- C'; C' <- [0..|V'|); Sigma' <- K' */
            for (int64_t i = 0; i < n; ++i) {
                CB[i] = Cp[i]; Cp[i] = (int32_t)i; Sig[i] = K[i]; Si[i] = Ki[i]; size[i] = 1;
            }
            /* refinement phase (Algorithm 3) */
            int single = (p->flags & OG_REFINE_SINGLE_SWEEP) != 0;
            const uint64_t rstate = p->seed + 0xD1B54A32D192ED03ULL * (uint64_t)(64 * lp); /* V3 draws */
            lj = sync ? refine_sync(&G, CB, Cp, Ki, Si, size, (int64_t)two_m, p->max_iterations, single,
                                    layer, nl, &H)
                      : refine_seq(&G, CB, Cp, K, Sig, size, gamma, two_m, p->max_iterations, single, &H,
                                   (p->flags & OG_RANDOM_REFINE) ? &rstate : NULL, newid);
            if (lj < 0) goto done;
        }
        if (cb) cb(ctx, lp, OG_T_REFINE, Cp, n);

        /* |Gamma| (R4): number of non-empty refined communities */
        int64_t ncomm = 0;
        for (int64_t c = 0; c < n; ++c) newid[c] = -1;
        for (int64_t i = 0; i < n; ++i) newid[Cp[i]] = 0;
        for (int64_t c = 0; c < n; ++c)
            if (newid[c] == 0) newid[c] = (int32_t)ncomm++; /* R9: ascending old id */
        if (cb) {
            int64_t counts[4] = {n, li, lj, ncomm};
            cb(ctx, lp, OG_T_COUNTS, counts, 4);
        }
        /* R5': number of local-moving communities */
        int64_t nbound = 0;
        for (int64_t c = 0; c < n; ++c) size[c] = 0;
        for (int64_t i = 0; i < n; ++i) { if (!size[CB[i]]) nbound++; size[CB[i]] = 1; }
        if (li <= 1 && nbound == ncomm && fresh) { broke = 1; break; }           /* R5' */
        int64_t z = 0; /* R4: vertices without edges */
        for (int64_t i = 0; i < n; ++i) z += G.deg[i] == 0;
        if ((double)(ncomm - z) / (double)(n - z) > p->aggregation_tolerance) { broke = 1; break; } /* R4 */
        /* R5': the next pass starts from singletons when every local-moving
         * community is one refined community (move-based labels, R3) or
         * under refine-based labels (V1) */
        fresh = (p->flags & OG_REFINE_LABELS) || nbound == ncomm;

        /* renumber communities in C' */
        for (int64_t i = 0; i < n; ++i) Cp[i] = newid[Cp[i]];
        if (cb) cb(ctx, lp, OG_T_RENUMBER, Cp, n);
        /* C <- lookup dendrogram using C to C' */
        for (int64_t v = 0; v < n0; ++v) C[v] = Cp[C[v]];
        if (cb) cb(ctx, lp, OG_T_DENDRO, C, n0);

        /* G' <- leidenAggregate(G', C') (Algorithm 4) */
        og_graph G2;
        if ((rc = aggregate(&G, Cp, ncomm, &G2)) != OG_OK) goto done;
        rc = OG_ERR_OOM;
        trace_graph(cb, ctx, lp, &G2);

        /* C' <- map C' to C'_B (move-based labels, R3): super-vertex s starts
         * in the community of the smallest super-vertex with the same bound */
        int32_t *bound_of = newid; /* reuse: bound of each super-vertex */
        for (int64_t i = 0; i < n; ++i) bound_of[Cp[i]] = CB[i];
        int32_t *rep = CB; /* reuse: smallest super-vertex per bound */
        for (int64_t b = 0; b < n; ++b) rep[b] = -1;
        for (int64_t s = 0; s < ncomm; ++s)
            if (rep[bound_of[s]] < 0) rep[bound_of[s]] = (int32_t)s;
        for (int64_t s = 0; s < ncomm; ++s) init[s] = rep[bound_of[s]];
        if (p->flags & OG_REFINE_LABELS) /* V1: every super-vertex alone */
            for (int64_t s = 0; s < ncomm; ++s) init[s] = (int32_t)s;

        graph_free(&G);
        G = G2;
        tau /= p->tolerance_drop; /* threshold scaling */
    }
    /* C <- lookup dendrogram using C to C' (R8: refined partition) */
    if (broke)
        for (int64_t v = 0; v < n0; ++v) C[v] = Cp[C[v]];
    /* canonical labels: rank of each community's smallest vertex id */
    for (int64_t c = 0; c < n0; ++c) newid[c] = -1;
    {
        int32_t next = 0;
        for (int64_t v = 0; v < n0; ++v) {
            if (newid[C[v]] < 0) newid[C[v]] = next++;
            membership[v] = newid[C[v]];
        }
    }
    if (q_out) *q_out = og_modularity(n0, off0, idx0, w0, membership, gamma);
    if (passes_out) *passes_out = passes;
    rc = OG_OK;
done:
    graph_free(&G);
    free(C); free(Cp); free(CB); free(init); free(size); free(newid); free(layer);
    free(K); free(Sig); free(Ki); free(Si);
    table_free(&H);
    return rc;
}
