/*
 * Seeded synthetic graph generators (input recipes only: no Leiden arithmetic).
 *
 * Every generator produces an undirected graph as a symmetric CSR:
 *   offsets[n+1] (int64), indices[nnz] (int32, rows sorted ascending, no
 *   duplicates), weights[nnz] (float32, w_ij == w_ji).
 * The graph model of the paper is undirected and weighted with w_ij = w_ji
 * (Section 3, "Preliminaries"); its |E| counts both directions of each edge
 * (Table 2 caption), which is what nnz counts here.
 *
 * Random numbers: splitmix64 seeds xoshiro256** (Blackman & Vigna,
 * "Scrambled linear pseudorandom number generators", 2021). Uniform doubles
 * take the top 53 bits. Results are identical on x86_64 and aarch64.
 *
 * Memory returned through the out-pointers is malloc'ed here and released
 * with gg_free().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int k = 0; k < 4; ++k) r->s[k] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return out;
}
/* uniform in [0,1) */
static inline double rng_u01(gg_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* uniform integer in [0, k) (k > 0), Lemire-free simple rejection */
static inline uint64_t rng_below(gg_rng *r, uint64_t k) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % k);
    uint64_t x;
    do { x = rng_next(r); } while (x >= lim);
    return x % k;
}

void gg_free(void *p) { free(p); }

/* -------------------------------------------------------- edge buffer */
typedef struct { int64_t n, cap; int32_t *u, *v; float *w; } ebuf;

static int eb_push(ebuf *b, int32_t u, int32_t v, float w) {
    if (b->n == b->cap) {
        int64_t nc = b->cap ? b->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(b->u, nc * sizeof(int32_t));
        if (!nu) return -1;
        b->u = nu;
        int32_t *nv = (int32_t *)realloc(b->v, nc * sizeof(int32_t));
        if (!nv) return -1;
        b->v = nv;
        float *nw = (float *)realloc(b->w, nc * sizeof(float));
        if (!nw) return -1;
        b->w = nw;
        b->cap = nc;
    }
    b->u[b->n] = u; b->v[b->n] = v; b->w[b->n] = w; b->n++;
    return 0;
}
static void eb_release(ebuf *b) { free(b->u); free(b->v); free(b->w); memset(b, 0, sizeof(*b)); }

/* sort one row's (idx, w) pairs ascending by idx: insertion sort for short
 * rows, heap sort for long ones (no recursion, no allocation). */
static void row_sort(int32_t *ix, float *wt, int64_t len) {
    if (len < 32) {
        for (int64_t a = 1; a < len; ++a) {
            int32_t k = ix[a]; float x = wt[a]; int64_t b = a - 1;
            while (b >= 0 && ix[b] > k) { ix[b + 1] = ix[b]; wt[b + 1] = wt[b]; --b; }
            ix[b + 1] = k; wt[b + 1] = x;
        }
        return;
    }
    /* heap sort */
    for (int64_t start = len / 2 - 1; ; --start) {
        int64_t root = start;
        for (;;) {
            int64_t c = 2 * root + 1;
            if (c >= len) break;
            if (c + 1 < len && ix[c + 1] > ix[c]) c++;
            if (ix[root] >= ix[c]) break;
            int32_t t = ix[root]; ix[root] = ix[c]; ix[c] = t;
            float tw = wt[root]; wt[root] = wt[c]; wt[c] = tw;
            root = c;
        }
        if (start == 0) break;
    }
    for (int64_t end = len - 1; end > 0; --end) {
        int32_t t = ix[0]; ix[0] = ix[end]; ix[end] = t;
        float tw = wt[0]; wt[0] = wt[end]; wt[end] = tw;
        int64_t root = 0;
        for (;;) {
            int64_t c = 2 * root + 1;
            if (c >= end) break;
            if (c + 1 < end && ix[c + 1] > ix[c]) c++;
            if (ix[root] >= ix[c]) break;
            int32_t t2 = ix[root]; ix[root] = ix[c]; ix[c] = t2;
            float tw2 = wt[root]; wt[root] = wt[c]; wt[c] = tw2;
            root = c;
        }
    }
}

/* Build a symmetric CSR from undirected pairs (u != v, or u == v for a
 * self-loop, stored once). If dedup != 0, repeated pairs keep the first weight
 * seen after sorting (callers that dedup use unit weights). */
static int build_csr(int64_t n, int64_t ne, const int32_t *eu, const int32_t *ev, const float *ew,
                     int dedup, int64_t **off_out, int32_t **idx_out, float **w_out, int64_t *nnz_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off) return -1;
    for (int64_t e = 0; e < ne; ++e) {
        off[eu[e] + 1]++;
        if (eu[e] != ev[e]) off[ev[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
    int64_t nnz = off[n];
    int32_t *idx = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    float *w = (float *)malloc((size_t)(nnz ? nnz : 1) * sizeof(float));
    int64_t *cur = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!idx || !w || !cur) { free(off); free(idx); free(w); free(cur); return -1; }
    memcpy(cur, off, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = eu[e], b = ev[e];
        idx[cur[a]] = b; w[cur[a]] = ew[e]; cur[a]++;
        if (a != b) { idx[cur[b]] = a; w[cur[b]] = ew[e]; cur[b]++; }
    }
    free(cur);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) row_sort(idx + off[i], w + off[i], off[i + 1] - off[i]);
    if (dedup) {
        int64_t wpos = 0;
        int64_t prev_end = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t s = prev_end, t = off[i + 1];
            prev_end = t;
            off[i] = wpos;
            for (int64_t k = s; k < t; ++k) {
                if (k > s && idx[k] == idx[k - 1]) continue;
                idx[wpos] = idx[k]; w[wpos] = w[k]; wpos++;
            }
        }
        off[n] = wpos;
        nnz = wpos;
    }
    *off_out = off; *idx_out = idx; *w_out = w; *nnz_out = nnz;
    return 0;
}

/* ------------------------------------------------------------------ SBM */
/* Emit the pairs of one block pair with Bernoulli(p) each, by geometric
 * skipping over the pair index space (Batagelj & Brandes 2005). For a == b
 * the space is the strict upper triangle of an s x s block. */
static int sbm_block_pair(gg_rng *r, ebuf *eb, int64_t sa, int64_t a0, int64_t sb, int64_t b0,
                          int same, double p) {
    double npairs = same ? (double)sa * (double)(sa - 1) / 2.0 : (double)sa * (double)sb;
    if (npairs <= 0 || p <= 0) return 0;
    double lq = (p < 1.0) ? log1p(-p) : 0.0;
    double k = -1.0;
    for (;;) {
        if (p >= 1.0) k += 1.0;
        else {
            double u = rng_u01(r);
            k += 1.0 + floor(log1p(-u) / lq);
        }
        if (k >= npairs) break;
        int64_t ui, vi;
        if (same) {
            /* row i of the triangle holds pairs (i, i+1..s-1): find i with
             * T(i) <= k < T(i+1), T(i) = i*s - i*(i+1)/2 */
            double s = (double)sa;
            double disc = (2.0 * s - 1.0) * (2.0 * s - 1.0) - 8.0 * k;
            int64_t i = (int64_t)floor(((2.0 * s - 1.0) - sqrt(disc > 0 ? disc : 0)) / 2.0);
            if (i < 0) i = 0;
            while (i > 0 && (double)i * s - (double)i * (i + 1) / 2.0 > k) --i;
            while ((double)(i + 1) * s - (double)(i + 1) * (i + 2) / 2.0 <= k) ++i;
            double ti = (double)i * s - (double)i * (i + 1) / 2.0;
            int64_t j = i + 1 + (int64_t)(k - ti);
            ui = a0 + i; vi = a0 + j;
        } else {
            int64_t kk = (int64_t)k;
            ui = a0 + kk / sb; vi = b0 + kk % sb;
        }
        if (eb_push(eb, (int32_t)ui, (int32_t)vi, 1.0f)) return -1;
    }
    return 0;
}

/* Stochastic block model: n vertices in `blocks` near-equal blocks (the first
 * n % blocks blocks hold one extra vertex), p_in inside a block, p_out across.
 * Unit weights, no self-loops. block_of (optional, n entries) gets the
 * planted block of each vertex. */
int gg_sbm(int64_t n, int32_t blocks, double p_in, double p_out, uint64_t seed,
           int64_t **off, int32_t **idx, float **w, int64_t *nnz, int32_t *block_of) {
    if (n < 0 || blocks < 1 || n > INT32_MAX) return -2;
    gg_rng r; rng_seed(&r, seed);
    ebuf eb = {0};
    int64_t base = n / blocks, extra = n % blocks;
    int64_t *start = (int64_t *)malloc(((size_t)blocks + 1) * sizeof(int64_t));
    if (!start) return -1;
    start[0] = 0;
    for (int32_t b = 0; b < blocks; ++b) start[b + 1] = start[b] + base + (b < extra ? 1 : 0);
    if (block_of)
        for (int32_t b = 0; b < blocks; ++b)
            for (int64_t v = start[b]; v < start[b + 1]; ++v) block_of[v] = b;
    for (int32_t a = 0; a < blocks; ++a)
        for (int32_t b = a; b < blocks; ++b) {
            int64_t sa = start[a + 1] - start[a], sb = start[b + 1] - start[b];
            if (sbm_block_pair(&r, &eb, sa, start[a], sb, start[b], a == b, a == b ? p_in : p_out)) {
                eb_release(&eb); free(start); return -1;
            }
        }
    free(start);
    int rc = build_csr(n, eb.n, eb.u, eb.v, eb.w, 0, off, idx, w, nnz);
    eb_release(&eb);
    return rc;
}

/* Batch of SBM graphs, each generated exactly as gg_sbm generates it alone
 * (graph g: n[g] vertices, blocks[g] near-equal blocks, p_in[g], p_out[g],
 * seeds[g]), in parallel over graphs, then packed one after another: vseg
 * (G+1 vertex offsets), off (N+1 offsets into the packed idx/w), idx (LOCAL
 * to each graph), w; *nnz = total entries. */
int gg_sbm_batch(int32_t G, const int64_t *n, const int32_t *blocks, const double *p_in, const double *p_out,
                 const uint64_t *seeds, int64_t **vseg_out, int64_t **off_out, int32_t **idx_out, float **w_out,
                 int64_t *nnz_out) {
    if (G < 0) return -2;
    int64_t **offs = (int64_t **)calloc((size_t)G + 1, sizeof(int64_t *));
    int32_t **idxs = (int32_t **)calloc((size_t)G + 1, sizeof(int32_t *));
    float **ws = (float **)calloc((size_t)G + 1, sizeof(float *));
    int64_t *m = (int64_t *)calloc((size_t)G + 1, sizeof(int64_t));
    int64_t *vseg = (int64_t *)malloc(((size_t)G + 1) * sizeof(int64_t));
    int64_t *eseg = (int64_t *)malloc(((size_t)G + 1) * sizeof(int64_t));
    int err = !offs || !idxs || !ws || !m || !vseg || !eseg;
    if (!err) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
        for (int32_t g = 0; g < G; ++g)
            err |= gg_sbm(n[g], blocks[g], p_in[g], p_out[g], seeds[g], &offs[g], &idxs[g], &ws[g], &m[g], NULL) != 0;
    }
    int64_t *off = NULL;
    int32_t *idx = NULL;
    float *w = NULL;
    if (!err) {
        vseg[0] = 0;
        eseg[0] = 0;
        for (int32_t g = 0; g < G; ++g) {
            vseg[g + 1] = vseg[g] + n[g];
            eseg[g + 1] = eseg[g] + m[g];
        }
        if (vseg[G] > INT32_MAX) err = 1;
    }
    if (!err) {
        off = (int64_t *)malloc(((size_t)vseg[G] + 1) * sizeof(int64_t));
        idx = (int32_t *)malloc((size_t)(eseg[G] ? eseg[G] : 1) * sizeof(int32_t));
        w = (float *)malloc((size_t)(eseg[G] ? eseg[G] : 1) * sizeof(float));
        err = !off || !idx || !w;
    }
    if (!err) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t g = 0; g < G; ++g) {
            for (int64_t i = 0; i < n[g]; ++i) off[vseg[g] + i] = offs[g][i] + eseg[g];
            if (m[g]) {
                memcpy(idx + eseg[g], idxs[g], (size_t)m[g] * sizeof(int32_t));
                memcpy(w + eseg[g], ws[g], (size_t)m[g] * sizeof(float));
            }
        }
        off[vseg[G]] = eseg[G];
    }
    for (int32_t g = 0; g < G && offs; ++g) {
        free(offs[g]);
        if (idxs) free(idxs[g]);
        if (ws) free(ws[g]);
    }
    free(offs); free(idxs); free(ws); free(eseg);
    if (err) {
        free(m); free(vseg); free(off); free(idx); free(w);
        return -1;
    }
    *nnz_out = vseg[G] >= 0 ? off[vseg[G]] : 0;
    free(m);
    *vseg_out = vseg;
    *off_out = off;
    *idx_out = idx;
    *w_out = w;
    return 0;
}

/* ------------------------------------------------------------- road grid */
/* side x side 4-neighbour lattice (vertex r*side+c). Each lattice edge is kept
 * with probability 1-drop. Then round(diag_frac * #lattice edges) diagonal
 * shortcuts (r,c)-(r+1,c+o), o in {-1,+1}, cell and orientation uniform,
 * out-of-grid and repeated draws redrawn. Integer weights uniform in
 * [wmin, wmax], stored as float. Draw order: horizontal edges row-major,
 * then vertical edges row-major (keep draw, then weight draw for kept ones),
 * then diagonals. */
int gg_road(int32_t side, double drop, double diag_frac, int32_t wmin, int32_t wmax, uint64_t seed,
            int64_t **off, int32_t **idx, float **w, int64_t *nnz) {
    if (side < 1 || wmin > wmax) return -2;
    int64_t n = (int64_t)side * side;
    if (n > INT32_MAX) return -2;
    gg_rng r; rng_seed(&r, seed);
    int64_t nlat = 2LL * side * (side - 1);
    int64_t ndiag = (int64_t)llround(diag_frac * (double)nlat);
    ebuf eb = {0};
    eb.cap = (int64_t)((double)nlat * (1.0 - drop) * 1.01) + ndiag + 1024;
    eb.u = (int32_t *)malloc(eb.cap * sizeof(int32_t));
    eb.v = (int32_t *)malloc(eb.cap * sizeof(int32_t));
    eb.w = (float *)malloc(eb.cap * sizeof(float));
    if (!eb.u || !eb.v || !eb.w) { eb_release(&eb); return -1; }
    uint64_t wspan = (uint64_t)(wmax - wmin + 1);
    for (int dir = 0; dir < 2; ++dir)
        for (int64_t rr = 0; rr < side; ++rr)
            for (int64_t cc = 0; cc < side; ++cc) {
                int64_t u = rr * side + cc, v;
                if (dir == 0) { if (cc + 1 >= side) continue; v = u + 1; }
                else { if (rr + 1 >= side) continue; v = u + side; }
                double x = rng_u01(&r);
                if (x < drop) continue;
                float wt = (float)(wmin + (int64_t)rng_below(&r, wspan));
                if (eb_push(&eb, (int32_t)u, (int32_t)v, wt)) { eb_release(&eb); return -1; }
            }
    if (ndiag > 0 && side > 1) {
        /* a diagonal is identified by its upper vertex (r,c) and orientation */
        size_t nbits = (size_t)n * 2;
        uint8_t *seen = (uint8_t *)calloc((nbits + 7) / 8, 1);
        if (!seen) { eb_release(&eb); return -1; }
        int64_t made = 0;
        while (made < ndiag) {
            int64_t rr = (int64_t)rng_below(&r, (uint64_t)(side - 1));
            int64_t cc = (int64_t)rng_below(&r, (uint64_t)side);
            int o = (rng_next(&r) >> 63) ? 1 : -1;
            if (cc + o < 0 || cc + o >= side) continue;
            size_t key = (size_t)(rr * side + cc) * 2 + (o > 0);
            if (seen[key >> 3] & (1u << (key & 7))) continue;
            seen[key >> 3] |= (uint8_t)(1u << (key & 7));
            float wt = (float)(wmin + (int64_t)rng_below(&r, wspan));
            if (eb_push(&eb, (int32_t)(rr * side + cc), (int32_t)((rr + 1) * side + cc + o), wt)) {
                free(seen); eb_release(&eb); return -1;
            }
            made++;
        }
        free(seen);
    }
    int rc = build_csr(n, eb.n, eb.u, eb.v, eb.w, 0, off, idx, w, nnz);
    eb_release(&eb);
    return rc;
}

/* ----------------------------------------------------------------- R-MAT */
/* R-MAT (Chakrabarti, Zhan & Faloutsos 2004): 2^scale vertices,
 * edge_factor * 2^scale generated directed edges, quadrant probabilities
 * (a, b, c, 1-a-b-c) at every bit level, no noise. Self-loops dropped; the
 * result is symmetrised and deduplicated; unit weights. Edges are drawn in
 * fixed chunks, each chunk with its own stream seeded from (seed, chunk), so
 * the graph does not depend on the thread count. */
/* The R-MAT edge list of gg_rmat before the CSR is built: the same draws,
 * self-loops compacted away, each edge oriented u < v (duplicates kept).
 * *m_out receives the edge count; eu/ev are malloc'ed (free with gg_free). */
int gg_rmat_edges(int32_t scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                  int32_t **eu_out, int32_t **ev_out, int64_t *m_out);

int gg_rmat(int32_t scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
            int64_t **off_out, int32_t **idx_out, float **w_out, int64_t *nnz_out) {
    int32_t *eu = NULL, *ev = NULL;
    int64_t m = 0;
    int rc = gg_rmat_edges(scale, edge_factor, a, b, c, seed, &eu, &ev, &m);
    if (rc) return rc;
    float *ew = (float *)malloc((size_t)(m ? m : 1) * sizeof(float));
    if (!ew) { free(eu); free(ev); return -1; }
    for (int64_t e = 0; e < m; ++e) ew[e] = 1.0f;
    rc = build_csr((int64_t)1 << scale, m, eu, ev, ew, 1, off_out, idx_out, w_out, nnz_out);
    free(eu); free(ev); free(ew);
    return rc;
}

int gg_rmat_edges(int32_t scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                  int32_t **eu_out, int32_t **ev_out, int64_t *m_out) {
    if (scale < 1 || scale > 30 || edge_factor < 0) return -2;
    int64_t n = 1LL << scale;
    int64_t ne = edge_factor * n;
    const int64_t CH = 1 << 20;
    int64_t nch = (ne + CH - 1) / CH;
    int32_t *eu = (int32_t *)malloc((size_t)(ne ? ne : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(ne ? ne : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return -1; }
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nch; ++ch) {
        gg_rng r;
        rng_seed(&r, seed ^ (0xD1B54A32D192ED03ULL * (uint64_t)(ch + 1)));
        int64_t e0 = ch * CH, e1 = e0 + CH < ne ? e0 + CH : ne;
        for (int64_t e = e0; e < e1; ++e) {
            int64_t u = 0, v = 0;
            for (int32_t l = 0; l < scale; ++l) {
                double x = rng_u01(&r);
                int bu = 0, bv = 0;
                if (x < a) { }
                else if (x < ab) bv = 1;
                else if (x < abc) bu = 1;
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu; v = (v << 1) | bv;
            }
            eu[e] = (int32_t)u; ev[e] = (int32_t)v;
        }
    }
    /* compact away self-loops, orient u < v so each undirected edge appears
     * once before symmetrisation (duplicates are removed after sorting) */
    (void)n;
    int64_t m = 0;
    for (int64_t e = 0; e < ne; ++e) {
        if (eu[e] == ev[e]) continue;
        int32_t x = eu[e], y = ev[e];
        if (x > y) { int32_t t = x; x = y; y = t; }
        eu[m] = x; ev[m] = y; m++;
    }
    *eu_out = eu;
    *ev_out = ev;
    *m_out = m;
    return 0;
}

/* ---------------------------------------------------- G(n, p) (tiny tests) */
int gg_gnp(int64_t n, double p, int32_t wmax, uint64_t seed,
           int64_t **off, int32_t **idx, float **w, int64_t *nnz) {
    if (n < 0 || n > 100000) return -2;
    gg_rng r; rng_seed(&r, seed);
    ebuf eb = {0};
    for (int64_t u = 0; u < n; ++u)
        for (int64_t v = u + 1; v < n; ++v)
            if (rng_u01(&r) < p) {
                float wt = wmax > 1 ? (float)(1 + rng_below(&r, (uint64_t)wmax)) : 1.0f;
                if (eb_push(&eb, (int32_t)u, (int32_t)v, wt)) { eb_release(&eb); return -1; }
            }
    int rc = build_csr(n, eb.n, eb.u, eb.v, eb.w, 0, off, idx, w, nnz);
    eb_release(&eb);
    return rc;
}

/* Generic: symmetric CSR from an undirected edge list (u, v, w); u == v is a
 * self-loop stored once. Duplicate pairs are the caller's responsibility. */
int gg_from_edges(int64_t n, int64_t ne, const int32_t *u, const int32_t *v, const float *wt,
                  int64_t **off, int32_t **idx, float **w, int64_t *nnz) {
    for (int64_t e = 0; e < ne; ++e)
        if (u[e] < 0 || v[e] < 0 || u[e] >= n || v[e] >= n) return -2;
    return build_csr(n, ne, u, v, wt, 0, off, idx, w, nnz);
}
