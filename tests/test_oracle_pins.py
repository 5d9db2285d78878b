"""Pins for the CPU oracle against what the paper and the mathematics fix.

Every check here ties the oracle to something other than itself: closed forms
of Eq. 1, a dense all-pairs form of Eq. 1, exact integer arithmetic, brute
force over all set partitions, the connectivity guarantee of the Leiden
method, hand-derived fixtures under tests/golden/, and published SplitMix64
test vectors. They run on the CPU only.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import gen
import oracle
from tests._graphs import ari, dense, q_dense, q_times_4m2_exact, random_graph_with_loops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = (oracle.SEQ, oracle.SYNC)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _from_golden_edges(d):
    e = d["edges"]
    u = [x[0] for x in e]
    v = [x[1] for x in e]
    w = [x[2] if len(x) > 2 else 1.0 for x in e]
    return gen.from_edges(d["n"], u, v, w)


# ----------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("k,r", [(3, 4), (5, 16), (8, 30), (4, 7)])
def test_ring_of_cliques_closed_form(k, r):
    """Clique partition of r cliques K_k in a ring: Q = L/(L+1) - 1/r, L = k(k-1)/2."""
    g = gen.ring_of_cliques(k, r)
    L = k * (k - 1) / 2
    memb = np.repeat(np.arange(r), k).astype(np.int32)
    assert abs(oracle.modularity(g, memb) - (L / (L + 1) - 1.0 / r)) < 1e-12


def test_two_disjoint_cliques_and_complete_graph():
    # two disjoint K5: each community holds half of all edge weight -> Q = 2*(1/2 - 1/4) = 1/2
    u, v = [], []
    for base in (0, 5):
        for a in range(5):
            for b in range(a + 1, 5):
                u.append(base + a)
                v.append(base + b)
    g = gen.from_edges(10, u, v)
    assert abs(oracle.modularity(g, np.array([0] * 5 + [1] * 5)) - 0.5) < 1e-15
    # K_n as one community: Q = 1 - 1 = 0
    kn = gen.gnp(9, 1.0, seed=1)
    assert abs(oracle.modularity(kn, np.zeros(9, np.int32))) < 1e-15
    # no edges: Q = 0 by the convention for m = 0
    empty = gen.from_edges(4, [], [])
    assert oracle.modularity(empty, np.arange(4)) == 0.0


def test_golden_two_triangles():
    d = _golden("two_triangles_bridge.json")
    g = _from_golden_edges(d)
    assert abs(oracle.modularity(g, np.array(d["optimal_partition"])) - d["optimal_q"]) < 1e-15
    assert abs(oracle.modularity(g, np.zeros(6, np.int32)) - d["single_community_q"]) < 1e-15
    q, best = oracle.brute_force(g)
    assert abs(q - d["optimal_q"]) < 1e-15
    assert ari(best, d["optimal_partition"]) == 1.0
    for mode in MODES:
        r = oracle.leiden(g, mode=mode)
        assert r.status == 0
        assert abs(r.modularity - d["optimal_q"]) < 1e-15


@pytest.mark.parametrize("gamma", [1.0, 0.5, 2.0])
@pytest.mark.parametrize("seed", range(6))
def test_modularity_matches_all_pairs_form(seed, gamma):
    """Community form of Eq. 1 equals the all-pairs form (self-loops included)."""
    g = random_graph_with_loops(14, 0.3, seed)
    rng = np.random.default_rng(seed)
    memb = rng.integers(0, 4, g.n).astype(np.int32)
    assert abs(oracle.modularity(g, memb, gamma) - q_dense(dense(g), memb, gamma)) < 1e-12


# ----------------------------------------------------------------- Eq. 2
def test_golden_delta_q():
    d = _golden("delta_q_star.json")
    g = _from_golden_edges(d)
    memb = np.array(d["membership"], np.int32)
    mv = d["move"]
    assert abs(oracle.delta_modularity(g, memb, mv["vertex"], mv["to"]) - d["expected_dq"]) < 1e-15


@pytest.mark.parametrize("gamma", [1.0, 0.7])
@pytest.mark.parametrize("seed", range(8))
def test_delta_modularity_against_recomputation(seed, gamma):
    """Eq. 2 equals Q(after) - Q(before) recomputed from scratch (dense form)."""
    g = random_graph_with_loops(12, 0.35, seed)
    A = dense(g)
    rng = np.random.default_rng(100 + seed)
    memb = rng.integers(0, 5, g.n).astype(np.int32)
    for _ in range(20):
        i = int(rng.integers(0, g.n))
        c = int(rng.integers(0, 5))
        if c == memb[i]:
            continue
        after = memb.copy()
        after[i] = c
        want = q_dense(A, after, gamma) - q_dense(A, memb, gamma)
        got = oracle.delta_modularity(g, memb, i, c, gamma)
        assert abs(got - want) < 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_delta_key_is_exact(seed):
    """The integer key difference equals 2m^2 * dQ exactly: 2*key = (2m)^2 dQ."""
    g = random_graph_with_loops(11, 0.4, seed, wmax=9)
    A = dense(g)
    rng = np.random.default_rng(200 + seed)
    memb = rng.integers(0, 4, g.n).astype(np.int32)
    base = q_times_4m2_exact(A, memb)
    for _ in range(20):
        i = int(rng.integers(0, g.n))
        c = int(rng.integers(0, 4))
        if c == memb[i]:
            continue
        after = memb.copy()
        after[i] = c
        assert 2 * oracle.delta_key(g, memb, i, c) == q_times_4m2_exact(A, after) - base


# ------------------------------------------------------------ brute force
def test_brute_force_enumerates_bell_numbers():
    """On a graph with no edges every partition scores 0 except through the
    enumeration count, so check the optimum on K_4 minus an edge instead and
    the restricted-growth enumeration on a planted 3-block graph."""
    g = gen.from_edges(4, [0, 0, 1, 1, 2], [1, 2, 2, 3, 3])  # K4 minus edge 0-3
    q, best = oracle.brute_force(g)
    # the best is a single community or two pairs; compare with the dense form
    assert abs(q - q_dense(dense(g), best)) < 1e-15
    # planted: three disjoint triangles -> optimum 3*(1/3 - 1/9) = 2/3
    u, v = [], []
    for b in range(3):
        for a, c in ((0, 1), (0, 2), (1, 2)):
            u.append(3 * b + a)
            v.append(3 * b + c)
    h = gen.from_edges(9, u, v)
    q, best = oracle.brute_force(h)
    assert abs(q - 2.0 / 3.0) < 1e-15
    assert ari(best, np.repeat(np.arange(3), 3)) == 1.0


@pytest.mark.parametrize("mode", MODES)
def test_oracle_never_beats_brute_force(mode):
    """Q_oracle <= Q_opt on seeded G(n, p) graphs with n <= 10 (a heuristic may fall short)."""
    gaps = []
    for seed in range(60):
        n = 6 + seed % 5
        g = gen.gnp(n, 0.45, seed=seed, wmax=3)
        if g.nnz == 0:
            continue
        q_opt, _ = oracle.brute_force(g)
        r = oracle.leiden(g, mode=mode)
        assert r.status == 0
        assert r.modularity <= q_opt + 1e-12
        assert abs(r.modularity - oracle.modularity(g, r.membership)) < 1e-15
        gaps.append(q_opt - r.modularity)
    assert np.median(gaps) < 0.02


@pytest.mark.parametrize("mode", MODES)
def test_oracle_reaches_optimum_on_designated_family(mode):
    """Equality with brute force on graphs with a clear optimum (n <= 12)."""
    fams = [gen.ring_of_cliques(3, 4),                       # ring of triangles (12 vertices)
            gen.from_edges(8, [0, 0, 0, 1, 1, 2, 4, 4, 4, 5, 5, 6, 3],
                           [1, 2, 3, 2, 3, 3, 5, 6, 7, 6, 7, 7, 4]),  # barbell: two K4 + bridge
            _from_golden_edges(_golden("two_triangles_bridge.json"))]
    for g in fams:
        q_opt, _ = oracle.brute_force(g)
        r = oracle.leiden(g, mode=mode)
        assert abs(r.modularity - q_opt) < 1e-12


# ---------------------------------------------------------- whole method
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,r", [(5, 16), (8, 30)])
def test_oracle_finds_the_cliques(mode, k, r):
    g = gen.ring_of_cliques(k, r)
    res = oracle.leiden(g, mode=mode)
    assert res.status == 0
    L = k * (k - 1) / 2
    assert abs(res.modularity - (L / (L + 1) - 1.0 / r)) < 1e-12
    assert np.array_equal(res.membership, np.repeat(np.arange(r), k))


@pytest.mark.parametrize("mode", MODES)
def test_special_cases(mode):
    # empty graph
    r = oracle.leiden(gen.from_edges(0, [], []), mode=mode)
    assert r.status == 0 and r.membership.size == 0 and r.modularity == 0.0
    # vertices without edges: singletons, Q = 0
    r = oracle.leiden(gen.from_edges(5, [], []), mode=mode)
    assert r.status == 0 and np.array_equal(r.membership, np.arange(5)) and r.modularity == 0.0
    # K_n: one community
    r = oracle.leiden(gen.gnp(8, 1.0, seed=3), mode=mode)
    assert np.array_equal(r.membership, np.zeros(8)) and abs(r.modularity) < 1e-15
    # isolated vertices stay alone next to a triangle
    g = gen.from_edges(5, [0, 0, 1], [1, 2, 2])
    r = oracle.leiden(g, mode=mode)
    assert np.array_equal(r.membership, [0, 0, 0, 1, 2])


def test_sync_mode_validation():
    g = gen.ring_of_cliques(4, 4)
    w = g.weights.copy()
    w[0] = w[1] = 0.5
    bad = gen.CSR(g.n, g.offsets, g.indices, w)
    assert oracle.leiden(bad, mode=oracle.SYNC).status == oracle.ERR_UNSUPPORTED
    assert oracle.leiden(g, mode=oracle.SYNC, resolution=0.5).status == oracle.ERR_UNSUPPORTED
    # S1: 2m < 2^53 (48 entries of weight 2^48 give 2m = 1.5 * 2^53)
    big = gen.CSR(g.n, g.offsets, g.indices, np.full_like(g.weights, 2.0 ** 48))
    assert g.nnz * 2.0 ** 48 >= 2.0 ** 53
    assert oracle.leiden(big, mode=oracle.SYNC).status == oracle.ERR_OVERFLOW
    idx = g.indices.copy()
    idx[3] = g.n
    assert oracle.leiden(gen.CSR(g.n, g.offsets, idx, g.weights)).status == oracle.ERR_INVALID
    assert oracle.leiden(g, mode=oracle.SEQ, resolution=0.5).status == 0


@pytest.mark.parametrize("shift", [26, 32])
def test_sync_keys_exact_beyond_32_bits(shift):
    """S1/S4: scaling every integer weight by 2^shift scales each key by
    2^(2 shift) and a sweep's gain sum and (2m)^2 alike, so every decision and
    every tolerance test is the same: the run equals the unscaled one pass for
    pass, although 2m (~2^44 and ~2^50) and the keys (~2^90 and ~2^102) are
    far beyond 64-bit products."""
    g = gen.road(60)
    scaled = gen.CSR(g.n, g.offsets, g.indices, (g.weights.astype(np.float64) * 2.0 ** shift).astype(np.float32))
    assert float(scaled.weights.astype(np.float64).sum()) >= 2.0 ** 40
    a = oracle.leiden(g, mode=oracle.SYNC, trace=True)
    b = oracle.leiden(scaled, mode=oracle.SYNC, trace=True)
    assert a.status == 0 and b.status == 0
    assert np.array_equal(a.membership, b.membership)
    assert a.passes == b.passes
    assert a.modularity == b.modularity
    assert sorted(a.trace) == sorted(b.trace)
    for p in a.trace:
        assert sorted(a.trace[p]) == sorted(b.trace[p])
        for w, x in a.trace[p].items():
            y = b.trace[p][w]
            assert np.array_equal(x * 2.0 ** shift if w == oracle.T_AGG_W else x, y), (p, w)


def test_planted_partition_recovered():
    """SBM workload: the planted 50 blocks are found (ARI >= 0.95) and Q is
    close to the planted partition's modularity (~9.95/14.85 - 1/50)."""
    g, blocks = gen.sbm(10_000, 50, 0.05, 0.0005, seed=1, return_blocks=True)
    q_planted = oracle.modularity(g, blocks)
    assert abs(q_planted - (9.95 / 14.85 - 1 / 50)) < 0.01
    for mode in MODES:
        r = oracle.leiden(g, mode=mode)
        assert r.status == 0
        assert ari(r.membership, blocks) >= 0.95
        assert r.modularity >= q_planted - 0.005


# ------------------------------------------------------------- Algorithm 5
def test_disconnected_counter():
    g = gen.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])  # two paths 0-1-2 and 3-4-5
    assert oracle.disconnected(g, np.array([0, 0, 0, 3, 3, 3]))[0] == 0
    k, flags = oracle.disconnected(g, np.array([0, 0, 0, 0, 3, 3]))  # vertex 3 cut off from 0..2
    assert k == 1 and flags[0] == 1 and flags[3] == 0
    assert oracle.disconnected(g, np.array([0, 1, 0, 3, 4, 3]))[0] == 2


@pytest.mark.parametrize("seed", range(6))
def test_disconnected_counter_against_scipy(seed):
    """Algorithm 5's count on random labellings (few labels, so that most
    communities span several pieces; singletons; one label for all) equals
    the count from scipy's connected components of the intra-community
    subgraph, and a community is flagged exactly when it is counted."""
    rng = np.random.default_rng(seed)
    g = gen.gnp(400, 0.006 + 0.002 * seed, seed=seed + 11, wmax=3)
    for labels in (rng.integers(0, 5 + 10 * seed, g.n), np.arange(g.n), np.zeros(g.n, dtype=np.int64),
                   rng.integers(0, g.n, g.n)):
        m = np.asarray(labels, dtype=np.int32)
        k, flags = oracle.disconnected(g, m)
        assert k == _components_inside(g, m)
        assert int(np.count_nonzero(flags)) == k


@pytest.mark.parametrize("mode", MODES)
def test_every_community_connected(mode):
    graphs = [gen.sbm_workload(), gen.road(150), gen.rmat(12, 16), gen.gnp(300, 0.02, seed=5, wmax=4)]
    for g in graphs:
        r = oracle.leiden(g, mode=mode, trace=True)
        assert r.status == 0
        assert oracle.disconnected(g, r.membership)[0] == 0
        # refinement invariant (pass 0): every refined community lies inside one
        # local-moving community and is connected
        t0 = r.trace[0]
        bound, refined = t0[oracle.T_MOVE], t0[oracle.T_REFINE]
        for c in np.unique(refined):
            assert np.unique(bound[refined == c]).size == 1
        assert oracle.disconnected(g, refined)[0] == 0


# ------------------------------------------------------------- Algorithm 4
def test_golden_aggregate():
    d = _golden("path4_aggregate.json")
    g = _from_golden_edges(d)
    off, deg, idx, w = oracle.aggregate(g.n, g.offsets, np.diff(g.offsets), g.indices, g.weights,
                                        np.array(d["membership"]), 2)
    assert off.tolist() == d["expected_offsets"]
    assert deg.tolist() == d["expected_degree"]
    for c, row in enumerate(d["expected_rows"]):
        got = [[int(idx[e]), float(w[e])] for e in range(off[c], off[c] + deg[c])]
        assert got == row
    K = [float(w[off[c]:off[c] + deg[c]].sum()) for c in range(2)]
    assert K == d["expected_K"]


@pytest.mark.parametrize("seed", range(5))
def test_aggregation_invariants(seed):
    g = random_graph_with_loops(40, 0.12, seed, wmax=7)
    rng = np.random.default_rng(seed)
    ncomm = 7
    memb = rng.permutation(np.arange(g.n) % ncomm).astype(np.int32)
    deg = np.diff(g.offsets).astype(np.int32)
    off2, deg2, idx2, w2 = oracle.aggregate(g.n, g.offsets, deg, g.indices, g.weights, memb, ncomm)
    # total weight (2m) preserved; K'' = sum of member K
    real = np.concatenate([np.arange(off2[c], off2[c] + deg2[c]) for c in range(ncomm)])
    assert w2[real].sum() == g.weights.astype(np.float64).sum()
    K = np.bincount(np.repeat(np.arange(g.n), deg), weights=g.weights.astype(np.float64), minlength=g.n)
    K2 = np.array([w2[off2[c]:off2[c] + deg2[c]].sum() for c in range(ncomm)])
    assert np.array_equal(K2, np.bincount(memb, weights=K, minlength=ncomm))
    # row capacity = communityTotalDegree; rows sorted, unique, symmetric weights
    assert np.array_equal(np.diff(off2), np.bincount(memb, weights=deg, minlength=ncomm).astype(np.int64))
    W = np.zeros((ncomm, ncomm))
    for c in range(ncomm):
        row = idx2[off2[c]:off2[c] + deg2[c]]
        assert np.all(np.diff(row) > 0)
        W[c, row] = w2[off2[c]:off2[c] + deg2[c]]
    assert np.array_equal(W, W.T)
    # closed form of Algorithm 4: W = S^T A S with S the n x |Gamma| indicator
    # of the membership (integer weights, so the fp64 sums are exact)
    S = np.zeros((g.n, ncomm))
    S[np.arange(g.n), memb] = 1.0
    assert np.array_equal(W, S.T @ dense(g) @ S)
    # Q(G'', L) == Q(G, L o memb) for any partition L of the super-vertices
    for _ in range(5):
        L = rng.integers(0, 3, ncomm).astype(np.int32)
        q2 = oracle.modularity_holey(ncomm, off2, deg2, idx2, w2, L)
        assert abs(q2 - oracle.modularity(g, L[memb])) < 1e-12
    # community-vertex CSR is a permutation grouped by label
    coff, members = oracle.community_vertices(memb, ncomm)
    assert np.array_equal(np.sort(members), np.arange(g.n))
    for c in range(ncomm):
        assert np.all(memb[members[coff[c]:coff[c + 1]]] == c)


# ---------------------------------------------------- local optimality
@pytest.mark.parametrize("seed", range(4))
def test_local_moving_reaches_local_optimum(seed):
    """SEQ, tau = 0, no pruning, one pass: once a sweep moves nobody no single
    move has dQ > 0 (checked against the dense all-pairs form of Eq. 1)."""
    g = gen.gnp(60, 0.08, seed=seed, wmax=3)
    r = oracle.leiden(g, mode=oracle.SEQ, tolerance=0.0, max_passes=1, max_iterations=10_000,
                      flags=oracle.NO_PRUNE, trace=True)
    assert r.trace[0][oracle.T_COUNTS][1] < 10_000
    memb = r.trace[0][oracle.T_MOVE]
    A = dense(g)
    q0 = q_dense(A, memb)
    for i in range(g.n):
        for c in set(memb[g.indices[g.offsets[i]:g.offsets[i + 1]]]) - {memb[i]}:
            after = memb.copy()
            after[i] = c
            assert q_dense(A, after) - q0 <= 1e-12


# ----------------------------------------------------------- schedule (S0)
def test_splitmix64_reference_vectors():
    """Published SplitMix64 outputs (Vigna's reference splitmix64.c)."""
    lib = oracle._lib()
    lib.og_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.og_splitmix64_at.restype = ctypes.c_uint64
    assert [lib.og_splitmix64_at(1234567, i) for i in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]
    assert lib.og_splitmix64_at(0, 0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("L,B", [(32, 16), (4, 3), (1, 1)])
def test_schedule_properties(L, B):
    g = gen.road(60)
    deg = np.diff(g.offsets).astype(np.int32)
    step, used = oracle.schedule(g.n, g.offsets, deg, g.indices, 7, L, B)
    assert used == step.max() + 1 and used <= L - 1 + B
    rows = np.repeat(np.arange(g.n), deg)
    same = step[rows] == step[g.indices]
    lower = step[rows] < L - 1
    # below the cap no edge joins two vertices of the same step
    assert not np.any(same & lower & (rows != g.indices))
    # longest-path property: a vertex in layer k >= 1 (below the cap) has a neighbour in layer k-1
    for v in np.nonzero((step > 0) & (step < L - 1))[0][:500]:
        nb = g.indices[g.offsets[v]:g.offsets[v + 1]]
        assert np.any(step[nb] == step[v] - 1)


def test_ties_go_to_the_lowest_community_id():
    """Path 1-0-2: vertex 0 sees communities 1 and 2 with equal dQ (Eq. 2 is
    symmetric in them) and must take community 1 (reading R2); vertex 2 then
    joins community 1 as well."""
    g = gen.from_edges(3, [0, 0], [1, 2])
    r = oracle.leiden(g, mode=oracle.SEQ, max_passes=1, trace=True)
    assert r.trace[0][oracle.T_MOVE].tolist() == [1, 1, 1]


# ------------------------------------- variants: refine-based labels, Louvain
VARIANTS = (oracle.REFINE_LABELS, oracle.LOUVAIN)


def _components_inside(g, membership):
    """Disconnected communities counted with scipy's connected components on
    the subgraph that keeps only intra-community edges (independent of the
    oracle's own BFS)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    keep = membership[rows] == membership[g.indices]
    a = csr_matrix((np.ones(int(keep.sum())), (rows[keep], g.indices[keep])), shape=(g.n, g.n))
    _, comp = connected_components(a, directed=False)
    bad = 0
    for c in np.unique(membership):
        bad += np.unique(comp[membership == c]).size > 1
    return bad


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("flags", VARIANTS)
@pytest.mark.parametrize("k,r", [(5, 16), (8, 30)])
def test_variants_find_the_cliques(mode, flags, k, r):
    """Both variants keep the ring-of-cliques closed form of Eq. 1."""
    res = oracle.leiden(gen.ring_of_cliques(k, r), mode=mode, flags=flags)
    assert res.status == 0
    L = k * (k - 1) / 2
    assert abs(res.modularity - (L / (L + 1) - 1.0 / r)) < 1e-12
    assert np.array_equal(res.membership, np.repeat(np.arange(r), k))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("flags", VARIANTS)
def test_variants_against_brute_force(mode, flags):
    """Q <= Q_opt on seeded G(n, p) graphs, equality on the designated family."""
    for seed in range(40):
        g = gen.gnp(6 + seed % 5, 0.45, seed=seed, wmax=3)
        if g.nnz == 0:
            continue
        q_opt, _ = oracle.brute_force(g)
        r = oracle.leiden(g, mode=mode, flags=flags)
        assert r.status == 0 and r.modularity <= q_opt + 1e-12
    for g in (gen.ring_of_cliques(3, 4), _from_golden_edges(_golden("two_triangles_bridge.json"))):
        q_opt, _ = oracle.brute_force(g)
        assert abs(oracle.leiden(g, mode=mode, flags=flags).modularity - q_opt) < 1e-12


@pytest.mark.parametrize("mode", MODES)
def test_louvain_first_pass_is_the_local_moving_phase(mode):
    """One Louvain pass is Algorithm 2 alone: its partition equals the
    local-moving partition of the Leiden method's first pass."""
    for g in (gen.sbm(2000, 10, 0.05, 0.002, seed=11), gen.road(40), gen.rmat(10, 8, seed=2)):
        lv = oracle.leiden(g, mode=mode, flags=oracle.LOUVAIN, max_passes=1)
        ld = oracle.leiden(g, mode=mode, trace=True)
        moved = ld.trace[0][oracle.T_MOVE]
        assert ari(lv.membership, moved) == 1.0
        # and it stops with the local-moving count as |Gamma| (no refinement sweeps)
        lt = oracle.leiden(g, mode=mode, flags=oracle.LOUVAIN, trace=True).trace[0]
        assert lt[oracle.T_COUNTS][2] == 0
        assert lt[oracle.T_COUNTS][3] == np.unique(lt[oracle.T_MOVE]).size


def test_louvain_can_leave_a_community_disconnected():
    """The shortcoming the refinement phase removes (Sections 3.3-3.4): on this
    graph the Louvain variant returns an internally disconnected community,
    while the Leiden method (either label rule) returns connected ones."""
    g = gen.gnp(18, 0.25, seed=2108, wmax=3)
    lv = oracle.leiden(g, mode=oracle.SEQ, flags=oracle.LOUVAIN)
    assert _components_inside(g, lv.membership) >= 1
    assert oracle.disconnected(g, lv.membership)[0] == _components_inside(g, lv.membership)
    for flags in (0, oracle.REFINE_LABELS):
        r = oracle.leiden(g, mode=oracle.SEQ, flags=flags)
        assert _components_inside(g, r.membership) == 0


@pytest.mark.parametrize("mode", MODES)
def test_refine_labels_start_every_pass_from_singletons(mode):
    g = gen.sbm(3000, 12, 0.04, 0.002, seed=17)
    r = oracle.leiden(g, mode=mode, flags=oracle.REFINE_LABELS, trace=True)
    assert r.passes >= 2
    for lp in range(1, r.passes):
        init = r.trace[lp][oracle.T_INIT_LABELS]
        assert np.array_equal(init, np.arange(init.size))
    # the default (move-based) rule does not: some super-vertices share a label
    d = oracle.leiden(g, mode=mode, trace=True)
    assert np.unique(d.trace[1][oracle.T_INIT_LABELS]).size < d.trace[1][oracle.T_INIT_LABELS].size
    for flags in (0, oracle.REFINE_LABELS):
        m = oracle.leiden(g, mode=mode, flags=flags).membership
        assert _components_inside(g, m) == 0


def _splitmix64_at(state, i):
    """SplitMix64 output number i+1 from state (Steele, Lea & Flood 2014),
    in Python integers (independent of the oracle's C)."""
    M = (1 << 64) - 1
    z = (state + (i + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


@pytest.mark.parametrize("name", ["rmat", "road"])
def test_schedule_follows_degree_then_hash_priority(name):
    """S0: on every edge below the cap the end of higher priority (longer
    row, then larger hash, then smaller id) takes the earlier step."""
    g = gen.rmat(10, 16, seed=4) if name == "rmat" else gen.road(40)
    deg = np.diff(g.offsets).astype(np.int32)
    state = 11
    L = 1000
    step, used = oracle.schedule(g.n, g.offsets, deg, g.indices, state, L, 4)
    prio = [(int(deg[v]) << 32) | (_splitmix64_at(state, v) >> 32) for v in range(g.n)]
    rows = np.repeat(np.arange(g.n), deg)
    checked = 0
    for u, v in zip(rows.tolist(), g.indices.tolist()):
        if u == v or step[u] >= L - 1 or step[v] >= L - 1:
            continue
        first = u if (prio[u] > prio[v] or (prio[u] == prio[v] and u < v)) else v
        other = v if first == u else u
        assert step[first] < step[other], (u, v)
        checked += 1
    assert checked > 0
    # vertices of the largest degree have no preceding neighbour: step 0
    assert step[np.argmax(deg)] == 0


def test_rmat_sync_schedule_keeps_sequential_quality():
    """The layered schedule lands within 0.005 of the sequential sweep on a
    heavy-tailed graph, where a hashed order without the degree key falls
    well short (the refinement of the last pass fragments large
    communities)."""
    g = gen.rmat(16, 56, 0.57, 0.19, 0.19, seed=3)
    seq = oracle.leiden(g, mode=oracle.SEQ)
    syn = oracle.leiden(g, mode=oracle.SYNC)
    assert syn.modularity >= seq.modularity - 0.005, (syn.modularity, seq.modularity)
    assert oracle.disconnected(g, syn.membership)[0] == 0


def heavy_tailed(g):
    """S0's graph property: the largest degree exceeds 64 times the mean
    degree nnz/n."""
    return int(np.diff(g.offsets).max()) * g.n > 64 * g.nnz


def test_schedule_layers_by_graph():
    """S0: schedule_layers = 0 takes L = 1000 for a heavy-tailed input
    (largest degree above 64 times the mean degree), else L = 32. A star's
    hub is heavy-tailed at any size; a block model, a lattice and a small
    R-MAT graph are not."""
    light = gen.sbm(3000, 12, 0.04, 0.002, seed=4)
    heavy = gen.rmat(14, 56, 0.57, 0.19, 0.19, seed=3)
    star = gen.from_edges(200, np.zeros(199, np.int64), np.arange(1, 200))
    for g, h in ((light, False), (heavy, True), (star, True), (gen.road(50), False),
                 (gen.rmat(12, 16), False)):
        assert heavy_tailed(g) == h
    for g, L in ((light, 32), (heavy, 1000), (star, 1000)):
        auto = oracle.leiden(g, mode=oracle.SYNC, trace=True)
        fixed = oracle.leiden(g, mode=oracle.SYNC, schedule_layers=L, trace=True)
        assert np.array_equal(auto.membership, fixed.membership)
        for p in fixed.trace:
            assert np.array_equal(auto.trace[p][oracle.T_MOVE], fixed.trace[p][oracle.T_MOVE])


@pytest.mark.parametrize("mode", MODES)
def test_vertices_without_edges_do_not_stop_the_passes(mode):
    """R4: vertices without edges are left out of the aggregation-tolerance
    ratio, so adding any number of them changes nothing else."""
    g = gen.sbm(2000, 10, 0.05, 0.002, seed=11)
    z = 6000
    g2 = gen.CSR(g.n + z, np.concatenate([g.offsets, np.full(z, g.offsets[-1], dtype=g.offsets.dtype)]),
                 g.indices, g.weights)
    r = oracle.leiden(g, mode=mode)
    r2 = oracle.leiden(g2, mode=mode)
    assert r.passes >= 2
    assert r2.passes == r.passes
    assert np.array_equal(r2.membership[:g.n], r.membership)
    assert np.array_equal(r2.membership[g.n:], np.arange(z) + r.membership.max() + 1)
    # the ratio without the rule would be above the tolerance after the first pass
    t = oracle.leiden(g2, mode=mode, trace=True).trace[0][oracle.T_COUNTS]
    assert (t[3]) / t[0] > 0.8 and (t[3] - z) / (t[0] - z) <= 0.8


# ------------------------------------------- V3: randomized refinement
def test_random_refinement_draws_in_proportion_to_the_gain():
    """V3: the first isolated vertex of the refinement (vertex 0, with every
    vertex still alone) joins the community of a neighbour j inside its
    local-moving community with probability gain_j / (sum of the positive
    gains), the gains from Eq. 2 on the singleton partition."""
    u = [0, 0, 0, 0, 1, 2, 3, 4]
    v = [1, 2, 3, 4, 2, 3, 4, 1]
    w = [1.0, 2.0, 3.0, 4.0, 1.0, 1.0, 1.0, 1.0]
    g = gen.from_edges(5, u, v, w)
    bound = oracle.leiden(g, mode=oracle.SEQ, max_passes=1, trace=True).trace[0][oracle.T_MOVE]
    cands = [j for j in range(1, 5) if bound[j] == bound[0]]
    single = np.arange(5)
    gains = np.array([oracle.delta_modularity(g, single, 0, j) for j in cands])
    pos = np.clip(gains, 0, None)
    assert len(cands) >= 2 and np.count_nonzero(pos) >= 2
    expect = pos / pos.sum()
    seeds = 600
    counts = np.zeros(len(cands))
    for s in range(seeds):
        t = oracle.leiden(g, mode=oracle.SEQ, flags=oracle.RANDOM_REFINE, seed=s, max_passes=1, trace=True).trace[0]
        assert np.array_equal(t[oracle.T_MOVE], bound)  # local-moving draws nothing
        counts[cands.index(int(t[oracle.T_REFINE][0]))] += 1
    freq = counts / seeds
    sigma = np.sqrt(expect * (1 - expect) / seeds)
    assert np.all(np.abs(freq - expect) <= 4 * sigma + 1e-12), (freq, expect)
    # the greedy rule takes the largest gain every time
    r = oracle.leiden(g, mode=oracle.SEQ, max_passes=1, trace=True)
    assert int(r.trace[0][oracle.T_REFINE][0]) == cands[int(np.argmax(gains))]


def test_random_refinement_keeps_the_leiden_guarantees():
    for g in (gen.sbm(3000, 12, 0.04, 0.002, seed=4), gen.road(100), gen.rmat(12, 16, seed=2)):
        r = oracle.leiden(g, mode=oracle.SEQ, flags=oracle.RANDOM_REFINE, seed=5, trace=True)
        assert r.status == 0
        assert _components_inside(g, r.membership) == 0
        t0 = r.trace[0]
        for c in np.unique(t0[oracle.T_REFINE]):
            assert np.unique(t0[oracle.T_MOVE][t0[oracle.T_REFINE] == c]).size == 1
    res = oracle.leiden(gen.ring_of_cliques(5, 16), mode=oracle.SEQ, flags=oracle.RANDOM_REFINE, seed=3)
    assert np.array_equal(res.membership, np.repeat(np.arange(16), 5))
    # SYNC mode has no randomized variant
    assert oracle.leiden(gen.road(10), mode=oracle.SYNC, flags=oracle.RANDOM_REFINE).status == oracle.ERR_UNSUPPORTED


def test_golden_edges_to_csr():
    """The edge-list to CSR definition on a hand-derived example."""
    d = _golden("edges_to_csr.json")
    e = np.array(d["edges"])
    u, v, w = e[:, 0].astype(int), e[:, 1].astype(int), e[:, 2]
    for name, kw in (("sum", {}), ("max", {"combine": "max"}), ("sum_drop_self", {"drop_self_loops": True})):
        off, idx, ww = oracle.csr_from_edges(d["n"], u, v, w, **kw)
        assert off.tolist() == d[name]["offsets"], name
        assert idx.tolist() == d[name]["indices"], name
        assert ww.tolist() == d[name]["weights"], name
    # a generated symmetric CSR comes back from its edges (u <= v) unchanged
    g = gen.gnp(60, 0.1, seed=3, wmax=4)
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    up = rows <= g.indices
    off, idx, ww = oracle.csr_from_edges(g.n, rows[up], g.indices[up], g.weights[up])
    assert np.array_equal(off, g.offsets) and np.array_equal(idx, g.indices) and np.array_equal(ww, g.weights)


# ---------------------------------------------------- pass-loop controls (Algorithm 1)
def _li(r):
    """Local-moving sweeps of every pass (the trace's counts: n, l_i, l_j, |Gamma|)."""
    return [int(r.trace[p][oracle.T_COUNTS][1]) for p in sorted(r.trace)]


def test_threshold_scaling_divides_tau_between_passes():
    """tau is divided by the drop factor after each pass: a factor below 1 makes
    tau grow past any sweep's gain, so every pass after the first stops after
    one sweep; kept constant or shrinking, the second pass sweeps several times.
    The first pass, on tau0 alone, is the same in every run."""
    g = gen.gnp(300, 0.03, seed=1, wmax=3)
    grow = oracle.leiden(g, mode=oracle.SEQ, tolerance=1e-3, tolerance_drop=1e-6, trace=True)
    same = oracle.leiden(g, mode=oracle.SEQ, tolerance=1e-3, tolerance_drop=1.0, trace=True)
    shrink = oracle.leiden(g, mode=oracle.SEQ, tolerance=1e-3, tolerance_drop=1e6, trace=True)
    assert grow.passes >= 2 and _li(grow)[0] > 1 and all(x == 1 for x in _li(grow)[1:])
    assert _li(same)[1] > 1 and _li(shrink)[1] > 1
    for r in (same, shrink):
        assert np.array_equal(r.trace[0][oracle.T_MOVE], grow.trace[0][oracle.T_MOVE])


def test_huge_tolerance_and_one_iteration_stop_after_one_sweep():
    """A sweep's total gain never exceeds a tau of 1e9, and max_iterations = 1
    allows one sweep: either way l_i = 1 in every pass, and the second also
    caps the refinement at one sweep."""
    g = gen.gnp(300, 0.03, seed=1, wmax=3)
    huge = oracle.leiden(g, mode=oracle.SEQ, tolerance=1e9, trace=True)
    assert all(x == 1 for x in _li(huge))
    one = oracle.leiden(g, mode=oracle.SEQ, max_iterations=1, trace=True)
    assert all(x == 1 for x in _li(one))
    assert all(int(one.trace[p][oracle.T_COUNTS][2]) <= 1 for p in one.trace)


def test_aggregation_tolerance_zero_stops_after_the_first_pass():
    """With tau_agg = 0 any non-empty refined partition exceeds the ratio, so
    the result is pass 0's refined partition in canonical labels."""
    g = gen.gnp(300, 0.03, seed=1, wmax=3)
    r = oracle.leiden(g, mode=oracle.SEQ, aggregation_tolerance=0.0, trace=True)
    assert r.passes == 1
    ref = r.trace[0][oracle.T_REFINE]
    _, canon = np.unique(ref, return_index=True)
    first = {c: k for k, c in enumerate(ref[np.sort(canon)])}
    assert np.array_equal(r.membership, np.array([first[c] for c in ref], dtype=np.int32))


def test_convergence_stop_without_the_ratio():
    """Two disjoint triangles: pass 0 finds them; in pass 1 nobody moves and
    the refinement keeps both super-vertices, so the loop stops there (R5)
    even with tau_agg = 1, where the ratio test never fires."""
    t = gen.from_edges(6, np.array([0, 1, 2, 3, 4, 5]), np.array([1, 2, 0, 4, 5, 3]))
    r = oracle.leiden(t, mode=oracle.SEQ, aggregation_tolerance=1.0, max_passes=10, trace=True)
    assert r.passes == 2 and _li(r) == [2, 1]
    assert r.membership.tolist() == [0, 0, 0, 1, 1, 1] and r.modularity == 0.5


@pytest.mark.parametrize("gamma", [1.0, 0.6])
def test_zero_passes_leave_singletons(gamma):
    """max_passes = 0 runs no pass: every vertex alone, whose Eq. 1 score is
    trace(A)/2m - gamma * sum_i (K_i / 2m)^2 (self-loops included)."""
    g = random_graph_with_loops(40, 0.12, 3, wmax=5)
    r = oracle.leiden(g, mode=oracle.SEQ, max_passes=0, resolution=gamma)
    assert r.passes == 0
    assert np.array_equal(r.membership, np.arange(g.n))
    A = dense(g)
    two_m = A.sum()
    q = np.trace(A) / two_m - gamma * np.sum((A.sum(axis=1) / two_m) ** 2)
    assert abs(r.modularity - q) < 1e-12
