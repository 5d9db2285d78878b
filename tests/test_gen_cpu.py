"""The seeded input recipes on CPU: the sizes the workloads are quoted with,
the structure each recipe promises, and determinism. The sizes were first
measured on an aarch64 host, so matching them here (x86_64) also shows the
generators give the same graphs on both architectures."""
import numpy as np
import pytest

import gen


def _edges(g):
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    return src, g.indices.astype(np.int64), g.weights


def _symmetric(g):
    """Every entry (i, j, w) has its mirror (j, i, w), and rows hold no duplicate."""
    s, d, w = _edges(g)
    fwd = np.lexsort((w, d, s))
    bwd = np.lexsort((w, s, d))
    if not (np.array_equal(s[fwd], d[bwd]) and np.array_equal(d[fwd], s[bwd]) and np.array_equal(w[fwd], w[bwd])):
        return False
    key = s * g.n + d
    return len(np.unique(key)) == len(key)


def test_road_workload_size():
    """5000 x 5000 lattice, seed 2: 25M vertices and 90,981,444 entries. The
    1% diagonal shortcuts are an exact count (redrawn on duplicates), so the
    kept lattice edges are the rest: about 90% of the 2 s (s - 1)."""
    g = gen.road_workload()
    assert g.n == 25_000_000 and g.nnz == 90_981_444
    lattice = 2 * 5000 * 4999
    kept = g.nnz // 2 - lattice // 100
    assert abs(kept / lattice - 0.9) < 5 * np.sqrt(0.09 / lattice)


def test_road_structure():
    side = 300
    g = gen.road(side, seed=2)
    assert _symmetric(g)
    s, d, w = _edges(g)
    assert np.all(s != d)
    dx = np.abs(s % side - d % side)
    dy = np.abs(s // side - d // side)
    assert np.all((dx <= 1) & (dy <= 1))
    diag = np.sum((dx == 1) & (dy == 1)) // 2
    assert diag == round(0.01 * 2 * side * (side - 1))
    assert np.all(w == np.round(w)) and w.min() >= 1 and w.max() <= 10
    assert set(np.unique(w).tolist()) == set(range(1, 11))


def test_sbm_workload_size_and_blocks():
    """10,000 vertices in 50 blocks of 200, p_in 0.05, p_out 0.0005, seed 1:
    149,260 entries; the intra- and inter-block densities sit within five
    standard deviations of p_in and p_out."""
    g = gen.sbm_workload()
    assert g.n == 10_000 and g.nnz == 149_260
    g2, blk = gen.sbm(10_000, 50, 0.05, 0.0005, seed=1, return_blocks=True)
    assert np.array_equal(g2.indices, g.indices) and np.array_equal(g2.offsets, g.offsets)
    assert np.array_equal(np.bincount(blk), np.full(50, 200))
    assert _symmetric(g)
    s, d, w = _edges(g)
    assert np.all(s != d) and np.all(w == 1.0)
    intra = np.sum(blk[s] == blk[d]) // 2
    pairs_in = 50 * 200 * 199 // 2
    pairs_out = 10_000 * 9_999 // 2 - pairs_in
    for count, pairs, p in ((intra, pairs_in, 0.05), (g.nnz // 2 - intra, pairs_out, 0.0005)):
        assert abs(count - p * pairs) < 5 * np.sqrt(pairs * p * (1 - p))


def test_rmat_structure():
    """Symmetrised, deduplicated, no self-loops, unit weights, heavy-tailed."""
    g = gen.rmat(12, 16, seed=3)
    assert g.n == 4096
    assert _symmetric(g)
    s, d, w = _edges(g)
    assert np.all(s != d) and np.all(w == 1.0)
    deg = np.diff(g.offsets)
    assert deg.max() > 20 * deg.mean()


def test_sbm_batch_recipe():
    """The batch's per-graph parameters follow their stated formulas, the
    4096-graph batch holds 61,102,249 vertices, and graph g of a batch is the
    SBM recipe with its own parameters and seed (4 << 32) + g."""
    p = gen.sbm_batch_params(4096, 4)
    n, b, d = p["n"], p["blocks"], p["mean_degree"]
    assert int(n.sum()) == 61_102_249
    assert n.min() >= 100 and n.max() <= 100_000
    assert b.min() >= 2 and np.all(b <= np.maximum(n // 2, 1)) and b.max() <= 64
    assert d.min() >= 8 and d.max() <= 32
    s = n / b
    assert np.allclose(p["p_in"], np.minimum(1.0, d / ((s - 1) + 0.02 * (n - s))), rtol=1e-12)
    assert np.allclose(p["p_out"], 0.02 * p["p_in"], rtol=1e-12)
    assert np.array_equal(p["seeds"], (np.uint64(4) << np.uint64(32)) + np.arange(4096, dtype=np.uint64))
    small = gen.sbm_batch(6, seed=4, nmin=50, nmax=400)
    q = gen.sbm_batch_params(6, 4, nmin=50, nmax=400)
    for k in range(6):
        ref = gen.sbm(int(q["n"][k]), int(q["blocks"][k]), float(q["p_in"][k]), float(q["p_out"][k]),
                      int(q["seeds"][k]))
        got = small.graph(k)
        assert got.n == ref.n
        assert np.array_equal(got.offsets, ref.offsets) and np.array_equal(got.indices, ref.indices)


@pytest.mark.parametrize("make", [lambda s: gen.road(80, seed=s), lambda s: gen.rmat(10, 8, seed=s),
                                  lambda s: gen.sbm(500, 5, 0.1, 0.01, seed=s), lambda s: gen.gnp(300, 0.02, seed=s)])
def test_seeded_determinism(make):
    a, b, c = make(7), make(7), make(8)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.weights, b.weights)
    assert not (len(a.indices) == len(c.indices) and np.array_equal(a.indices, c.indices))
