"""GPU tests of the edge-list to CSR step (leiden_csr_from_edges): the
symmetric CSR must equal the oracle's definition entry for entry (offsets,
targets, weights), on edge lists with duplicates in both directions,
self-loops, vertices without edges and empty input, from device and host
memory; invalid endpoints and short capacities are refused."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2312_13936_gb300 as lg

pytestmark = pytest.mark.gpu


def random_edges(n, m, seed, wmax=5):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, m).astype(np.int32)
    v = rng.integers(0, n, m).astype(np.int32)
    # repeat some edges, reversed
    k = m // 5
    if k:
        u[m - k:], v[m - k:] = v[:k], u[:k]
    w = rng.integers(1, wmax + 1, m).astype(np.float32)
    return u, v, w


def gpu_csr(n, u, v, w, **kw):
    cu = torch.from_numpy(u).cuda()
    cv = torch.from_numpy(v).cuda()
    cw = torch.from_numpy(w).cuda() if w is not None else None
    off, idx, ww = lg.csr_from_edges(n, cu, cv, cw, **kw)
    torch.cuda.synchronize()
    return off.cpu().numpy(), idx.cpu().numpy(), ww.cpu().numpy()


@pytest.mark.parametrize("n,m,seed", [(10, 40, 1), (1000, 5000, 2), (300_000, 2_000_000, 3), (70_000, 1, 4)])
@pytest.mark.parametrize("kw", [{}, {"combine": "max"}, {"drop_self_loops": True}])
def test_edges_to_csr_matches_definition(n, m, seed, kw):
    u, v, w = random_edges(n, m, seed)
    got = gpu_csr(n, u, v, w, **kw)
    ref = oracle.csr_from_edges(n, u, v, w, **kw)
    for a, b, what in zip(got, ref, ("offsets", "indices", "weights")):
        assert np.array_equal(a, b), what


def test_edges_to_csr_unit_weights_and_round_trip():
    g = gen.rmat(12, 16, seed=2)
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets)).astype(np.int32)
    up = rows <= g.indices
    off, idx, ww = gpu_csr(g.n, rows[up], g.indices[up], None)
    assert np.array_equal(off, g.offsets) and np.array_equal(idx, g.indices) and np.array_equal(ww, g.weights)
    # the result runs through leiden_create unchanged
    h = lg.Leiden(off, idx, ww, validate=True)
    h.close()


def test_edges_to_csr_edge_cases_and_errors():
    # no edges: every row empty
    off, idx, ww = gpu_csr(7, np.zeros(0, np.int32), np.zeros(0, np.int32), None)
    assert np.array_equal(off, np.zeros(8, np.int64)) and idx.size == 0
    # only self-loops, dropped: empty rows too
    off, idx, ww = gpu_csr(3, np.array([0, 2], np.int32), np.array([0, 2], np.int32), None, drop_self_loops=True)
    assert np.array_equal(off, np.zeros(4, np.int64))
    # host memory in, host memory out
    u, v, w = random_edges(50, 200, 9)
    off = np.zeros(51, np.int64)
    idx = np.zeros(400, np.int32)
    ww = np.zeros(400, np.float32)
    vp = ctypes.c_void_p
    nnz = lg.leiden_csr_from_edges(50, 200, vp(u.ctypes.data), vp(v.ctypes.data), vp(w.ctypes.data), lg.LEIDEN_HOST, 0,
                                   0, vp(off.ctypes.data), vp(idx.ctypes.data), vp(ww.ctypes.data), 400, None)
    ref = oracle.csr_from_edges(50, u, v, w)
    assert np.array_equal(off, ref[0]) and np.array_equal(idx[:nnz], ref[1]) and np.array_equal(ww[:nnz], ref[2])
    # an endpoint outside [0, n)
    bad = v.copy()
    bad[3] = 50
    with pytest.raises(lg.LeidenError) as e:
        lg.leiden_csr_from_edges(50, 200, vp(u.ctypes.data), vp(bad.ctypes.data), None, lg.LEIDEN_HOST, 0, 0,
                                 vp(off.ctypes.data), vp(idx.ctypes.data), vp(ww.ctypes.data), 400, None)
    assert e.value.status == -1
    # too small a capacity
    with pytest.raises(lg.LeidenError) as e:
        lg.leiden_csr_from_edges(50, 200, vp(u.ctypes.data), vp(v.ctypes.data), None, lg.LEIDEN_HOST, 0, 0,
                                 vp(off.ctypes.data), vp(idx.ctypes.data), vp(ww.ctypes.data), 10, None)
    assert e.value.status == -1
