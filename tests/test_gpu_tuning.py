"""Launch shapes on the GPU: every candidate shape of the autotuner leaves
the deterministic mode bit-exact against the oracle's SYNC mode (single
graphs, including hubs, and batches; rows copied in list order for every
pass, for passes of 1000 vertices and more, and never), an asynchronous run under a tuned
shape keeps the quality checks, and a handle created with
LEIDEN_TUNING_CACHE set takes the cache's entry for the GPU and the graph's
class."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
import paper_2312_13936_gb300 as lg
from tests._gpu import compare_traces
from tests.test_gpu_parity import hub_graph

pytestmark = pytest.mark.gpu

SHAPES = [
    {"thread_max_deg": 4, "warp_max_deg": 64, "block_max_deg": 512, "coop_blocks_per_sm": 2,
     "vertices_per_block": 1024, "list_order_min_vertices": 1},
    {"thread_max_deg": 1, "warp_max_deg": 32, "block_max_deg": 128, "coop_blocks_per_sm": 1,
     "vertices_per_block": 256, "list_order_min_vertices": 0},
    {"thread_max_deg": 8, "warp_max_deg": 128, "block_max_deg": 1024, "coop_blocks_per_sm": 3,
     "vertices_per_block": 4096, "list_order_min_vertices": 1000},
]
GRAPHS = {"road_200": lambda: gen.road(200), "hubs": hub_graph, "rmat_12": lambda: gen.rmat(12, 16),
          "sbm": lambda: gen.sbm(4000, 16, 0.04, 0.002, seed=5)}


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_tuned_shapes_stay_bit_exact(name, shape):
    g = GRAPHS[name]()
    ref = oracle.leiden(g, mode=oracle.SYNC, trace=True)
    h = lg.Leiden(g.offsets, g.indices, g.weights, tuning=SHAPES[shape])
    try:
        assert h.tuning() == SHAPES[shape]
        memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC, trace=True)
        tr = {p: {w: h.trace(p, w) for w in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10) if _has(h, p, w)}
              for p in range(st.passes)}
        assert not compare_traces(tr, ref.trace)
        assert np.array_equal(memb.cpu().numpy(), ref.membership)
    finally:
        h.close()


def _has(h, p, w):
    try:
        h.trace(p, w)
        return True
    except lg.LeidenError:
        return False


def test_tuned_batch_stays_bit_exact():
    b = gen.sbm_batch(12, seed=13, nmin=200, nmax=3000)
    graphs = [b.graph(g) for g in range(b.num_graphs)] + [hub_graph()]
    vseg, off, idx, w = lg.pack_batch(graphs)
    hb = lg.LeidenBatch(vseg, off, idx, w, tuning=SHAPES[0])
    try:
        memb, q, st = hb.run(mode=lg.LEIDEN_DETERMINISTIC)
        memb = memb.cpu().numpy()
    finally:
        hb.close()
    for k, G in enumerate(graphs):
        ref = oracle.leiden(G, mode=oracle.SYNC)
        assert np.array_equal(memb[vseg[k]:vseg[k + 1]], ref.membership), k


def test_tuned_shape_async_quality():
    g = hub_graph()
    h = lg.Leiden(g.offsets, g.indices, g.weights, tuning=SHAPES[0])
    try:
        memb, q, st = h.run(mode=lg.LEIDEN_ASYNC)
        memb = memb.cpu().numpy()
    finally:
        h.close()
    assert oracle.disconnected(g, memb)[0] == 0
    assert abs(q - oracle.modularity(g, memb)) <= 1e-9


def test_cache_applied_at_create(tmp_path, monkeypatch):
    import torch
    g = gen.road(100)
    c = lg.tune.graph_class(g.n, g.nnz, int(np.diff(g.offsets).max()))
    entry = {"gpu": torch.cuda.get_device_name(), **c, **SHAPES[2]}
    path = tmp_path / "cache.json"
    path.write_text(json.dumps({"format": 1, "entries": [entry]}))
    monkeypatch.setenv("LEIDEN_TUNING_CACHE", str(path))
    h = lg.Leiden(g.offsets, g.indices, g.weights)
    try:
        assert h.tuning() == SHAPES[2]
    finally:
        h.close()
    monkeypatch.delenv("LEIDEN_TUNING_CACHE")
    h = lg.Leiden(g.offsets, g.indices, g.weights, tuning=None)
    try:
        assert h.tuning() == lg.leiden_tuning_default().as_dict()
    finally:
        h.close()
