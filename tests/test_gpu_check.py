"""GPU tests of the disconnected-community checker (Appendix A.1, Algorithm 5)
against the oracle's per-community BFS."""
import numpy as np
import pytest

import gen
import oracle
import paper_2312_13936_gb300 as lg
from tests.test_gpu_parity import hub_graph

pytestmark = pytest.mark.gpu


def gpu_count(g, memb):
    import torch
    dev = torch.device("cuda")
    off = torch.as_tensor(g.offsets).to(dev)
    idx = torch.as_tensor(g.indices).to(dev)
    m = torch.as_tensor(np.ascontiguousarray(memb, dtype=np.int32)).to(dev)
    return lg.disconnected(off, idx, m)


@pytest.mark.parametrize("seed", range(4))
def test_random_memberships_match_oracle(seed):
    rng = np.random.default_rng(seed)
    g = gen.gnp(3000, 0.002, seed=seed)
    for k in (2, 40, 1500):  # few labels: many disconnected; many labels: few
        memb = rng.integers(0, k, g.n).astype(np.int32)
        assert gpu_count(g, memb) == oracle.disconnected(g, memb)[0], k


def test_long_rows_match_oracle():
    g = hub_graph()
    rng = np.random.default_rng(3)
    memb = rng.integers(0, 50, g.n).astype(np.int32)
    assert gpu_count(g, memb) == oracle.disconnected(g, memb)[0]
    memb[:] = 0  # one community: connected iff the graph is
    assert gpu_count(g, memb) == oracle.disconnected(g, memb)[0]


def test_planted_cases():
    # two triangles and an isolated vertex, all in community 0: disconnected
    g = gen.from_edges(7, [0, 0, 1, 3, 3, 4], [1, 2, 2, 4, 5, 5])
    assert gpu_count(g, np.zeros(7, np.int32)) == 1
    assert gpu_count(g, np.array([0, 0, 0, 1, 1, 1, 2], np.int32)) == 0
    # vertex 2 in the second triangle's community, without an edge to it
    assert gpu_count(g, np.array([0, 0, 1, 1, 1, 1, 2], np.int32)) == 1
    assert gpu_count(gen.from_edges(0, [], []), np.zeros(0, np.int32)) == 0


def test_leiden_results_are_connected():
    for g in (gen.road(300), gen.sbm_workload(), gen.rmat(12, 16)):
        memb = lg.Leiden(g.offsets, g.indices, g.weights).run()[0]
        m = memb.cpu().numpy()
        assert gpu_count(g, m) == 0 == oracle.disconnected(g, m)[0]


def test_labels_out_of_range_rejected():
    g = gen.ring_of_cliques(4, 3)
    memb = np.zeros(g.n, np.int32)
    memb[3] = g.n
    with pytest.raises(lg.LeidenError) as e:
        gpu_count(g, memb)
    assert e.value.status == -1
    memb[3] = -1
    with pytest.raises(lg.LeidenError) as e:
        gpu_count(g, memb)
    assert e.value.status == -1
