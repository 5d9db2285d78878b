"""GPU tests of the served form: continuous batching (leiden_server_*).

Graphs are submitted while others are in flight; each step admits waiting
graphs at the pass boundary and runs one pass of every graph in flight.
Deterministic mode: every graph's result (membership, passes, communities,
modularity) is bit-exact the single-graph result of leiden_run, whatever it
was mixed with. Asynchronous mode: every community connected, reported
modularity equal to the recomputation, and every graph's expected modularity
within 0.005 of the oracle's sequential reference, alone and served (see the
batched-form tests).
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2312_13936_gb300 as lg
from tests._gpu import SEEDS, run_gpu, seq_reference

pytestmark = pytest.mark.gpu


def serve_mix():
    b = gen.sbm_batch(16, seed=21, nmin=50, nmax=4000)
    graphs = [b.graph(g) for g in range(b.num_graphs)]
    graphs.insert(2, gen.ring_of_cliques(5, 8))
    graphs.insert(5, gen.road(40))
    graphs.insert(6, gen.from_edges(4, [], []))
    graphs.insert(8, gen.from_edges(0, [], []))
    graphs.insert(11, gen.from_edges(1, [0], [0], [2.0]))
    graphs.append(gen.rmat(11, 8, seed=5))
    return graphs


def serve(graphs, mode, arrivals_per_step=3, **kw):
    """Submit a few graphs before every step (so later graphs join graphs
    already in flight) and run steps until everything finished."""
    cap_v = max(1, sum(g.n for g in graphs))
    cap_e = max(1, sum(g.nnz for g in graphs))
    srv = lg.LeidenServer(cap_v, cap_e, max_graphs=len(graphs) + 1, mode=mode, **kw)
    ids, res = [], {}
    k = 0
    steps = 0
    try:
        while k < len(graphs) or len(res) < len(graphs):
            for _ in range(arrivals_per_step):
                if k < len(graphs):
                    g = graphs[k]
                    ids.append(srv.submit(g.offsets, g.indices, g.weights))
                    k += 1
            srv.step()
            steps += 1
            for rid, memb, q, passes, comm in srv.results():
                res[rid] = (memb, q, passes, comm)
            assert steps < 1000
        info = srv.info()
    finally:
        srv.close()
    return [res[i] for i in ids], info, steps


def test_serve_deterministic_same_alone_and_in_mix():
    graphs = serve_mix()
    out, info, steps = serve(graphs, lg.LEIDEN_DETERMINISTIC)
    assert info["in_flight"] == 0 and info["waiting"] == 0 and info["finished"] == 0
    assert info["device_bytes"] == 0
    assert steps > 3
    for g, (G, (memb, q, passes, comm)) in enumerate(zip(graphs, out)):
        ms, qs, sts, _ = run_gpu(G, lg.LEIDEN_DETERMINISTIC)
        assert np.array_equal(memb, ms), g
        assert abs(q - qs) <= 1e-12 * max(1.0, abs(qs)), (g, q, qs)
        if G.n > 0:
            assert passes == sts.passes, (g, passes, sts.passes)
            assert comm == sts.communities


def test_serve_deterministic_matches_oracle():
    graphs = serve_mix()[:8]
    out, _, _ = serve(graphs, lg.LEIDEN_DETERMINISTIC, arrivals_per_step=2)
    for g, G in enumerate(graphs):
        ref = oracle.leiden(G, mode=oracle.SYNC)
        assert np.array_equal(out[g][0], ref.membership), g


def test_serve_deterministic_limits():
    graphs = serve_mix()[:10]
    for kw in ({"max_passes": 2}, {"max_iterations": 3}, {"schedule_layers": 5, "schedule_buckets": 2, "seed": 3},
               {"flags": lg.FLAG_LOUVAIN}, {"flags": lg.FLAG_REFINE_LABELS}):
        out, _, _ = serve(graphs, lg.LEIDEN_DETERMINISTIC, arrivals_per_step=4, **kw)
        for g, G in enumerate(graphs):
            ms = run_gpu(G, lg.LEIDEN_DETERMINISTIC, **kw)[0]
            assert np.array_equal(out[g][0], ms), (kw, g)


def test_serve_async_quality():
    """In the mix, every graph connected, its reported modularity equal to
    the recomputation, and its expected modularity (the mean over schedule
    seeds) within 0.005 of the oracle's sequential reference, alone and
    served; the served mean within 0.005 of the mean alone."""
    graphs = serve_mix()
    ref = np.array([seq_reference(G) for G in graphs])
    qs_srv, qs_alone = [], []
    for seed in range(SEEDS):
        out, _, _ = serve(graphs, lg.LEIDEN_ASYNC, seed=seed)
        for g, (G, (memb, q, passes, comm)) in enumerate(zip(graphs, out)):
            assert oracle.disconnected(G, memb)[0] == 0, g
            q_re = oracle.modularity(G, memb)
            assert abs(q - q_re) <= 1e-9 * max(1.0, abs(q_re)), g
        qs_srv.append([o[1] for o in out])
        qs_alone.append([run_gpu(G, lg.LEIDEN_ASYNC, seed=seed)[1] for G in graphs])
    qs_srv, qs_alone = np.mean(qs_srv, axis=0), np.mean(qs_alone, axis=0)
    assert abs(qs_srv.mean() - qs_alone.mean()) <= 0.005
    for g in range(len(graphs)):
        assert qs_srv[g] >= ref[g] - 0.005, (g, qs_srv[g], ref[g])
        assert qs_alone[g] >= ref[g] - 0.005, (g, qs_alone[g], ref[g])


def test_serve_admission_waits_for_capacity():
    # room for two graphs in flight and a device budget of about one graph:
    # the others wait (on the host) and still come out exact
    graphs = [gen.sbm(800, 6, 0.05, 0.003, seed=s) for s in range(6)]
    cap_v = 2 * max(g.n for g in graphs)
    cap_e = 2 * max(g.nnz for g in graphs)
    budget = 20 * (graphs[0].n + graphs[0].nnz)
    srv = lg.LeidenServer(cap_v, cap_e, max_graphs=2, device_budget=budget, mode=lg.LEIDEN_DETERMINISTIC)
    try:
        ids = [srv.submit(g.offsets, g.indices, g.weights) for g in graphs]
        info = srv.info()
        assert info["waiting"] == len(graphs) and info["in_flight"] == 0
        res = {}
        peak = 0
        for _ in range(200):
            srv.step()
            peak = max(peak, srv.info()["in_flight"])
            for rid, memb, q, passes, comm in srv.results():
                res[rid] = memb
            if len(res) == len(graphs):
                break
        assert peak <= 2
        for rid, G in zip(ids, graphs):
            assert np.array_equal(res[rid], run_gpu(G, lg.LEIDEN_DETERMINISTIC)[0])
        assert srv.info()["device_bytes"] == 0
        # a graph larger than the capacity is refused
        big = gen.sbm(cap_v + 1, 4, 0.01, 0.001, seed=1)
        with pytest.raises(lg.LeidenError) as e:
            srv.submit(big.offsets, big.indices, big.weights)
        assert e.value.status == -1
    finally:
        srv.close()


def test_serve_refuses_a_graph_over_the_budget():
    """A graph whose own buffers exceed the device budget could never be
    admitted: it is refused at submit, and later graphs still run."""
    g = gen.ring_of_cliques(4, 5)  # 20 vertices, 70 entries: 8*21 + 4*20 + 8*70 = 808 bytes
    small = gen.from_edges(2, np.array([0]), np.array([1]))  # 8*3 + 4*2 + 8*2 = 48 bytes
    srv = lg.LeidenServer(1000, 10000, device_budget=200, mode=lg.LEIDEN_DETERMINISTIC)
    try:
        with pytest.raises(lg.LeidenError) as e:
            srv.submit(g.offsets, g.indices, g.weights)
        assert e.value.status == -3
        rid = srv.submit(small.offsets, small.indices, small.weights)
        res = {}
        for _ in range(50):
            srv.step()
            for r in srv.results():
                res[r[0]] = r[1]
            if res:
                break
        assert np.array_equal(res[rid], oracle.leiden(small, mode=oracle.SYNC).membership)
    finally:
        srv.close()


def test_serve_rejects_bad_graphs():
    g = gen.ring_of_cliques(4, 5)
    srv = lg.LeidenServer(1000, 10000, mode=lg.LEIDEN_DETERMINISTIC)
    try:
        w = g.weights.copy()
        w[0] = 2.0
        with pytest.raises(lg.LeidenError) as e:
            srv.submit(g.offsets, g.indices, w)
        assert e.value.status == -2
        with pytest.raises(lg.LeidenError) as e:
            srv.submit(g.offsets, g.indices, g.weights * 0.5)
        assert e.value.status == -6
        # the server still works afterwards
        rid = srv.submit(g.offsets, g.indices, g.weights)
        for _ in range(50):
            srv.step()
            r = srv.results()
            if r:
                break
        assert r[0][0] == rid and np.array_equal(r[0][1], run_gpu(g, lg.LEIDEN_DETERMINISTIC)[0])
        assert srv.info()["device_bytes"] == 0
    finally:
        srv.close()


def test_serve_mixed_layer_caps_same_alone_and_in_mix():
    """Graphs of layer cap 1000 and 32 (reading S0) in flight together: each
    equals its single run bit for bit."""
    from tests.test_gpu_batch import mixed_layer_caps
    graphs = mixed_layer_caps()
    out, info, _ = serve(graphs, lg.LEIDEN_DETERMINISTIC, arrivals_per_step=2)
    for g, (G, (memb, q, passes, comm)) in enumerate(zip(graphs, out)):
        ms, qs, sts, _ = run_gpu(G, lg.LEIDEN_DETERMINISTIC)
        assert np.array_equal(memb, ms), g
        assert passes == sts.passes, g


def test_serve_lanes_by_layer_cap():
    """A heavy-tailed graph (layer cap 1000) and light ones go to separate
    lanes, and a step runs one pass of one lane: the steps add up to the
    graphs' passes (one union would advance all of them together), and each
    result still equals its single run bit for bit."""
    from tests.test_gpu_parity import hub_graph
    heavy, light = hub_graph(), gen.road(40)
    assert int(np.diff(heavy.offsets).max()) * heavy.n > 64 * heavy.nnz
    assert int(np.diff(light.offsets).max()) * light.n <= 64 * light.nnz
    out, info, steps = serve([heavy, light], lg.LEIDEN_DETERMINISTIC, arrivals_per_step=2)
    alone = [run_gpu(G, lg.LEIDEN_DETERMINISTIC) for G in (heavy, light)]
    assert steps == info["steps"] == alone[0][2].passes + alone[1][2].passes
    for (memb, q, passes, comm), (ms, qs, sts, _) in zip(out, alone):
        assert np.array_equal(memb, ms) and passes == sts.passes
    # with a fixed layer cap every graph shares one lane
    out, info, steps = serve([heavy, light], lg.LEIDEN_DETERMINISTIC, arrivals_per_step=2, schedule_layers=32)
    p = [run_gpu(G, lg.LEIDEN_DETERMINISTIC, schedule_layers=32)[2].passes for G in (heavy, light)]
    assert steps == max(p)


def test_serve_device_submissions_take_their_lanes():
    """Graphs submitted as CUDA tensors are classed on the device (their
    largest row length) like host ones: a heavy-tailed graph and a light one
    in separate lanes (the steps add up to their passes), each result equal to
    its single run, and results read back to device memory."""
    import torch
    from tests.test_gpu_parity import hub_graph
    heavy, light = hub_graph(), gen.road(40)
    srv = lg.LeidenServer(heavy.n + light.n, heavy.nnz + light.nnz, max_graphs=4, mode=lg.LEIDEN_DETERMINISTIC)
    try:
        ids = [srv.submit(torch.as_tensor(G.offsets).cuda(), torch.as_tensor(G.indices).cuda(),
                          torch.as_tensor(G.weights).cuda()) for G in (heavy, light)]
        res, steps = {}, 0
        while len(res) < 2:
            srv.step()
            steps += 1
            for rid, memb, q, passes, comm in srv.results(device=True):
                assert memb.is_cuda
                res[rid] = (memb.cpu().numpy(), passes)
            assert steps < 200
        alone = [run_gpu(G, lg.LEIDEN_DETERMINISTIC) for G in (heavy, light)]
        assert steps == alone[0][2].passes + alone[1][2].passes
        for rid, (ms, qs, sts, _) in zip(ids, alone):
            assert np.array_equal(res[rid][0], ms) and res[rid][1] == sts.passes
    finally:
        srv.close()


def test_router_on_one_device_matches_the_oracle():
    """The multi-device router (paper_2312_13936_gb300.shard.ServeRouter) on the
    one GPU of the test: its server runs on the router's own thread for the
    device, and every graph's deterministic result equals the oracle's SYNC
    run, under the router's ids."""
    import torch

    from paper_2312_13936_gb300.shard import ServeRouter
    graphs = serve_mix()[:10]
    cap_v = max(1, sum(g.n for g in graphs))
    cap_e = max(1, sum(g.nnz for g in graphs))
    r = ServeRouter([torch.cuda.current_device()], max_vertices=cap_v, max_entries=cap_e,
                    max_graphs=len(graphs) + 1, mode=lg.LEIDEN_DETERMINISTIC)
    res = {}
    try:
        ids = []
        for k, g in enumerate(graphs):
            ids.append(r.submit(g.offsets, g.indices, g.weights))
            if k % 3 == 2:
                r.step()
                res.update({rid: memb for rid, memb, *_ in r.results()})
        steps = 0
        while r.busy():
            r.step()
            res.update({rid: memb for rid, memb, *_ in r.results()})
            steps += 1
            assert steps < 1000
    finally:
        r.close()
    assert ids == list(range(len(graphs)))
    for rid, G in zip(ids, graphs):
        assert np.array_equal(res[rid], oracle.leiden(G, mode=oracle.SYNC).membership), rid
