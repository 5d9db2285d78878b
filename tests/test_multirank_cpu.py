"""The multi-GPU batch API on CPU (paper_2312_13936_gb300.shard): two
processes over the gloo backend (127.0.0.1). A batch's graphs are dealt to
ranks longest-first by entry count, in shares that cover the batch exactly
once; each rank packs its share, solves it (here with the oracle standing in
for leiden_batch_run, which needs a GPU), and gather_results brings every
graph's labels and modularity to every rank in the batch's own order; the
bench's per-rank sums add up and times reduce to the largest, as they do over
NCCL on GPUs."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

import paper_2312_13936_gb300 as lg  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import gen
        import oracle
        import paper_2312_13936_gb300 as lg
        b = gen.sbm_batch(9, seed=3, nmin=50, nmax=600)
        ids = lg.shard.lpt_shares(lg.shard.graph_entries(b), world)[rank]
        vseg, off, idx, w = lg.shard.pack_share(b, ids)
        q, labels = [], []
        for g in range(len(ids)):
            a, c = int(vseg[g]), int(vseg[g + 1])
            e0, e1 = int(off[a]), int(off[c])
            G = gen.CSR(c - a, off[a:c + 1] - e0, idx[e0:e1].copy(), w[e0:e1].copy())
            r = oracle.leiden(G, mode=oracle.SEQ)
            q.append(r.modularity)
            labels.append(r.membership)
        memb_all, q_all = lg.shard.gather_results(b.num_graphs, ids, np.diff(vseg),
                                                  np.concatenate(labels), q, world)
        stats = torch.tensor([float(rank + 1), float(np.sum(q)), float(len(q))], dtype=torch.float64)
        red = bench.reduce_stats(stats, 1, world)
        out.put((rank, ids.tolist(), red.tolist(), [m.tolist() for m in memb_all], q_all.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    import sys
    sys.path.insert(0, ROOT)
    import gen
    import oracle
    b = gen.sbm_batch(9, seed=3, nmin=50, nmax=600)
    # the shares are disjoint and cover every graph once
    assert sorted(res[0][1] + res[1][1]) == list(range(b.num_graphs))
    # every rank holds the same reduced stats: the largest time, the sums
    assert res[0][2] == res[1][2]
    t, qsum, count = res[0][2]
    assert t == float(world)
    assert count == b.num_graphs
    ref = sum(oracle.leiden(b.graph(g), mode=oracle.SEQ).modularity for g in range(b.num_graphs))
    assert abs(qsum - ref) <= 1e-12 * max(1.0, abs(ref))
    # the gather gives every rank every graph's own result, in batch order
    assert res[0][3] == res[1][3] and res[0][4] == res[1][4]
    for g in range(b.num_graphs):
        r = oracle.leiden(b.graph(g), mode=oracle.SEQ)
        assert res[0][3][g] == r.membership.tolist()
        assert res[0][4][g] == r.modularity


def test_one_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    s = torch.tensor([3.0, 4.0])
    assert bench.reduce_stats(s, 1, 1).tolist() == [3.0, 4.0]
    (only,) = lg.shard.lpt_shares([5, 1, 7], 1)
    assert only.tolist() == [0, 1, 2]


def test_lpt_shares_by_hand():
    # 7, 5, 4, 3, 3, 2 onto 2 ranks: 7->r0, 5->r1, 4->r1 (9), 3->r0 (10),
    # 3->r1 (12), 2->r0 (12)
    m = [3, 7, 2, 5, 4, 3]
    r0, r1 = lg.shard.lpt_shares(m, 2)
    assert r0.tolist() == [0, 1, 2] and r1.tolist() == [3, 4, 5]
    # more ranks than graphs: some shares are empty, none repeats a graph
    sh = lg.shard.lpt_shares([4, 4], 3)
    assert [x.tolist() for x in sh] == [[0], [1], []]


def test_lpt_within_graham_bound_of_brute_force():
    """The largest load is at most 4/3 of the optimum, which brute force over
    every assignment finds on tiny instances."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        n, world = int(rng.integers(1, 8)), int(rng.integers(2, 4))
        m = rng.integers(1, 50, size=n)
        sh = lg.shard.lpt_shares(m, world)
        assert sorted(np.concatenate(sh).tolist()) == list(range(n))
        lpt = max(int(m[x].sum()) for x in sh)
        best = min(max(sum(int(m[g]) for g in range(n) if a[g] == r) for r in range(world))
                   for a in itertools.product(range(world), repeat=n))
        assert lpt * 3 <= 4 * best
        assert lpt <= m.sum() / world + m.max()


def test_pack_graphs_round_trip():
    """A packed share holds each chosen graph entry for entry."""
    import gen
    b = gen.sbm_batch(7, seed=2, nmin=30, nmax=300)
    ids = np.array([1, 4, 6])
    vseg, off, idx, w = lg.shard.pack_share(b, ids)
    assert len(vseg) == 4 and off[-1] == len(idx) == len(w)
    for k, g in enumerate(ids):
        a, c = int(vseg[k]), int(vseg[k + 1])
        e0, e1 = int(off[a]), int(off[c])
        ref = b.graph(int(g))
        assert c - a == ref.n
        assert np.array_equal(off[a:c + 1] - e0, ref.offsets)
        assert np.array_equal(idx[e0:e1], ref.indices)
        assert np.array_equal(w[e0:e1], ref.weights)
    assert np.array_equal(lg.shard.graph_entries(b)[ids], np.diff(off[vseg]))
    empty = lg.shard.pack_share(b, np.zeros(0, dtype=np.int64))
    assert empty[0].tolist() == [0] and empty[1].tolist() == [0] and len(empty[2]) == 0
