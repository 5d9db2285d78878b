"""The multi-rank host logic of bench.py on CPU: two processes over the gloo
backend (127.0.0.1). The batched form's graphs are split in contiguous
shares that cover the batch exactly once; per-rank sums add up and per-rank
times reduce to the largest, as they do over NCCL on GPUs; each rank's work
here is the oracle on its share."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
        b = gen.sbm_batch(9, seed=3, nmin=50, nmax=600)
        lo, hi = bench.shard_range(b.num_graphs, rank, world)
        vseg, off, idx, w = bench.shard_batch(b, lo, hi)
        q = []
        for g in range(hi - lo):
            a, c = int(vseg[g]), int(vseg[g + 1])
            e0, e1 = int(off[a]), int(off[c])
            G = gen.CSR(c - a, off[a:c + 1] - e0, idx[e0:e1].copy(), w[e0:e1].copy())
            q.append(oracle.leiden(G, mode=oracle.SEQ).modularity)
        stats = torch.tensor([float(rank + 1), float(np.sum(q)), float(len(q))], dtype=torch.float64)
        red = bench.reduce_stats(stats, 1, world)
        out.put((rank, lo, hi, red.tolist()))
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
    # the shares are contiguous, disjoint and cover every graph once
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == b.num_graphs
    # every rank holds the same reduced stats: the largest time, the sums
    assert res[0][3] == res[1][3]
    t, qsum, count = res[0][3]
    assert t == float(world)
    assert count == b.num_graphs
    ref = sum(oracle.leiden(b.graph(g), mode=oracle.SEQ).modularity for g in range(b.num_graphs))
    assert abs(qsum - ref) <= 1e-12 * max(1.0, abs(ref))


def test_one_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    s = torch.tensor([3.0, 4.0])
    assert bench.reduce_stats(s, 1, 1).tolist() == [3.0, 4.0]
    assert bench.shard_range(10, 0, 1) == (0, 10)
    assert [bench.shard_range(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
