"""Batches of graphs on several GPUs (one process per GPU).

The graphs of a batch are independent problems, so a batch shards with no
data-path collective: the graphs are dealt to the ranks by estimated work --
longest-processing-time first by CSR entry count, each graph to the rank with
the least work so far -- every rank packs its share as one segmented CSR and
solves it with one ``leiden_batch_run`` on its own GPU, and the results come
back to every rank by one gather of host arrays at the end.

``lpt_shares``, ``pack_share`` and ``gather_results`` are plain host logic;
``run_sharded`` puts them around the library's batch handle. A packed batch is
any object with ``num_graphs``, ``vseg`` (G+1 vertex offsets), ``offsets``,
``indices`` (local to each graph) and ``weights`` numpy arrays, the layout of
``pack_batch``.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_shares(m, world: int):
    """Graph ids of each rank: longest-processing-time first by entry count.

    Graphs in decreasing m (ties by smaller id) go one by one to the rank with
    the least load so far (ties by smaller rank). Each rank's ids come back in
    increasing order. The largest load is at most 4/3 of the best possible
    one (Graham's LPT bound) and at most the mean load plus the largest m."""
    m = np.asarray(m, dtype=np.int64)
    order = np.lexsort((np.arange(len(m)), -m))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        shares[r].append(int(g))
        heapq.heappush(heap, (load + int(m[g]), r))
    return [np.array(sorted(x), dtype=np.int64) for x in shares]


def graph_entries(b):
    """Directed CSR entries of every graph of a packed batch."""
    return np.asarray(b.offsets)[b.vseg[1:]] - np.asarray(b.offsets)[b.vseg[:-1]]


def pack_share(b, ids):
    """The graphs ``ids`` (increasing) of a packed batch as a packed batch of
    their own: vertex segments, offsets, local indices, weights."""
    ids = np.asarray(ids, dtype=np.int64)
    if len(ids) == b.num_graphs and np.array_equal(ids, np.arange(b.num_graphs)):
        return b.vseg, b.offsets, b.indices, b.weights  # the whole batch: no copy
    nv = b.vseg[ids + 1] - b.vseg[ids]
    vseg = np.zeros(len(ids) + 1, dtype=np.int64)
    np.cumsum(nv, out=vseg[1:])
    offs, idxs, ws = [np.zeros(1, dtype=np.int64)], [], []
    base = 0
    for g in ids:
        v0, v1 = int(b.vseg[g]), int(b.vseg[g + 1])
        e0, e1 = int(b.offsets[v0]), int(b.offsets[v1])
        offs.append(b.offsets[v0 + 1:v1 + 1] - e0 + base)
        idxs.append(b.indices[e0:e1])  # local to their graph already
        ws.append(b.weights[e0:e1])
        base += e1 - e0
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt, copy=False) if xs else np.zeros(0, dtype=dt))
    return vseg, cat(offs, np.int64), cat(idxs, b.indices.dtype), cat(ws, b.weights.dtype)


def gather_results(num_graphs: int, ids, sizes, membership, modularity, world: int, group=None):
    """Every rank's results, on every rank, in the batch's own graph order.

    ``ids`` are the rank's graphs, ``sizes`` their vertex counts,
    ``membership`` their labels one after another (in the order of ``ids``)
    and ``modularity`` one value per graph. Returns (a list of num_graphs
    label arrays, a float64 array of num_graphs modularities). With one rank
    nothing is exchanged."""
    part = (np.asarray(ids, dtype=np.int64), np.asarray(sizes, dtype=np.int64),
            np.asarray(membership, dtype=np.int32), np.asarray(modularity, dtype=np.float64))
    parts = [part]
    if world > 1:
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, part, group=group)
    memb = [np.zeros(0, dtype=np.int32)] * num_graphs
    q = np.zeros(num_graphs, dtype=np.float64)
    for gids, gsz, labels, mod in parts:
        ends = np.cumsum(gsz)
        starts = ends - gsz
        for k, g in enumerate(gids.tolist()):
            memb[g] = labels[starts[k]:ends[k]]
            q[g] = mod[k]
    return memb, q


def run_sharded(b, rank: int, world: int, mode: int = 0, group=None, **params):
    """Solve a packed batch on ``world`` GPUs: this rank's LPT share as one
    leiden_batch_run on the current device, then every rank's results
    gathered to every rank. Returns (list of per-graph label arrays, per-graph
    modularity, this rank's graph ids, this rank's run statistics)."""
    from . import LeidenBatch
    ids = lpt_shares(graph_entries(b), world)[rank]
    vseg, off, idx, w = pack_share(b, ids)
    h = LeidenBatch(vseg, off, idx, w)
    try:
        memb, q, st = h.run(mode=mode, **params)
        labels = memb.cpu().numpy()
    finally:
        h.close()
    memb_all, q_all = gather_results(b.num_graphs, ids, np.diff(vseg), labels, q, world, group)
    return memb_all, q_all, ids, st
