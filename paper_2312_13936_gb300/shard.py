"""Batches of graphs on several GPUs (one process per GPU).

The graphs of a batch are independent problems, so a batch shards with no
data-path collective: the graphs are dealt to the ranks by estimated work --
longest-processing-time first by CSR entry count, each graph to the rank with
the least work so far -- every rank packs its share as one segmented CSR and
solves it with one ``leiden_batch_run`` on its own GPU, and the results come
back to every rank by one gather of host arrays at the end.

``lpt_shares``, ``pack_share`` and ``gather_results`` are plain host logic;
``run_sharded`` puts them around the library's batch handle.

The served form spreads over the GPUs of one process with ``ServeRouter``:
one continuous-batching server per device, each request admitted to the
device with the least outstanding work, every device stepped by its own host
thread. A packed batch is
any object with ``num_graphs``, ``vseg`` (G+1 vertex offsets), ``offsets``,
``indices`` (local to each graph) and ``weights`` numpy arrays, the layout of
``pack_batch``.
"""
from __future__ import annotations

import heapq
import itertools
from concurrent.futures import ThreadPoolExecutor

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


class ServeRouter:
    """Continuous batching on several GPUs of one process.

    One server per device (``make_server(device)``, by default a
    ``LeidenServer`` created on that device). A request goes to the device
    with the least outstanding work -- the CSR entries of its requests not
    yet returned by ``results`` -- ties to the earlier device, so that the
    devices fill like the LPT dealing of a batch, but online: a request is
    placed when it arrives. Every device has one host thread of its own,
    bound to it by ``bind(device)`` (by default ``torch.cuda.set_device``),
    and all calls to its server run there; ``step`` steps every server at
    once, each in its thread (the library's calls release the interpreter
    lock), and returns the number of graphs finished. Request ids are the
    router's own; ``results`` drains every device, device by device, each in
    its finishing order, as (id, membership, modularity, passes,
    communities), the membership a numpy array, or with ``device=True`` a
    tensor on the GPU that ran the graph. ``close`` releases every server and
    thread."""

    def __init__(self, devices, make_server=None, bind=None, **server_args):
        self.devices = list(devices)
        if not self.devices:
            raise ValueError("ServeRouter needs at least one device")
        if make_server is None:
            from . import LeidenServer

            def make_server(device):
                return LeidenServer(**server_args)
        if bind is None:
            def bind(device):
                import torch
                torch.cuda.set_device(device)
        self._pools = [ThreadPoolExecutor(max_workers=1, initializer=bind, initargs=(d,)) for d in self.devices]
        self.servers = [self._on(k, make_server, d) for k, d in enumerate(self.devices)]
        self.load = [0] * len(self.devices)  # outstanding CSR entries per device
        self._ids = itertools.count()
        self._route = {}  # (device index, server id) -> (router id, entries)

    def _on(self, k, fn, *args):
        return self._pools[k].submit(fn, *args).result()

    def pick(self) -> int:
        """Index of the device a request would go to now."""
        return min(range(len(self.devices)), key=lambda k: (self.load[k], k))

    def submit(self, offsets, indices, weights=None) -> int:
        k = self.pick()
        m = int(len(indices))
        sid = self._on(k, self.servers[k].submit, offsets, indices, weights)
        rid = next(self._ids)
        self._route[(k, sid)] = (rid, m)
        self.load[k] += m
        return rid

    def step(self) -> int:
        futs = [pool.submit(srv.step) for pool, srv in zip(self._pools, self.servers)]
        return sum(int(f.result()) for f in futs)

    def results(self, device: bool = False):
        out = []
        for k, srv in enumerate(self.servers):
            for sid, memb, q, passes, comm in self._on(k, srv.results, device):
                rid, m = self._route.pop((k, sid))
                self.load[k] -= m
                out.append((rid, memb, q, passes, comm))
        return out

    def busy(self) -> bool:
        """Requests submitted and not yet returned by ``results``."""
        return bool(self._route)

    def close(self):
        servers, pools = getattr(self, "servers", []), getattr(self, "_pools", [])
        self.servers, self._pools = [], []
        err = None
        try:
            for pool, srv in zip(pools, servers):  # every server, even after one fails
                try:
                    pool.submit(srv.close).result()
                except Exception as e:
                    err = err or e
        finally:
            for pool in pools:
                pool.shutdown()
        if err is not None:
            raise err

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
