"""The served form on several devices (paper_2312_13936_gb300.shard.ServeRouter)
on CPU: one server per device, each request to the device with the least
outstanding CSR entries, every device's calls on one host thread bound to it,
all devices stepped at once, and every result returned under the router's own
id. The servers here are stand-ins that solve their graphs with the oracle
(a real server needs a GPU); the GPU test of the same router is in
test_gpu_serve.py."""
import os
import sys
import threading

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402
from paper_2312_13936_gb300.shard import ServeRouter  # noqa: E402

_bound = threading.local()


def _bind(device):
    _bound.device = device


class OracleServer:
    """A server stand-in: a submitted graph finishes at the next step, solved
    by the oracle (SEQ mode). Records the thread of every call and the
    device bound to it."""

    def __init__(self, device, barrier=None):
        self.device = device
        self.barrier = barrier
        self.threads = set()
        self.bound = set()
        self.pending, self.done = [], []
        self.next_id = 0  # every server numbers its requests from 0, as the library's do
        self.closed = False

    def _seen(self):
        self.threads.add(threading.get_ident())
        self.bound.add(getattr(_bound, "device", None))

    def submit(self, offsets, indices, weights=None):
        self._seen()
        sid = self.next_id
        self.next_id += 1
        n = len(offsets) - 1
        w = np.ones(len(indices), dtype=np.float32) if weights is None else np.asarray(weights, dtype=np.float32)
        self.pending.append((sid, gen.CSR(n, np.asarray(offsets, dtype=np.int64),
                                          np.asarray(indices, dtype=np.int32), w)))
        return sid

    def step(self):
        self._seen()
        if self.barrier is not None:
            self.barrier.wait(timeout=20)  # passes only when every device steps at the same time
        fin = 0
        for sid, g in self.pending:
            r = oracle.leiden(g, mode=oracle.SEQ)
            self.done.append((sid, r.membership, r.modularity, r.passes, int(r.membership.max()) + 1 if g.n else 0))
            fin += 1
        self.pending = []
        return fin

    def results(self, device=False):
        self._seen()
        out, self.done = self.done, []
        return out

    def close(self):
        self._seen()
        self.closed = True


def _graphs():
    gs = [gen.sbm(n, 4, 0.3, 0.01, seed=s) for s, n in enumerate((120, 40, 40, 40, 90, 60))]
    return gs


def test_requests_go_to_the_least_loaded_device():
    servers = {}
    make = lambda d: servers.setdefault(d, OracleServer(d))  # noqa: E731
    r = ServeRouter([0, 1], make_server=make, bind=_bind)
    try:
        gs = _graphs()
        placed, expect, load = [], [], [0, 0]
        for g in gs:
            k = min((0, 1), key=lambda j: (load[j], j))
            expect.append(k)
            load[k] += g.nnz
            placed.append(r.pick())
            r.submit(g.offsets, g.indices, g.weights)
        assert placed == expect and r.load == load
        assert len(set(placed)) == 2  # both devices took work
    finally:
        r.close()


def test_results_come_back_under_router_ids_and_release_the_load():
    servers = {}
    make = lambda d: servers.setdefault(d, OracleServer(d))  # noqa: E731
    r = ServeRouter([0, 1], make_server=make, bind=_bind)
    try:
        gs = _graphs()
        ids = [r.submit(g.offsets, g.indices, g.weights) for g in gs]
        assert ids == list(range(len(gs))) and r.busy()
        assert r.step() == len(gs)
        got = {rid: (memb, q, passes) for rid, memb, q, passes, _ in r.results()}
        assert sorted(got) == ids and not r.busy() and r.load == [0, 0]
        for rid, g in zip(ids, gs):
            ref = oracle.leiden(g, mode=oracle.SEQ)
            memb, q, passes = got[rid]
            assert np.array_equal(memb, ref.membership) and q == ref.modularity and passes == ref.passes
        assert r.results() == [] and r.step() == 0
    finally:
        r.close()
    assert all(s.closed for s in servers.values())


def test_each_device_has_its_own_bound_thread_and_steps_run_together():
    servers = {}
    barrier = threading.Barrier(3)
    make = lambda d: servers.setdefault(d, OracleServer(d, barrier))  # noqa: E731
    r = ServeRouter([0, 1, 2], make_server=make, bind=_bind)
    try:
        for g in _graphs():
            r.submit(g.offsets, g.indices, g.weights)
        assert r.step() == 6  # the barrier of three passes only if all steps run at once
        r.results()
    finally:
        r.close()
    threads = [s.threads for s in servers.values()]
    assert all(len(t) == 1 for t in threads)
    assert len(set.union(*threads)) == 3
    for d, s in servers.items():
        assert s.bound == {d}


def test_one_device_is_a_plain_server_and_no_device_is_refused():
    servers = {}
    make = lambda d: servers.setdefault(d, OracleServer(d))  # noqa: E731
    r = ServeRouter([0], make_server=make, bind=_bind)
    try:
        g = _graphs()[0]
        rid = r.submit(g.offsets, g.indices, None)
        r.step()
        (got,) = r.results()
        assert got[0] == rid and got[2] == oracle.leiden(g, mode=oracle.SEQ).modularity
    finally:
        r.close()
    with pytest.raises(ValueError):
        ServeRouter([], make_server=make, bind=_bind)


def test_close_shuts_every_device_thread_down_when_a_server_fails_to_close():
    class Failing(OracleServer):
        def close(self):
            raise RuntimeError("close failed")

    servers = {}
    make = lambda d: servers.setdefault(d, (Failing if d == 0 else OracleServer)(d))  # noqa: E731
    r = ServeRouter([0, 1], make_server=make, bind=_bind)
    pools = list(r._pools)
    with pytest.raises(RuntimeError):
        r.close()
    assert all(p._shutdown for p in pools) and r.servers == []
    assert servers[1].closed  # the other device's server was closed all the same
    r.close()  # a second close does nothing
