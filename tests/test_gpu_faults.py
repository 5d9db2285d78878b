"""GPU tests of the failure paths, made without faulting the GPU.

A persistent sweep's grid barrier waits a bounded time: with the testing
flag LEIDEN_FLAG_TEST_STALL_BARRIER one block ends without arriving, the
others give up after a short bounded wait, the launch ends, and leiden_run
returns LEIDEN_ERR_TIMEOUT; the same handle then runs normally. Device
allocation failures are injected on the host (leiden_test_fail_allocation):
every create or run either succeeds or returns LEIDEN_ERR_OOM, and the
library works normally afterwards.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2312_13936_gb300 as lg

pytestmark = pytest.mark.gpu


def test_barrier_timeout_returns_status_and_handle_recovers():
    g = gen.road(100)  # 10,000 vertices: persistent sweeps of several blocks
    ref = oracle.leiden(g, mode=oracle.SYNC)
    h = lg.Leiden(g.offsets, g.indices, g.weights)
    try:
        for _ in range(2):
            with pytest.raises(lg.LeidenError) as e:
                h.run(mode=lg.LEIDEN_DETERMINISTIC, flags=lg.FLAG_TEST_STALL_BARRIER)
            assert e.value.status == -5
            assert "timed out" in lg.leiden_last_error()
            memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC)
            assert np.array_equal(memb.cpu().numpy(), ref.membership)
            memb, q, st = h.run(mode=lg.LEIDEN_ASYNC)
            assert oracle.disconnected(g, memb.cpu().numpy())[0] == 0
    finally:
        h.close()


def test_injected_allocation_failures_leave_the_library_usable():
    g = gen.sbm(3000, 12, 0.04, 0.002, seed=4)
    ref = oracle.leiden(g, mode=oracle.SYNC)
    outcomes = {"create": 0, "run": 0, "ok": 0}
    try:
        for k in range(0, 160, 3):
            lg.leiden_test_fail_allocation(k)
            h = None
            try:
                h = lg.Leiden(g.offsets, g.indices, g.weights)
                memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC)
                assert np.array_equal(memb.cpu().numpy(), ref.membership)
                outcomes["ok"] += 1
            except lg.LeidenError as e:
                assert e.status == -3, e
                assert "injected" in lg.leiden_last_error()
                outcomes["run" if h is not None else "create"] += 1
            finally:
                lg.leiden_test_fail_allocation(-1)
            if h is not None:  # the handle that saw the failure runs normally now
                memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC)
                assert np.array_equal(memb.cpu().numpy(), ref.membership), k
                h.close()
    finally:
        lg.leiden_test_fail_allocation(-1)
    assert outcomes["create"] > 0 and outcomes["run"] > 0 and outcomes["ok"] > 0, outcomes


def test_iteration_limit_beyond_the_barrier_count_is_refused():
    """The persistent sweep's grid barrier counts arrivals in 32 bits: an
    iteration limit under which one phase could count past that is refused
    (LEIDEN_ERR_INVALID) before any work, by leiden_run and by
    leiden_server_create, and the handle then runs normally."""
    g = gen.road(60)
    ref = oracle.leiden(g, mode=oracle.SYNC)
    h = lg.Leiden(g.offsets, g.indices, g.weights)
    try:
        for mode in (lg.LEIDEN_ASYNC, lg.LEIDEN_DETERMINISTIC):
            with pytest.raises(lg.LeidenError) as e:
                h.run(mode=mode, max_iterations=2_000_000_000)
            assert e.value.status == -1 and "barrier" in lg.leiden_last_error()
            with pytest.raises(lg.LeidenError):
                h.run(mode=mode, max_iterations=20_000, schedule_layers=1000)
        memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC, max_iterations=200)  # well inside the count
        assert np.array_equal(memb.cpu().numpy(), oracle.leiden(g, mode=oracle.SYNC, max_iterations=200).membership)
        memb, q, st = h.run(mode=lg.LEIDEN_DETERMINISTIC)
        assert np.array_equal(memb.cpu().numpy(), ref.membership)
    finally:
        h.close()
    with pytest.raises(lg.LeidenError):
        lg.LeidenServer(1000, 10000, mode=lg.LEIDEN_DETERMINISTIC, max_iterations=2_000_000_000)
