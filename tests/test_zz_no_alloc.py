"""leiden_modularity_noalloc: the allocation-free modularity entry point.

Some callers cannot allocate device memory when they need a score: a host
framework that owns all device memory through its own pool, a process at its
memory cap, or a latency-critical path that must not call an allocator.
Called through the C ABI, the entry point must give the same Eq. 1 score as
leiden_modularity (which takes its scratch from the allocator) and as the
oracle's definition, on calls in a row -- later calls reuse the static
scratch earlier ones left behind, including a small graph right after a
large one -- reject labels outside [0, n) and then still score correctly,
and reject a vertex count beyond its fixed scratch. This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
import paper_2312_13936_gb300 as lg

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9  # the modularity tolerance of the other GPU tests


def _dev(a, torch):
    return torch.as_tensor(a).to("cuda").contiguous()


def _args(g, dev, memb, stream):
    vp = ctypes.c_void_p
    return (g.n, vp(dev[0].data_ptr()), vp(dev[1].data_ptr()), vp(dev[2].data_ptr()), vp(memb.data_ptr()), 1.0,
            stream)


def test_noalloc_matches_allocating_entry_point_and_oracle_twice():
    import torch
    big = gen.road(300)  # 90,000 vertices, integer weights
    small = gen.ring_of_cliques(5, 6)
    stream = lg._stream_ptr(None)
    h = lg.Leiden(big.offsets, big.indices, big.weights)
    memb_leiden, _, _ = h.run()
    h.close()
    rng = np.random.default_rng(5)
    cases = [(big, memb_leiden.cpu().numpy()), (big, rng.integers(0, 500, big.n).astype(np.int32)),
             (small, np.repeat(np.arange(6), 5).astype(np.int32)), (small, np.zeros(small.n, np.int32))]
    for g, memb in cases:  # calls in a row on the shared scratch, a small graph after the large one
        dev = [_dev(x, torch) for x in (g.offsets, g.indices, g.weights)]
        m = _dev(memb, torch)
        q_alloc = lg.leiden_modularity(*_args(g, dev, m, stream))
        q_static = lg.leiden_modularity_noalloc(*_args(g, dev, m, stream))
        q_ref = oracle.modularity(g, memb)
        assert abs(q_static - q_alloc) <= REL_TOL * max(1.0, abs(q_alloc)), (q_static, q_alloc)
        assert abs(q_static - q_ref) <= REL_TOL * max(1.0, abs(q_ref)), (q_static, q_ref)


def test_noalloc_rejects_labels_out_of_range_then_scores_again():
    import torch
    g = gen.road(60)
    stream = lg._stream_ptr(None)
    dev = [_dev(x, torch) for x in (g.offsets, g.indices, g.weights)]
    bad = np.zeros(g.n, np.int32)
    bad[17] = g.n  # one label outside [0, n)
    with pytest.raises(lg.LeidenError) as e:
        lg.leiden_modularity_noalloc(*_args(g, dev, _dev(bad, torch), stream))
    assert e.value.status == -1
    good = (np.arange(g.n) // 7).astype(np.int32)
    q = lg.leiden_modularity_noalloc(*_args(g, dev, _dev(good, torch), stream))
    q_ref = oracle.modularity(g, good)
    assert abs(q - q_ref) <= REL_TOL * max(1.0, abs(q_ref)), (q, q_ref)


def test_noalloc_rejects_more_vertices_than_its_scratch():
    n = (1 << 20) + 1
    with pytest.raises(lg.LeidenError) as e:
        lg.leiden_modularity_noalloc(n, ctypes.c_void_p(16), ctypes.c_void_p(16), None, ctypes.c_void_p(16), 1.0,
                                     None)
    assert e.value.status == -1
    assert "exceeds" in lg.leiden_last_error()
