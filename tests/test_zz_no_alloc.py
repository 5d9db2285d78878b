"""leiden_modularity_noalloc: the allocation-free modularity entry point.

Called through the C ABI, it must give the same score as leiden_modularity
(which takes scratch from the allocator) on two calls in a row -- the second
call reuses the static scratch the first one left behind -- and reject a
vertex count beyond its fixed scratch. This file is collected last so that a
failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import gen
import paper_2312_13936_gb300 as lg

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9  # the modularity tolerance of the other GPU tests


def _dev(a, torch):
    return torch.as_tensor(a).to("cuda").contiguous()


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    g = gen.road(300)  # 90,000 vertices, integer weights
    off, idx, w = (_dev(x, torch) for x in (g.offsets, g.indices, g.weights))
    h = lg.Leiden(off, idx, w)
    memb_leiden, _, _ = h.run()
    h.close()
    rng = np.random.default_rng(5)
    labelings = [memb_leiden, _dev(rng.integers(0, 500, g.n).astype(np.int32), torch)]
    stream = lg._stream_ptr(None)
    vp = ctypes.c_void_p
    for memb in labelings:  # two calls in a row on the shared scratch
        args = (g.n, vp(off.data_ptr()), vp(idx.data_ptr()), vp(w.data_ptr()), vp(memb.data_ptr()), 1.0, stream)
        q_alloc = lg.leiden_modularity(*args)
        q_static = lg.leiden_modularity_noalloc(*args)
        assert abs(q_static - q_alloc) <= REL_TOL * max(1.0, abs(q_alloc)), (q_static, q_alloc)


def test_noalloc_rejects_more_vertices_than_its_scratch():
    n = (1 << 20) + 1
    with pytest.raises(lg.LeidenError) as e:
        lg.leiden_modularity_noalloc(n, ctypes.c_void_p(16), ctypes.c_void_p(16), None, ctypes.c_void_p(16), 1.0,
                                     None)
    assert e.value.status == -1
    assert "exceeds" in lg.leiden_last_error()
