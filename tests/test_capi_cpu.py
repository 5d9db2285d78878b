"""The C-ABI library loads and exports every function include/leiden.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2312_13936_gb300 as lg

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "leiden.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(leiden_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("leiden_create", "leiden_run", "leiden_destroy", "leiden_modularity", "leiden_trace_get",
              "leiden_status_string", "leiden_last_error", "leiden_params_default"):
        assert f in names


def test_library_exports_every_declared_symbol():
    lib = lg.library(build_if_missing=True)
    for f in declared_functions():
        assert hasattr(lib, f), f"{f} missing from {lg._build.LIB}"


def test_host_only_entry_points():
    lib = lg.library(build_if_missing=True)
    p = lg.leiden_params_default()
    assert (p.resolution, p.tolerance, p.aggregation_tolerance, p.tolerance_drop) == (1.0, 0.01, 0.8, 10.0)
    assert (p.max_iterations, p.max_passes, p.mode, p.schedule_layers, p.schedule_buckets) == (20, 10, 0, 0, 16)
    assert lg.leiden_status_string(0) == "LEIDEN_OK"
    assert lg.leiden_status_string(-7) == "LEIDEN_ERR_OVERFLOW"
    # argument checks that fail before any device work
    h = ctypes.c_void_p()
    assert lib.leiden_create(None, 0, 0, None, None, None, 0, 0, None) == -1
    assert lib.leiden_create(ctypes.byref(h), -1, 0, None, None, None, 0, 0, None) == -1
    assert lib.leiden_run(None, None, None, 0, None, None) == -1
    assert lib.leiden_destroy(None) == 0


def test_argument_checks_before_device_work():
    """Every entry point rejects malformed arguments on the host, before any
    device call, with LEIDEN_ERR_INVALID and a one-line leiden_last_error;
    empty inputs of the stateless entry points succeed without a device."""
    import numpy as np
    lib = lg.library(build_if_missing=True)
    INV = -1
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    p = lg.leiden_params_default()
    i64 = ctypes.c_int64()

    def bad(rc):
        assert rc == INV
        assert lib.leiden_last_error()  # a description is left behind

    # single graph: bad where, huge n, missing indices, host offsets that do not frame nnz
    off = np.array([0, 1, 2], np.int64)
    idx = np.array([1, 0], np.int32)
    bad(lib.leiden_create(ctypes.byref(h), 2, 2, vp(off), vp(idx), None, 7, 0, None))
    bad(lib.leiden_create(ctypes.byref(h), 1 << 31, 2, vp(off), vp(idx), None, 0, 0, None))
    bad(lib.leiden_create(ctypes.byref(h), 2, 2, vp(off), None, None, 0, 0, None))
    bad(lib.leiden_create(ctypes.byref(h), 2, 3, vp(off), vp(idx), None, 0, 0, None))
    bad(lib.leiden_create(ctypes.byref(h), 2, 2, vp(np.array([1, 1, 2], np.int64)), vp(idx), None, 0, 0, None))
    assert h.value is None
    # batch: no graphs, vtx_seg not starting at 0 or decreasing, offsets not framing nnz
    bad(lib.leiden_batch_create(ctypes.byref(h), 0, vp(np.array([0], np.int64)), 0, vp(off), None, None, 0, 0,
                                None))
    bad(lib.leiden_batch_create(ctypes.byref(h), 1, vp(np.array([1, 2], np.int64)), 2, vp(off), vp(idx), None,
                                0, 0, None))
    bad(lib.leiden_batch_create(ctypes.byref(h), 2, vp(np.array([0, 2, 1], np.int64)), 2, vp(off), vp(idx),
                                None, 0, 0, None))
    bad(lib.leiden_batch_create(ctypes.byref(h), 1, vp(np.array([0, 2], np.int64)), 1, vp(off), vp(idx), None,
                                0, 0, None))
    # handles that are NULL
    bad(lib.leiden_batch_run(None, ctypes.byref(p), None, 0, None, None))
    bad(lib.leiden_batch_info(None, None, None, None))
    bad(lib.leiden_trace_get(None, 0, 0, None, ctypes.byref(i64)))
    bad(lib.leiden_profile_get(None, None))
    bad(lib.leiden_server_create(None, ctypes.byref(p), 10, 10, 1, 0, None))
    bad(lib.leiden_server_create(ctypes.byref(h), None, 10, 10, 1, 0, None))
    bad(lib.leiden_server_submit(None, 2, 2, vp(off), vp(idx), None, 0, ctypes.byref(i64)))
    bad(lib.leiden_server_step(None, None))
    bad(lib.leiden_server_next(None, ctypes.byref(i64)))
    bad(lib.leiden_server_result(None, 0, None, 0, None, None, None))
    bad(lib.leiden_server_info(None, None))
    assert lib.leiden_server_destroy(None) == 0
    # stateless entry points
    q = ctypes.c_double(5.0)
    bad(lib.leiden_modularity(-1, None, None, None, None, 1.0, None, ctypes.byref(q)))
    bad(lib.leiden_modularity(2, vp(off), vp(idx), None, None, 1.0, None, ctypes.byref(q)))
    bad(lib.leiden_modularity(2, vp(off), vp(idx), None, vp(idx), 1.0, None, None))
    bad(lib.leiden_modularity_noalloc(-1, None, None, None, None, 1.0, None, ctypes.byref(q)))
    bad(lib.leiden_modularity_noalloc(1 << 21, vp(off), vp(idx), None, vp(idx), 1.0, None, ctypes.byref(q)))
    bad(lib.leiden_disconnected(-1, None, None, None, None, ctypes.byref(i64)))
    bad(lib.leiden_disconnected(2, vp(off), None, vp(idx), None, ctypes.byref(i64)))
    assert lib.leiden_modularity(0, None, None, None, None, 1.0, None, ctypes.byref(q)) == 0 and q.value == 0.0
    q.value = 5.0
    assert lib.leiden_modularity_noalloc(0, None, None, None, None, 1.0, None, ctypes.byref(q)) == 0
    assert q.value == 0.0
    i64.value = 9
    assert lib.leiden_disconnected(0, None, None, None, None, ctypes.byref(i64)) == 0 and i64.value == 0
    # edge list to CSR: negative n, unknown combine or where, no nnz slot, missing sources
    src = np.array([0], np.int32)
    o3 = np.zeros(3, np.int64)
    i64.value = 4
    bad(lib.leiden_csr_from_edges(-1, 1, vp(src), vp(src), None, 0, 0, 0, vp(o3), None, None, ctypes.byref(i64),
                                  None))
    bad(lib.leiden_csr_from_edges(2, 1, vp(src), vp(src), None, 0, 0, 2, vp(o3), None, None, ctypes.byref(i64),
                                  None))
    bad(lib.leiden_csr_from_edges(2, 1, vp(src), vp(src), None, 3, 0, 0, vp(o3), None, None, ctypes.byref(i64),
                                  None))
    bad(lib.leiden_csr_from_edges(2, 1, vp(src), vp(src), None, 0, 0, 0, vp(o3), None, None, None, None))
    bad(lib.leiden_csr_from_edges(2, 1, None, vp(src), None, 0, 0, 0, vp(o3), None, None, ctypes.byref(i64),
                                  None))


def test_last_error_is_per_thread():
    """leiden_last_error describes the last failure of the calling thread."""
    import threading
    lib = lg.library(build_if_missing=True)
    seen = {}

    def worker():
        assert lib.leiden_create(None, 0, 0, None, None, None, 0, 0, None) == -1
        seen["worker"] = lib.leiden_last_error().decode()

    h = ctypes.c_void_p()
    assert lib.leiden_batch_create(ctypes.byref(h), 0, None, 0, None, None, None, 0, 0, None) == -1
    t = threading.Thread(target=worker)
    t.start()
    t.join()
    mine = lib.leiden_last_error().decode()
    assert "out is NULL" in seen["worker"]
    assert "batch" in mine and mine != seen["worker"]


def test_plain_c_consumer(tmp_path):
    """A C99 program includes the header, links the library and calls its
    host-only entry points: the boundary needs no C++ or Python on the caller's
    side."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    lg.library(build_if_missing=True)
    lib = lg._build.LIB
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "leiden.h"
int main(void) {
    leiden_params p;
    leiden_params_default(&p);
    leiden_graph_t g = 0;
    leiden_status s = leiden_create(&g, -1, 0, NULL, NULL, NULL, LEIDEN_HOST, 0, NULL);
    printf("%g %d %d %s %s|%s\n", p.resolution, p.max_passes, p.max_iterations, leiden_status_string(s),
           leiden_status_string(LEIDEN_OK), leiden_last_error());
    return (s == LEIDEN_ERR_INVALID && g == NULL && strlen(leiden_last_error()) > 0) ? 0 : 1;
}
''')
    exe = tmp_path / "consumer"
    inc = os.path.join(os.path.dirname(HEADER))
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), lib, "-o", str(exe),
                        f"-Wl,-rpath,{os.path.dirname(lib)}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("1 10 20 LEIDEN_ERR_INVALID LEIDEN_OK|")
