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
