"""GB300 (sm_103a) Leiden community detection: Python binding of the C ABI.

The binding only marshals arguments to ``libleiden_gb300.so`` (declared in
``include/leiden.h``); every step of the method runs in the library's CUDA
kernels. PyTorch provides device memory and streams. There is no CPU
fallback: if the library is missing, every call raises.

Functions carry the C names (``leiden_create``, ``leiden_run``, ...);
``Leiden`` is a small convenience wrapper around a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "LEIDEN_HOST", "LEIDEN_DEVICE", "LEIDEN_ASYNC", "LEIDEN_DETERMINISTIC", "FLAG_VALIDATE",
    "FLAG_REFINE_SINGLE_SWEEP", "FLAG_TRACE", "FLAG_PROFILE", "FLAG_STEP_LAUNCHES",
    "FLAG_REFINE_LABELS", "FLAG_LOUVAIN", "FLAG_RANDOM_REFINE", "LeidenError", "Params", "Stats", "KernelProfile",
    "library", "leiden_params_default", "leiden_create", "leiden_run", "leiden_destroy", "leiden_modularity",
    "leiden_trace_get", "leiden_profile_get", "leiden_modularity_noalloc",
    "leiden_status_string", "leiden_last_error", "Leiden", "modularity", "leiden_batch_create",
    "leiden_batch_run", "leiden_batch_info", "LeidenBatch", "pack_batch", "ServerState", "leiden_server_create",
    "leiden_server_submit", "leiden_server_step", "leiden_server_next", "leiden_server_result", "leiden_server_info",
    "leiden_server_destroy", "LeidenServer", "leiden_disconnected", "disconnected", "leiden_csr_from_edges",
    "csr_from_edges", "FLAG_TEST_STALL_BARRIER", "leiden_test_fail_allocation", "Tuning", "leiden_tuning_default",
    "leiden_set_tuning", "leiden_get_tuning", "leiden_tuning_lookup", "TUNING_CACHE",
]

LEIDEN_HOST, LEIDEN_DEVICE = 0, 1
LEIDEN_ASYNC, LEIDEN_DETERMINISTIC = 0, 1
FLAG_VALIDATE, FLAG_REFINE_SINGLE_SWEEP, FLAG_TRACE, FLAG_PROFILE, FLAG_STEP_LAUNCHES = 1, 2, 4, 8, 16
FLAG_REFINE_LABELS, FLAG_LOUVAIN, FLAG_RANDOM_REFINE = 64, 128, 256
FLAG_TEST_STALL_BARRIER = 512  # testing aid: the persistent sweep's barrier wait runs out
PROFILE_CLASSES = 24
PROFILE_PHASES = ("move", "refine", "aggregate")
PROFILE_BINS = ("sweep", "thread", "tile16", "tile32", "warp", "block", "global", "unused")
TRACE_INIT, TRACE_MOVE, TRACE_REFINE, TRACE_COUNTS, TRACE_RENUMBER = 1, 2, 3, 4, 5
TRACE_AGG_OFF, TRACE_AGG_DEG, TRACE_AGG_IDX, TRACE_AGG_W, TRACE_DENDRO = 6, 7, 8, 9, 10
_TRACE_DTYPE = {1: np.int32, 2: np.int32, 3: np.int32, 4: np.int64, 5: np.int32, 6: np.int64, 7: np.int32,
                8: np.int32, 9: np.float64, 10: np.int32}


class LeidenError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [{status}]")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("resolution", ctypes.c_double), ("tolerance", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("max_iterations", ctypes.c_int32), ("max_passes", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("schedule_layers", ctypes.c_int32),
                ("schedule_buckets", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("move_iterations", ctypes.c_int32),
                ("refine_iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("communities", ctypes.c_int64), ("modularity", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_move", ctypes.c_double), ("ms_refine", ctypes.c_double), ("ms_aggregate", ctypes.c_double),
                ("ms_other", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class KernelProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("items", ctypes.c_int64), ("skipped", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("distinct", ctypes.c_int64), ("moved", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    """Launch shape of a handle (leiden_tuning): degree-bin bounds and the
    persistent sweep's grid; none changes a deterministic result."""
    _fields_ = [("thread_max_deg", ctypes.c_int32), ("warp_max_deg", ctypes.c_int32),
                ("block_max_deg", ctypes.c_int32), ("coop_blocks_per_sm", ctypes.c_int32),
                ("vertices_per_block", ctypes.c_int32), ("list_order_min_vertices", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]
    KEYS = ("thread_max_deg", "warp_max_deg", "block_max_deg", "coop_blocks_per_sm", "vertices_per_block",
            "list_order_min_vertices")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.KEYS}


# the autotuner's cache shipped with the package (LEIDEN_TUNING_CACHE overrides it)
TUNING_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


class ServerState(ctypes.Structure):
    _fields_ = [("waiting", ctypes.c_int32), ("in_flight", ctypes.c_int32), ("finished", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("union_vertices", ctypes.c_int64), ("union_entries", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("steps", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_LIB = None
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64


def library(build_if_missing: bool = False) -> ctypes.CDLL:
    """The loaded libleiden_gb300.so (raises if it is not built)."""
    global _LIB
    if _LIB is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"{_build.LIB} is not built; run __graft_entry__.build() (needs nvcc)")
        lib = ctypes.CDLL(_build.LIB)
        lib.leiden_params_default.argtypes = [ctypes.POINTER(Params)]
        lib.leiden_params_default.restype = None
        lib.leiden_create.argtypes = [ctypes.POINTER(_VP), _I64, _I64, _VP, _VP, _VP, _I32, _I32, _VP]
        lib.leiden_run.argtypes = [_VP, ctypes.POINTER(Params), _VP, _I32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(Stats)]
        lib.leiden_destroy.argtypes = [_VP]
        lib.leiden_modularity.argtypes = [_I64, _VP, _VP, _VP, _VP, ctypes.c_double, _VP,
                                          ctypes.POINTER(ctypes.c_double)]
        lib.leiden_modularity_noalloc.argtypes = [_I64, _VP, _VP, _VP, _VP, ctypes.c_double, _VP,
                                                  ctypes.POINTER(ctypes.c_double)]
        lib.leiden_modularity_noalloc.restype = ctypes.c_int
        lib.leiden_trace_get.argtypes = [_VP, _I32, _I32, _VP, ctypes.POINTER(_I64)]
        lib.leiden_profile_get.argtypes = [_VP, ctypes.POINTER(KernelProfile)]
        lib.leiden_batch_create.argtypes = [ctypes.POINTER(_VP), _I32, _VP, _I64, _VP, _VP, _VP, _I32, _I32, _VP]
        lib.leiden_batch_run.argtypes = [_VP, ctypes.POINTER(Params), _VP, _I32, _VP, ctypes.POINTER(Stats)]
        lib.leiden_batch_info.argtypes = [_VP, ctypes.POINTER(_I32), _VP, _VP]
        lib.leiden_server_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Params), _I64, _I64, _I32, _I64,
                                             _VP]
        lib.leiden_server_submit.argtypes = [_VP, _I64, _I64, _VP, _VP, _VP, _I32, ctypes.POINTER(_I64)]
        lib.leiden_server_step.argtypes = [_VP, ctypes.POINTER(_I32)]
        lib.leiden_server_next.argtypes = [_VP, ctypes.POINTER(_I64)]
        lib.leiden_server_result.argtypes = [_VP, _I64, _VP, _I32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(_I32), ctypes.POINTER(_I64)]
        lib.leiden_server_info.argtypes = [_VP, ctypes.POINTER(ServerState)]
        lib.leiden_server_destroy.argtypes = [_VP]
        lib.leiden_disconnected.argtypes = [_I64, _VP, _VP, _VP, _VP, ctypes.POINTER(_I64)]
        lib.leiden_tuning_default.argtypes = [ctypes.POINTER(Tuning)]
        lib.leiden_tuning_default.restype = None
        lib.leiden_set_tuning.argtypes = [_VP, ctypes.POINTER(Tuning)]
        lib.leiden_set_tuning.restype = ctypes.c_int
        lib.leiden_get_tuning.argtypes = [_VP, ctypes.POINTER(Tuning)]
        lib.leiden_get_tuning.restype = ctypes.c_int
        lib.leiden_tuning_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _I64, _I64, _I64,
                                             ctypes.POINTER(Tuning)]
        lib.leiden_tuning_lookup.restype = ctypes.c_int
        lib.leiden_test_fail_allocation.argtypes = [_I64]
        lib.leiden_test_fail_allocation.restype = ctypes.c_int
        lib.leiden_csr_from_edges.argtypes = [_I64, _I64, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, _VP, _VP, _VP, ctypes.POINTER(_I64), _VP]
        for f in (lib.leiden_create, lib.leiden_run, lib.leiden_destroy, lib.leiden_modularity,
                  lib.leiden_trace_get, lib.leiden_profile_get, lib.leiden_batch_create, lib.leiden_batch_run,
                  lib.leiden_batch_info, lib.leiden_server_create, lib.leiden_server_submit, lib.leiden_server_step,
                  lib.leiden_server_next, lib.leiden_server_result, lib.leiden_server_info,
                  lib.leiden_server_destroy, lib.leiden_disconnected):
            f.restype = ctypes.c_int
        lib.leiden_status_string.argtypes = [_I32]
        lib.leiden_status_string.restype = ctypes.c_char_p
        lib.leiden_last_error.argtypes = []
        lib.leiden_last_error.restype = ctypes.c_char_p
        _LIB = lib
    return _LIB


def _check(rc: int):
    if rc != 0:
        lib = library()
        raise LeidenError(rc, f"{lib.leiden_status_string(rc).decode()}: {lib.leiden_last_error().decode()}")


def leiden_status_string(status: int) -> str:
    return library().leiden_status_string(status).decode()


def leiden_last_error() -> str:
    return library().leiden_last_error().decode()


def leiden_params_default() -> Params:
    p = Params()
    library().leiden_params_default(ctypes.byref(p))
    return p


def leiden_create(n, nnz, offsets_ptr, indices_ptr, weights_ptr, where, validate, stream) -> int:
    h = _VP()
    _check(library().leiden_create(ctypes.byref(h), n, nnz, offsets_ptr, indices_ptr, weights_ptr, where,
                                   validate, stream))
    return h.value


def leiden_run(handle, params: Params, membership_ptr, where):
    q = ctypes.c_double(0.0)
    st = Stats()
    _check(library().leiden_run(handle, ctypes.byref(params), membership_ptr, where, ctypes.byref(q),
                                ctypes.byref(st)))
    return q.value, st


def leiden_batch_create(num_graphs, vtx_seg, nnz, offsets_ptr, indices_ptr, weights_ptr, where, validate,
                        stream) -> int:
    """vtx_seg: host int64 array of num_graphs+1 vertex offsets; indices local to each graph."""
    seg = np.ascontiguousarray(vtx_seg, dtype=np.int64)
    h = _VP()
    _check(library().leiden_batch_create(ctypes.byref(h), num_graphs, seg.ctypes.data_as(_VP), nnz, offsets_ptr,
                                         indices_ptr, weights_ptr, where, validate, stream))
    return h.value


def leiden_batch_run(handle, params: Params, membership_ptr, where, num_graphs: int):
    """Returns (per-graph modularity as a numpy array, Stats of the whole batch)."""
    q = np.zeros(max(num_graphs, 1), dtype=np.float64)
    st = Stats()
    _check(library().leiden_batch_run(handle, ctypes.byref(params), membership_ptr, where,
                                      q.ctypes.data_as(_VP), ctypes.byref(st)))
    return q[:num_graphs], st


def leiden_batch_info(handle):
    """(passes, communities) per graph of the last run, as numpy arrays."""
    g = _I32(0)
    _check(library().leiden_batch_info(handle, ctypes.byref(g), None, None))
    passes = np.zeros(max(g.value, 1), dtype=np.int32)
    comm = np.zeros(max(g.value, 1), dtype=np.int64)
    _check(library().leiden_batch_info(handle, None, passes.ctypes.data_as(_VP), comm.ctypes.data_as(_VP)))
    return passes[:g.value], comm[:g.value]


def leiden_server_create(params: Params, max_vertices, max_entries, max_graphs, device_budget, stream) -> int:
    h = _VP()
    _check(library().leiden_server_create(ctypes.byref(h), ctypes.byref(params), max_vertices, max_entries,
                                          max_graphs, device_budget, stream))
    return h.value


def leiden_server_submit(server, n, nnz, offsets_ptr, indices_ptr, weights_ptr, where) -> int:
    rid = _I64(0)
    _check(library().leiden_server_submit(server, n, nnz, offsets_ptr, indices_ptr, weights_ptr, where,
                                          ctypes.byref(rid)))
    return rid.value


def leiden_server_step(server) -> int:
    f = _I32(0)
    _check(library().leiden_server_step(server, ctypes.byref(f)))
    return f.value


def leiden_server_next(server) -> int:
    rid = _I64(0)
    _check(library().leiden_server_next(server, ctypes.byref(rid)))
    return rid.value


def leiden_server_result(server, rid, membership_ptr, where):
    """(modularity, passes, communities) of a finished graph; its labels go to membership_ptr."""
    q = ctypes.c_double(0.0)
    passes = _I32(0)
    comm = _I64(0)
    _check(library().leiden_server_result(server, rid, membership_ptr, where, ctypes.byref(q), ctypes.byref(passes),
                                          ctypes.byref(comm)))
    return q.value, passes.value, comm.value


def leiden_server_info(server) -> dict:
    st = ServerState()
    _check(library().leiden_server_info(server, ctypes.byref(st)))
    return st.as_dict()


def leiden_server_destroy(server) -> None:
    _check(library().leiden_server_destroy(server))


def leiden_tuning_default() -> Tuning:
    t = Tuning()
    library().leiden_tuning_default(ctypes.byref(t))
    return t


def leiden_set_tuning(handle, t: Tuning) -> None:
    _check(library().leiden_set_tuning(handle, ctypes.byref(t)))


def leiden_get_tuning(handle) -> Tuning:
    t = Tuning()
    _check(library().leiden_get_tuning(handle, ctypes.byref(t)))
    return t


def leiden_tuning_lookup(cache_path: str, gpu_name: str, n: int, nnz: int, max_degree: int):
    """The cache entry for the GPU and the graph's class, or None."""
    t = Tuning()
    rc = library().leiden_tuning_lookup(cache_path.encode(), gpu_name.encode(), n, nnz, max_degree, ctypes.byref(t))
    return t if rc == 0 else None


def _apply_cached_tuning(handle, n, nnz, max_degree):
    """Launch shape of a new handle from the autotuner cache (the package's,
    or LEIDEN_TUNING_CACHE's) for the current GPU and the graph's class; the
    library's defaults when there is no entry."""
    if os.environ.get("LEIDEN_TUNING_CACHE"):
        return  # leiden_create has applied it already
    if not os.path.exists(TUNING_CACHE):
        return
    import torch
    t = leiden_tuning_lookup(TUNING_CACHE, torch.cuda.get_device_name(), n, nnz, max_degree)
    if t is not None:
        leiden_set_tuning(handle, t)


def _set_tuning(handle, tuning=None, **kw):
    t = leiden_get_tuning(handle) if tuning is None else tuning
    if isinstance(t, dict):
        kw = {**t, **kw}
        t = leiden_get_tuning(handle)
    for k, v in kw.items():
        setattr(t, k, int(v))
    leiden_set_tuning(handle, t)


def _init_tuning(handle, tuning, off, n, nnz):
    if isinstance(tuning, str) and tuning == "cache":
        maxdeg = int((off[1:] - off[:-1]).max().item()) if n > 0 else 0
        _apply_cached_tuning(handle, n, nnz, maxdeg)
    elif tuning is None:
        leiden_set_tuning(handle, leiden_tuning_default())
    else:
        _set_tuning(handle, tuning)


def leiden_test_fail_allocation(after: int) -> None:
    """Testing aid: the handle allocation after `after` more successful ones
    fails with LEIDEN_ERR_OOM (negative: no injection)."""
    _check(library().leiden_test_fail_allocation(after))


def leiden_destroy(handle) -> None:
    _check(library().leiden_destroy(handle))


def leiden_modularity(n, offsets_ptr, indices_ptr, weights_ptr, membership_ptr, gamma, stream) -> float:
    q = ctypes.c_double(0.0)
    _check(library().leiden_modularity(n, offsets_ptr, indices_ptr, weights_ptr, membership_ptr, gamma, stream,
                                       ctypes.byref(q)))
    return q.value


def leiden_disconnected(n, offsets_ptr, indices_ptr, membership_ptr, stream) -> int:
    c = _I64(0)
    _check(library().leiden_disconnected(n, offsets_ptr, indices_ptr, membership_ptr, stream, ctypes.byref(c)))
    return c.value


def leiden_csr_from_edges(n, m, src_ptr, dst_ptr, w_ptr, where, drop_self_loops, combine, offsets_ptr, indices_ptr,
                          weights_ptr, capacity, stream) -> int:
    """Edge list to symmetric CSR (see include/leiden.h); returns the entry count."""
    nnz = _I64(capacity)
    _check(library().leiden_csr_from_edges(n, m, src_ptr, dst_ptr, w_ptr, where, drop_self_loops, combine, offsets_ptr,
                                           indices_ptr, weights_ptr, ctypes.byref(nnz), stream))
    return nnz.value


def leiden_modularity_noalloc(n, offsets_ptr, indices_ptr, weights_ptr, membership_ptr, gamma, stream) -> float:
    """leiden_modularity without device allocation (static scratch, n <= 2**20)."""
    q = ctypes.c_double(0.0)
    _check(library().leiden_modularity_noalloc(n, offsets_ptr, indices_ptr, weights_ptr, membership_ptr, gamma,
                                               stream, ctypes.byref(q)))
    return q.value


def leiden_trace_get(handle, pass_: int, what: int):
    cnt = _I64(0)
    _check(library().leiden_trace_get(handle, pass_, what, None, ctypes.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), dtype=_TRACE_DTYPE[what])
    _check(library().leiden_trace_get(handle, pass_, what, out.ctypes.data_as(_VP), ctypes.byref(cnt)))
    return out[:cnt.value]


def leiden_profile_get(handle):
    """Per-class profile of the last profiled run: {(phase, bin): dict}."""
    arr = (KernelProfile * PROFILE_CLASSES)()
    _check(library().leiden_profile_get(handle, arr))
    out = {}
    for k in range(PROFILE_CLASSES):
        e = arr[k]
        if e.launches:
            out[(PROFILE_PHASES[k // 8], PROFILE_BINS[k % 8])] = {f: getattr(e, f) for f, _ in e._fields_}
    return out


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _VP(s.cuda_stream)


def _ptr(t):
    return _VP(t.data_ptr()) if t is not None else _VP(0)


class Leiden:
    """A graph resident on the GPU, ready for repeated leiden_run calls.

    ``offsets``/``indices``/``weights`` are a symmetric CSR, as numpy arrays
    or torch tensors (CPU or CUDA). ``run`` returns (membership, modularity,
    stats) with membership a torch.int32 CUDA tensor of canonical labels.
    """

    def __init__(self, offsets, indices, weights=None, validate: bool = False, stream=None, tuning="cache"):
        """tuning: "cache" (the autotuner cache's entry for this GPU and the
        graph's class, else the defaults), None (the defaults), or a Tuning
        or dict of its fields."""
        import torch
        self._torch = torch
        self.stream = stream
        dev = torch.device("cuda", torch.cuda.current_device())
        off = torch.as_tensor(offsets, dtype=torch.int64).to(dev).contiguous()
        idx = torch.as_tensor(indices, dtype=torch.int32).to(dev).contiguous()
        w = None if weights is None else torch.as_tensor(weights, dtype=torch.float32).to(dev).contiguous()
        self.n = int(off.numel() - 1)
        self.nnz = int(idx.numel())
        self.handle = leiden_create(self.n, self.nnz, _ptr(off), _ptr(idx), _ptr(w), LEIDEN_DEVICE,
                                    int(validate), _stream_ptr(stream))
        self.device = dev
        self._input = (off, idx, w)  # kept for modularity checks
        _init_tuning(self.handle, tuning, off, self.n, self.nnz)

    def set_tuning(self, tuning=None, **kw):
        """Set the launch shape: a Tuning, or fields by name over the current one."""
        _set_tuning(self.handle, tuning, **kw)

    def tuning(self) -> dict:
        return leiden_get_tuning(self.handle).as_dict()

    def run(self, mode: int = LEIDEN_ASYNC, trace: bool = False, **kw):
        p = leiden_params_default()
        p.mode = mode
        if trace:
            p.flags |= FLAG_TRACE
        for k, v in kw.items():
            if k == "flags":
                p.flags |= int(v)
            else:
                setattr(p, k, v)
        memb = self._torch.empty(max(self.n, 1), dtype=self._torch.int32, device=self.device)
        q, st = leiden_run(self.handle, p, _ptr(memb), LEIDEN_DEVICE)
        return memb[:self.n], q, st

    def trace(self, pass_: int, what: int):
        return leiden_trace_get(self.handle, pass_, what)

    def profile(self):
        return leiden_profile_get(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            leiden_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_batch(graphs):
    """Pack CSRs (objects with offsets/indices/weights numpy arrays) into the
    segmented layout of leiden_batch_create: (vtx_seg, offsets, indices,
    weights) with offsets shifted and indices kept local to each graph."""
    ns = [int(len(g.offsets) - 1) for g in graphs]
    ms = [int(g.offsets[-1]) for g in graphs]
    vseg = np.zeros(len(graphs) + 1, dtype=np.int64)
    vseg[1:] = np.cumsum(ns)
    eseg = np.zeros(len(graphs) + 1, dtype=np.int64)
    eseg[1:] = np.cumsum(ms)
    off = np.empty(int(vseg[-1]) + 1, dtype=np.int64)
    off[-1] = eseg[-1]
    for k, g in enumerate(graphs):
        off[vseg[k]:vseg[k + 1]] = np.asarray(g.offsets[:-1], dtype=np.int64) + eseg[k]
    idx = np.concatenate([np.asarray(g.indices, dtype=np.int32) for g in graphs]) if graphs else \
        np.zeros(0, np.int32)
    w = np.concatenate([np.asarray(g.weights, dtype=np.float32) for g in graphs]) if graphs else \
        np.zeros(0, np.float32)
    return vseg, off, idx, w


class LeidenBatch:
    """Many graphs resident on the GPU as one segmented CSR, solved together.

    Takes the packed layout of ``pack_batch``. ``run`` returns (membership,
    per-graph modularity, stats); membership holds every graph's labels,
    local to the graph, in the packed vertex order.
    """

    def __init__(self, vtx_seg, offsets, indices, weights=None, validate: bool = False, stream=None,
                 tuning="cache"):
        import torch
        self._torch = torch
        self.stream = stream
        dev = torch.device("cuda", torch.cuda.current_device())
        self.vtx_seg = np.ascontiguousarray(vtx_seg, dtype=np.int64)
        self.num_graphs = int(len(self.vtx_seg) - 1)
        off = torch.as_tensor(offsets, dtype=torch.int64).to(dev).contiguous()
        idx = torch.as_tensor(indices, dtype=torch.int32).to(dev).contiguous()
        w = None if weights is None else torch.as_tensor(weights, dtype=torch.float32).to(dev).contiguous()
        self.n = int(off.numel() - 1)
        self.nnz = int(idx.numel())
        self.handle = leiden_batch_create(self.num_graphs, self.vtx_seg, self.nnz, _ptr(off), _ptr(idx), _ptr(w),
                                          LEIDEN_DEVICE, int(validate), _stream_ptr(stream))
        self.device = dev
        _init_tuning(self.handle, tuning, off, self.n, self.nnz)

    def set_tuning(self, tuning=None, **kw):
        _set_tuning(self.handle, tuning, **kw)

    def tuning(self) -> dict:
        return leiden_get_tuning(self.handle).as_dict()

    def run(self, mode: int = LEIDEN_ASYNC, **kw):
        p = leiden_params_default()
        p.mode = mode
        for k, v in kw.items():
            if k == "flags":
                p.flags |= int(v)
            else:
                setattr(p, k, v)
        memb = self._torch.empty(max(self.n, 1), dtype=self._torch.int32, device=self.device)
        q, st = leiden_batch_run(self.handle, p, _ptr(memb), LEIDEN_DEVICE, self.num_graphs)
        return memb[:self.n], q, st

    def info(self):
        return leiden_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            leiden_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LeidenServer:
    """Serving with continuous batching: submit graphs as they arrive, call
    ``step`` (admission at the pass boundary, then one pass of every graph in
    flight), collect finished graphs with ``results``. Graphs are CSRs as
    numpy arrays (copied from host) or CUDA tensors (copied on the device).
    """

    def __init__(self, max_vertices: int, max_entries: int, max_graphs: int = 1024, device_budget: int = 0,
                 mode: int = LEIDEN_ASYNC, stream=None, **kw):
        import torch
        self._torch = torch
        p = leiden_params_default()
        p.mode = mode
        for k, v in kw.items():
            setattr(p, k, v)
        self.stream = stream
        self.handle = leiden_server_create(p, max_vertices, max_entries, max_graphs, device_budget,
                                           _stream_ptr(stream))
        self.sizes = {}

    def submit(self, offsets, indices, weights=None) -> int:
        t = self._torch
        if isinstance(offsets, t.Tensor) and offsets.is_cuda:
            off = offsets.to(t.int64).contiguous()
            idx = indices.to(t.int32).contiguous()
            w = None if weights is None else weights.to(t.float32).contiguous()
            n, m = int(off.numel() - 1), int(idx.numel())
            rid = leiden_server_submit(self.handle, n, m, _ptr(off), _ptr(idx), _ptr(w), LEIDEN_DEVICE)
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            idx = np.ascontiguousarray(indices, dtype=np.int32)
            w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
            n, m = int(len(off) - 1), int(len(idx))
            rid = leiden_server_submit(self.handle, n, m, off.ctypes.data_as(_VP), idx.ctypes.data_as(_VP),
                                       None if w is None else w.ctypes.data_as(_VP), LEIDEN_HOST)
        self.sizes[rid] = n
        return rid

    def step(self) -> int:
        return leiden_server_step(self.handle)

    def results(self, device: bool = False):
        """Drain finished graphs: list of (id, membership, modularity, passes, communities)."""
        out = []
        while True:
            rid = leiden_server_next(self.handle)
            if rid < 0:
                return out
            n = self.sizes.pop(rid)
            if device:
                memb = self._torch.empty(max(n, 1), dtype=self._torch.int32, device="cuda")
                q, passes, comm = leiden_server_result(self.handle, rid, _ptr(memb), LEIDEN_DEVICE)
                memb = memb[:n]
            else:
                memb = np.zeros(max(n, 1), dtype=np.int32)
                q, passes, comm = leiden_server_result(self.handle, rid, memb.ctypes.data_as(_VP), LEIDEN_HOST)
                memb = memb[:n]
            out.append((rid, memb, q, passes, comm))

    def info(self) -> dict:
        return leiden_server_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            leiden_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csr_from_edges(n: int, src, dst, weights=None, drop_self_loops: bool = False, combine: str = "sum",
                   stream=None):
    """Symmetric CSR (offsets int64[n+1], indices int32, weights float32, as
    CUDA tensors) of an undirected edge list held in CUDA tensors (src, dst
    int32[m], weights float32[m] or None for unit weights), built on the GPU:
    reverse entries added, duplicates merged (combine "sum" or "max"),
    self-loops kept as one entry or dropped, rows sorted by target."""
    import torch
    m = int(src.numel())
    dev = src.device
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    idx = torch.empty(max(2 * m, 1), dtype=torch.int32, device=dev)
    w = torch.empty(max(2 * m, 1), dtype=torch.float32, device=dev)
    nnz = leiden_csr_from_edges(n, m, _ptr(src), _ptr(dst), _ptr(weights) if weights is not None else None,
                                LEIDEN_DEVICE, 1 if drop_self_loops else 0, 0 if combine == "sum" else 1, _ptr(off),
                                _ptr(idx), _ptr(w), 2 * m, _stream_ptr(stream))
    return off, idx[:nnz], w[:nnz]


def disconnected(offsets, indices, membership, stream=None) -> int:
    """Communities of ``membership`` that are not connected (Algorithm 5), on
    a CSR held in CUDA tensors."""
    n = int(offsets.numel() - 1)
    return leiden_disconnected(n, _ptr(offsets), _ptr(indices), _ptr(membership), _stream_ptr(stream))


def modularity(offsets, indices, weights, membership, resolution: float = 1.0, stream=None) -> float:
    """Eq. 1 of ``membership`` (labels in [0, n)) on a CSR held in CUDA tensors."""
    n = int(offsets.numel() - 1)
    return leiden_modularity(n, _ptr(offsets), _ptr(indices), _ptr(weights), _ptr(membership), resolution,
                             _stream_ptr(stream))

from . import shard  # noqa: E402  (batches on several GPUs; uses the names above)
