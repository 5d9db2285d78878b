"""Leiden oracle -- TEST INFRASTRUCTURE ONLY.

Plain sequential CPU restatement of the GVE-Leiden method (Algorithms 1-4,
Eq. 1-2, Algorithm 5) in ``leiden_oracle.c``. Only ``tests/``, the package's
``__graft_entry__.smoke()`` check and ``bench.py``'s CPU-baseline / reference
leg may import this module. It shares no code with the CUDA implementation.

Modes: ``SEQ`` (sequential in-place moves, fp64) is the quality reference for
the GPU's asynchronous mode; ``SYNC`` (layered synchronous sweeps with exact
int64 decisions) is the bit-exact reference for the GPU's deterministic mode.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leiden_oracle.c")
_SO = os.path.join(_HERE, "libleiden_oracle.so")

SEQ, SYNC = 0, 1
REFINE_SINGLE_SWEEP = 1
NO_PRUNE = 2  # SEQ local-moving visits every vertex in every sweep (tests only)
REFINE_LABELS = 4  # refine-based super-vertex labels (Section 4.1)
LOUVAIN = 8  # no refinement: the Louvain method of the paper's comparison (Section 5)
RANDOM_REFINE = 16  # randomized refinement (Sections 3.4, 4.1), SEQ mode only

T_INIT_LABELS, T_MOVE, T_REFINE, T_COUNTS, T_RENUMBER = 1, 2, 3, 4, 5
T_AGG_OFF, T_AGG_DEG, T_AGG_IDX, T_AGG_W, T_DENDRO = 6, 7, 8, 9, 10
_TRACE_DTYPE = {
    T_INIT_LABELS: np.int32, T_MOVE: np.int32, T_REFINE: np.int32, T_COUNTS: np.int64,
    T_RENUMBER: np.int32, T_AGG_OFF: np.int64, T_AGG_DEG: np.int32, T_AGG_IDX: np.int32,
    T_AGG_W: np.float64, T_DENDRO: np.int32,
}

OK, ERR_INVALID, ERR_OOM, ERR_UNSUPPORTED, ERR_OVERFLOW = 0, -1, -3, -6, -7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE fp64, no contraction, no fast-math)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp,
                    "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("resolution", ctypes.c_double), ("tolerance", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("max_iterations", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("schedule_layers", ctypes.c_int32), ("schedule_buckets", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.c_int64)
_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.og_leiden.argtypes = [i64, vp, vp, vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(dbl),
                                  ctypes.POINTER(i32), _TRACE_FN, vp]
        lib.og_leiden.restype = ctypes.c_int
        lib.og_params_default.argtypes = [ctypes.POINTER(_Params)]
        lib.og_modularity.argtypes = [i64, vp, vp, vp, vp, dbl]
        lib.og_modularity.restype = dbl
        lib.og_modularity_holey.argtypes = [i64, vp, vp, vp, vp, vp, dbl]
        lib.og_modularity_holey.restype = dbl
        lib.og_delta_modularity.argtypes = [i64, vp, vp, vp, vp, vp, i64, i32, dbl]
        lib.og_delta_modularity.restype = dbl
        lib.og_delta_key.argtypes = [i64, vp, vp, vp, vp, vp, i64, i32]
        lib.og_delta_key.restype = i64
        lib.og_disconnected.argtypes = [i64, vp, vp, vp, vp]
        lib.og_disconnected.restype = i64
        lib.og_brute_force.argtypes = [i64, vp, vp, vp, dbl, vp]
        lib.og_brute_force.restype = dbl
        lib.og_aggregate.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
        lib.og_aggregate.restype = ctypes.c_int
        lib.og_schedule.argtypes = [i64, vp, vp, vp, ctypes.c_uint64, i32, i32, vp]
        lib.og_schedule.restype = i32
        lib.og_community_vertices.argtypes = [i64, vp, i64, vp, vp]
        lib.og_community_vertices.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Result:
    status: int
    membership: np.ndarray
    modularity: float
    passes: int
    trace: dict = field(default_factory=dict)  # trace[pass][what] -> ndarray


def leiden(g, mode: int = SEQ, resolution: float = 1.0, tolerance: float = 0.01,
           aggregation_tolerance: float = 0.8, tolerance_drop: float = 10.0, max_iterations: int = 20,
           max_passes: int = 10, flags: int = 0, schedule_layers: int = 0, schedule_buckets: int = 16,
           seed: int = 0,
           trace: bool = False) -> Result:
    """Algorithm 1 on a symmetric CSR ``g`` (fields n, offsets, indices, weights)."""
    lib = _lib()
    prm = _Params(resolution, tolerance, aggregation_tolerance, tolerance_drop, max_iterations,
                  max_passes, mode, flags, schedule_layers, schedule_buckets, seed)
    off = _c(g.offsets, np.int64)
    idx = _c(g.indices, np.int32)
    w = None if g.weights is None else _c(g.weights, np.float32)
    memb = np.zeros(max(g.n, 1), dtype=np.int32)
    q = ctypes.c_double(0.0)
    passes = ctypes.c_int32(0)
    store: dict = {}

    def _cb(_ctx, lp, what, data, count):
        dt = _TRACE_DTYPE[what]
        arr = np.ctypeslib.as_array(ctypes.cast(data, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                    shape=(max(count, 1),))[:count].copy() if count > 0 else np.zeros(0, dt)
        store.setdefault(lp, {})[what] = arr

    fn = _TRACE_FN(_cb) if trace else ctypes.cast(None, _TRACE_FN)
    rc = lib.og_leiden(g.n, _p(off), _p(idx), _p(w), ctypes.byref(prm), _p(memb), ctypes.byref(q),
                       ctypes.byref(passes), fn, None)
    return Result(rc, memb[:g.n].copy(), q.value, passes.value, store)


def modularity(g, membership, resolution: float = 1.0) -> float:
    """Eq. 1 (community form) of ``membership`` (labels in [0, n)) on ``g``."""
    off, idx = _c(g.offsets, np.int64), _c(g.indices, np.int32)
    w = None if g.weights is None else _c(g.weights, np.float32)
    c = _c(membership, np.int32)
    return _lib().og_modularity(g.n, _p(off), _p(idx), _p(w), _p(c), resolution)


def modularity_holey(n, off, deg, idx, w, membership, resolution: float = 1.0) -> float:
    """Eq. 1 on a holey CSR with fp64 weights."""
    a = [_c(off, np.int64), _c(deg, np.int32), _c(idx, np.int32), _c(w, np.float64),
         _c(membership, np.int32)]
    return _lib().og_modularity_holey(n, *[_p(x) for x in a], resolution)


def _holey(g):
    off = _c(g.offsets, np.int64)
    deg = np.diff(off).astype(np.int32)
    return off, deg, _c(g.indices, np.int32), _c(g.weights, np.float64)


def delta_modularity(g, membership, i: int, c: int, resolution: float = 1.0) -> float:
    """Eq. 2 for moving vertex i from membership[i] to community c."""
    off, deg, idx, w = _holey(g)
    m = _c(membership, np.int32)
    return _lib().og_delta_modularity(g.n, _p(off), _p(deg), _p(idx), _p(w), _p(m), i, c, resolution)


def delta_key(g, membership, i: int, c: int) -> int:
    """Exact integer key difference (2m^2 * Eq. 2) for integer weights."""
    off, deg, idx, w = _holey(g)
    m = _c(membership, np.int32)
    return int(_lib().og_delta_key(g.n, _p(off), _p(deg), _p(idx), _p(w), _p(m), i, c))


def disconnected(g, membership):
    """Algorithm 5: (number of disconnected communities, per-label flags)."""
    off, idx = _c(g.offsets, np.int64), _c(g.indices, np.int32)
    m = _c(membership, np.int32)
    flags = np.zeros(max(g.n, 1), np.uint8)
    k = _lib().og_disconnected(g.n, _p(off), _p(idx), _p(m), _p(flags))
    if k < 0:
        raise ValueError("invalid membership")
    return int(k), flags[:g.n]


def brute_force(g, resolution: float = 1.0):
    """max Eq. 1 over all set partitions (n <= 12): (Q_opt, one optimal labelling)."""
    off, idx = _c(g.offsets, np.int64), _c(g.indices, np.int32)
    w = _c(g.weights, np.float32)
    best = np.zeros(max(g.n, 1), np.int32)
    q = _lib().og_brute_force(g.n, _p(off), _p(idx), _p(w), resolution, _p(best))
    return q, best[:g.n]


def aggregate(n, off, deg, idx, w, membership, ncomm):
    """Algorithm 4 on a holey CSR: returns (off'', deg'', idx'', w'')."""
    off, deg, idx, w = _c(off, np.int64), _c(deg, np.int32), _c(idx, np.int32), _c(w, np.float64)
    m = _c(membership, np.int32)
    cap = int(deg.sum()) if n else 0
    o_off = np.zeros(ncomm + 1, np.int64)
    o_deg = np.zeros(max(ncomm, 1), np.int32)
    o_idx = np.zeros(max(cap, 1), np.int32)
    o_w = np.zeros(max(cap, 1), np.float64)
    rc = _lib().og_aggregate(n, _p(off), _p(deg), _p(idx), _p(w), _p(m), ncomm, _p(o_off), _p(o_deg),
                             _p(o_idx), _p(o_w))
    if rc != 0:
        raise ValueError(f"aggregate failed: {rc}")
    return o_off, o_deg[:ncomm], o_idx[:cap], o_w[:cap]


def community_vertices(membership, ncomm):
    """countCommunityVertices + exclusiveScan + fill (Algorithm 4)."""
    m = _c(membership, np.int32)
    coff = np.zeros(ncomm + 1, np.int64)
    mem = np.zeros(max(len(m), 1), np.int32)
    rc = _lib().og_community_vertices(len(m), _p(m), ncomm, _p(coff), _p(mem))
    if rc != 0:
        raise ValueError(f"community_vertices failed: {rc}")
    return coff, mem[:len(m)]


def schedule(n, off, deg, idx, state: int, layers: int = 1000, buckets: int = 16):
    """S0 priority steps of a holey CSR: (step per vertex, steps used)."""
    off, deg, idx = _c(off, np.int64), _c(deg, np.int32), _c(idx, np.int32)
    out = np.zeros(max(n, 1), np.int32)
    used = _lib().og_schedule(n, _p(off), _p(deg), _p(idx), ctypes.c_uint64(state), layers, buckets, _p(out))
    if used < 0:
        raise ValueError("schedule failed")
    return out[:n], int(used)


def csr_from_edges(n: int, src, dst, weights=None, drop_self_loops: bool = False, combine: str = "sum"):
    """Symmetric CSR of an undirected edge list, by its definition (the input
    preparation of Section 5.1 and Table 2): every edge u != v gives the
    entries (u, v) and (v, u), a self-loop one entry (u, u) or none when
    dropped; entries with the same (row, target) merged by summing their
    weights (or keeping the largest); rows in ascending target order.
    Returns (offsets int64[n+1], indices int32, weights float32), the weights
    summed in fp64 and then rounded once."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.ones(src.size) if weights is None else np.asarray(weights, dtype=np.float64)
    keep = ~(src == dst) if drop_self_loops else np.ones(src.size, bool)
    back = src != dst
    rows = np.concatenate([src[keep], dst[back]])
    cols = np.concatenate([dst[keep], src[back]])
    ws = np.concatenate([w[keep], w[back]])
    key = rows * max(n, 1) + cols
    uniq, inv = np.unique(key, return_inverse=True)
    merged = np.zeros(uniq.size)
    if combine == "sum":
        np.add.at(merged, inv, ws)
    else:
        merged[:] = -np.inf
        np.maximum.at(merged, inv, ws)
    r = uniq // max(n, 1)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, r + 1, 1)
    return np.cumsum(off), (uniq % max(n, 1)).astype(np.int32), merged.astype(np.float32)
