"""Seeded synthetic input graphs shared by the oracle tests, the GPU tests and
the benchmark.

This module only builds inputs: it holds none of the Leiden arithmetic. All
graphs are undirected with w_ij == w_ji (paper, Section 3 "Preliminaries") and
are returned as a symmetric CSR whose nnz counts both directions of an edge
(paper, Table 2 caption: |E| after adding reverse edges).

The recipes stand in for the paper's SuiteSparse graphs (Table 2), which are
not available here:
  * ``sbm``  -- stochastic block model, well-clustered structure;
  * ``road`` -- 2D lattice with dropped edges and diagonal shortcuts, standing
    in for the road networks asia_osm / europe_osm (low average degree);
  * ``rmat`` -- heavy-tailed R-MAT graph standing in for the web graphs
    (sk-2005 class, ~3.8B directed entries at scale 25, edge factor 56).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")


@dataclass
class CSR:
    """Symmetric CSR of an undirected weighted graph."""

    n: int
    offsets: np.ndarray  # int64[n+1]
    indices: np.ndarray  # int32[nnz]
    weights: np.ndarray  # float32[nnz]

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1]) if self.n >= 0 else 0

    def degree(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P64 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))
        P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
        PF = ctypes.POINTER(ctypes.POINTER(ctypes.c_float))
        out = [P64, P32, PF, ctypes.POINTER(ctypes.c_int64)]
        lib.gg_sbm.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64] + out + [ctypes.c_void_p]
        lib.gg_road.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_uint64] + out
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64] + out
        lib.gg_gnp.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64] + out
        lib.gg_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p] + out
        for f in (lib.gg_sbm, lib.gg_road, lib.gg_rmat, lib.gg_gnp, lib.gg_from_edges):
            f.restype = ctypes.c_int
        lib.gg_sbm_batch.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, P64] + out
        lib.gg_sbm_batch.restype = ctypes.c_int
        lib.gg_rmat_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, P32, P32, ctypes.POINTER(ctypes.c_int64)]
        lib.gg_rmat_edges.restype = ctypes.c_int
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_free.restype = None
        _lib_handle = lib
    return _lib_handle


def _call(fn, *args, n: int) -> CSR:
    lib = _lib()
    off = ctypes.POINTER(ctypes.c_int64)()
    idx = ctypes.POINTER(ctypes.c_int32)()
    w = ctypes.POINTER(ctypes.c_float)()
    nnz = ctypes.c_int64(0)
    extra = ()
    if fn is lib.gg_sbm:
        args, extra = args[:-1], (args[-1],)
    rc = fn(*args, ctypes.byref(off), ctypes.byref(idx), ctypes.byref(w), ctypes.byref(nnz), *extra)
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    try:
        m = nnz.value
        offsets = np.ctypeslib.as_array(off, shape=(n + 1,)).copy()
        indices = np.ctypeslib.as_array(idx, shape=(max(m, 1),))[:m].copy()
        weights = np.ctypeslib.as_array(w, shape=(max(m, 1),))[:m].copy()
    finally:
        for p in (off, idx, w):
            lib.gg_free(ctypes.cast(p, ctypes.c_void_p))
    return CSR(n, offsets, indices.astype(np.int32, copy=False), weights.astype(np.float32, copy=False))


def sbm(n: int, blocks: int, p_in: float, p_out: float, seed: int, return_blocks: bool = False):
    """Stochastic block model with near-equal blocks and unit weights."""
    lib = _lib()
    blk = np.zeros(max(n, 1), dtype=np.int32)
    g = _call(lib.gg_sbm, n, blocks, p_in, p_out, seed, blk.ctypes.data_as(ctypes.c_void_p), n=n)
    return (g, blk[:n].copy()) if return_blocks else g


def road(side: int, drop: float = 0.10, diag_frac: float = 0.01, wmin: int = 1, wmax: int = 10,
         seed: int = 2) -> CSR:
    """side x side lattice with dropped edges, diagonal shortcuts, integer weights."""
    return _call(_lib().gg_road, side, drop, diag_frac, wmin, wmax, seed, n=side * side)


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 3) -> CSR:
    """Symmetrised, deduplicated R-MAT graph without self-loops, unit weights."""
    return _call(_lib().gg_rmat, scale, edge_factor, a, b, c, seed, n=1 << scale)


def rmat_edges(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 3):
    """The edge list of rmat() before its CSR is built: (u, v) int32 arrays
    with u < v, self-loops dropped, duplicates kept. Turning it into the
    symmetric deduplicated CSR (reverse entries added, duplicates merged to
    weight 1) gives rmat()'s graph."""
    lib = _lib()
    u = ctypes.POINTER(ctypes.c_int32)()
    v = ctypes.POINTER(ctypes.c_int32)()
    m = ctypes.c_int64(0)
    rc = lib.gg_rmat_edges(scale, edge_factor, a, b, c, seed, ctypes.byref(u), ctypes.byref(v), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    try:
        k = m.value
        uu = np.ctypeslib.as_array(u, shape=(max(k, 1),))[:k].copy()
        vv = np.ctypeslib.as_array(v, shape=(max(k, 1),))[:k].copy()
    finally:
        for p in (u, v):
            lib.gg_free(ctypes.cast(p, ctypes.c_void_p))
    return uu, vv


def gnp(n: int, p: float, seed: int, wmax: int = 1) -> CSR:
    """Erdos-Renyi G(n, p); integer weights uniform in [1, wmax]."""
    return _call(_lib().gg_gnp, n, p, wmax, seed, n=n)


def from_edges(n: int, u, v, w=None) -> CSR:
    """Symmetric CSR from an undirected edge list; u == v is one self-loop entry."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    w = np.ones(len(u), np.float32) if w is None else np.ascontiguousarray(w, dtype=np.float32)
    vp = ctypes.c_void_p
    return _call(_lib().gg_from_edges, n, len(u), vp(u.ctypes.data), vp(v.ctypes.data),
                 vp(w.ctypes.data), n=n)


def ring_of_cliques(k: int, r: int) -> CSR:
    """r cliques K_k joined in a ring by one edge between consecutive cliques
    (vertex k*q of clique q to vertex k*(q+1)+1 of the next)."""
    us, vs = [], []
    for q in range(r):
        base = q * k
        for a in range(k):
            for b in range(a + 1, k):
                us.append(base + a)
                vs.append(base + b)
        nxt = ((q + 1) % r) * k
        us.append(base)
        vs.append(nxt + 1 if k > 1 else nxt)
    return from_edges(k * r, us, vs)


@dataclass
class Batch:
    """Independent graphs packed one after another: graph g owns vertices
    [vseg[g], vseg[g+1]); offsets index the packed indices/weights; indices
    are local to each graph."""

    vseg: np.ndarray     # int64[G+1]
    offsets: np.ndarray  # int64[N+1]
    indices: np.ndarray  # int32[nnz], local
    weights: np.ndarray  # float32[nnz]
    params: dict         # per-graph recipe parameters (numpy arrays)

    @property
    def num_graphs(self) -> int:
        return int(len(self.vseg) - 1)

    @property
    def n(self) -> int:
        return int(self.vseg[-1])

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def graph(self, g: int) -> CSR:
        """Graph g as a standalone CSR."""
        a, b = int(self.vseg[g]), int(self.vseg[g + 1])
        e0, e1 = int(self.offsets[a]), int(self.offsets[b])
        return CSR(b - a, self.offsets[a:b + 1] - e0, self.indices[e0:e1].copy(), self.weights[e0:e1].copy())


def sbm_batch_params(count: int, seed: int, nmin: int = 100, nmax: int = 100_000, bmin: int = 4, bmax: int = 64,
                     dmin: float = 8.0, dmax: float = 32.0, ratio: float = 0.02) -> dict:
    """Per-graph SBM parameters of a batch: n log-uniform in [nmin, nmax],
    blocks uniform in {bmin..bmax} (at most n/2), mean degree uniform in
    [dmin, dmax], p_out = ratio * p_in with p_in = d / ((s-1) + ratio (n-s)),
    s = n / blocks, p_in clamped to 1. Drawn with numpy's PCG64 from seed."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))).astype(np.int64)
    blocks = rng.integers(bmin, bmax + 1, count).astype(np.int32)
    blocks = np.maximum(1, np.minimum(blocks, n // 2)).astype(np.int32)
    dbar = rng.uniform(dmin, dmax, count)
    s = n / blocks
    p_in = np.minimum(1.0, dbar / ((s - 1) + ratio * (n - s)))
    p_out = ratio * p_in
    seeds = (np.uint64(seed) << np.uint64(32)) + np.arange(count, dtype=np.uint64)
    return {"n": n, "blocks": blocks, "mean_degree": dbar, "p_in": p_in, "p_out": p_out, "seeds": seeds}


def sbm_batch(count: int, seed: int, **kw) -> Batch:
    """A batch of seeded SBM graphs (see sbm_batch_params), generated in
    parallel; graph g equals sbm(n[g], blocks[g], p_in[g], p_out[g], seeds[g])."""
    prm = sbm_batch_params(count, seed, **kw)
    lib = _lib()
    vp = ctypes.c_void_p
    arrs = [np.ascontiguousarray(prm[k]) for k in ("n", "blocks", "p_in", "p_out", "seeds")]
    vseg = ctypes.POINTER(ctypes.c_int64)()
    off = ctypes.POINTER(ctypes.c_int64)()
    idx = ctypes.POINTER(ctypes.c_int32)()
    w = ctypes.POINTER(ctypes.c_float)()
    nnz = ctypes.c_int64(0)
    rc = lib.gg_sbm_batch(count, *[vp(a.ctypes.data) for a in arrs], ctypes.byref(vseg), ctypes.byref(off),
                          ctypes.byref(idx), ctypes.byref(w), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"batch generator failed with code {rc}")
    try:
        vs = np.ctypeslib.as_array(vseg, shape=(count + 1,)).copy()
        N, m = int(vs[-1]), nnz.value
        offsets = np.ctypeslib.as_array(off, shape=(N + 1,)).copy()
        indices = np.ctypeslib.as_array(idx, shape=(max(m, 1),))[:m].copy()
        weights = np.ctypeslib.as_array(w, shape=(max(m, 1),))[:m].copy()
    finally:
        for p in (vseg, off, idx, w):
            lib.gg_free(ctypes.cast(p, ctypes.c_void_p))
    return Batch(vs, offsets, indices, weights, prm)


def sbm_batch_workload(count: int = 4096) -> Batch:
    """4096 SBM graphs, n log-uniform in [100, 100000], 4-64 blocks, mean
    degree in [8, 32], p_out / p_in = 0.02, unit weights, seed 4."""
    return sbm_batch(count, seed=4)


# Workload recipes (seeds fixed; sizes as the workloads define them).
def sbm_workload() -> CSR:
    """10,000 vertices, 50 blocks of 200, p_in 0.05, p_out 0.0005, seed 1."""
    return sbm(10_000, 50, 0.05, 0.0005, seed=1)


def road_workload(side: int = 5000) -> CSR:
    """5000 x 5000 lattice, 10% of lattice edges dropped, 1% diagonals, w in [1,10], seed 2."""
    return road(side, 0.10, 0.01, 1, 10, seed=2)


def rmat_workload(scale: int = 25, edge_factor: int = 56) -> CSR:
    """R-MAT scale 25, edge factor 56, (0.57, 0.19, 0.19, 0.05), seed 3."""
    return rmat(scale, edge_factor, 0.57, 0.19, 0.19, seed=3)
