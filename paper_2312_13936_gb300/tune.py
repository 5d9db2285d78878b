"""Autotuner of the launch shape (leiden_tuning) per GPU and graph class.

The paper fixes its parallel schedule by measurement (OpenMP dynamic
scheduling with a chunk size chosen per machine, Section 4.1); here the
choices that play that role -- the degree-bin bounds (thread, warp and block
per vertex), the persistent sweep's blocks per SM and its vertices per block,
and the graph size from which the sweeps read rows copied in schedule order
-- are measured per GPU and graph class, and the best shape goes into a JSON
cache that handles read when they are created (leiden_tuning_lookup). None of
the choices changes a result of the deterministic mode.

The search is coordinate descent from the defaults: each field in turn takes
each of its candidate values with the others fixed, and keeps the value whose
run is fastest (the median of device-timed leiden_run calls), when it beats
the current one by more than ``min_gain``; the whole sweep repeats ``rounds``
times.

  python -m paper_2312_13936_gb300.tune --out CACHE.json [--graphs road:2000,rmat:21,...]

tunes on the repository's synthetic recipes (road lattices, block models,
R-MAT graphs, batches of block models; needs the ``gen`` module beside the
package) and merges the entries into CACHE.json.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

CANDIDATES = {
    "thread_max_deg": [4, 8],
    "warp_max_deg": [64, 128, 256],
    "block_max_deg": [512, 1024, 2048],
    "coop_blocks_per_sm": [0, 2, 3],
    "vertices_per_block": [1024, 2048, 4096],
    "list_order_min_vertices": [0, 1 << 18, 1 << 20, 1 << 22],
}


def graph_class(n: int, nnz: int, max_degree: int) -> dict:
    """The cache's class of a graph (leiden_tuning_lookup)."""
    return {"heavy_tailed": int(max_degree * n > 64 * nnz),
            "log2_vertices": int(round(math.log2(n))) if n > 0 else 0,
            "log2_mean_degree": int(round(math.log2(nnz / n))) if n > 0 and nnz > 0 else 0}


def time_runs(h, mode: int, runs: int) -> float:
    """Median device time (ms) of `runs` leiden_run calls on a handle."""
    import torch
    ts = []
    for _ in range(runs):
        _, _, st = h.run(mode=mode)
        torch.cuda.synchronize()
        ts.append(st.ms_total)
    return statistics.median(ts)


def tune_handle(h, mode: int = 0, runs: int = 3, rounds: int = 2, min_gain: float = 0.02,
                candidates: dict | None = None):
    """Coordinate descent over the candidate shapes on a Leiden (or
    LeidenBatch) handle. Returns (best shape as a dict, ms with the defaults,
    ms with the best shape, every trial as (shape, ms))."""
    from . import leiden_tuning_default
    cand = candidates or CANDIDATES
    best = leiden_tuning_default().as_dict()
    h.set_tuning(**best)
    h.run(mode=mode)  # warm-up
    ms_default = best_ms = time_runs(h, mode, runs)
    trials = [(dict(best), ms_default)]
    for _ in range(rounds):
        improved = False
        for key, values in cand.items():
            for v in values:
                if v == best[key]:
                    continue
                shape = dict(best, **{key: v})
                if shape["block_max_deg"] < shape["warp_max_deg"]:
                    continue
                h.set_tuning(**shape)
                ms = time_runs(h, mode, runs)
                trials.append((shape, ms))
                if ms < best_ms * (1.0 - min_gain):
                    best, best_ms, improved = shape, ms, True
            h.set_tuning(**best)
        if not improved:
            break
    h.set_tuning(**best)
    return best, ms_default, best_ms, trials


def merge_cache(path: str, entries: list) -> dict:
    """Add entries to the cache at path (an entry of the same GPU and class
    is replaced) and write it back."""
    cache = {"format": 1, "entries": []}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    keys = ("gpu", "heavy_tailed", "log2_vertices", "log2_mean_degree")
    for e in entries:
        cache["entries"] = [x for x in cache["entries"] if any(x.get(k) != e[k] for k in keys)] + [e]
    with open(path, "w") as f:
        json.dump(cache, f, indent=1)
        f.write("\n")
    return cache


def _graph(spec: str):
    import gen  # the repository's seeded input recipes
    kind, _, arg = spec.partition(":")
    if kind == "road":
        side = int(arg or 2000)
        return f"road lattice {side}x{side}", gen.road(side, 0.10, 0.01, 1, 10, seed=2)
    if kind == "rmat":
        scale = int(arg or 20)
        return f"R-MAT scale {scale}, edge factor 56", gen.rmat(scale, 56, 0.57, 0.19, 0.19, seed=3)
    if kind == "sbm":
        n = int(arg or 100000)
        return f"SBM {n} vertices, 100 blocks", gen.sbm(n, 100, 15.0 / (n / 100), 0.0003 * 1e4 / n, seed=7)
    if kind == "batch":
        G = int(arg or 4096)
        return f"batch of {G} SBM graphs, 100-100000 vertices", gen.sbm_batch(G, seed=4)
    raise ValueError(f"unknown graph spec {spec}")


def main(argv=None):
    import numpy as np
    import torch

    from . import LEIDEN_ASYNC, LEIDEN_DETERMINISTIC, Leiden, LeidenBatch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True, help="cache file to create or extend")
    ap.add_argument("--graphs", default="road:2000,sbm:200000,rmat:21",
                    help="comma-separated specs: road:SIDE, sbm:N, rmat:SCALE, batch:GRAPHS")
    ap.add_argument("--mode", default="async", choices=["async", "det"])
    ap.add_argument("--runs", type=int, default=3)
    ap.add_argument("--rounds", type=int, default=2)
    args = ap.parse_args(argv)
    mode = LEIDEN_ASYNC if args.mode == "async" else LEIDEN_DETERMINISTIC
    gpu = torch.cuda.get_device_name()
    entries = []
    for spec in args.graphs.split(","):
        name, g = _graph(spec)
        if hasattr(g, "num_graphs"):  # a packed batch: one LeidenBatch handle
            h = LeidenBatch(g.vseg, g.offsets, g.indices, g.weights, tuning=None)
            n, nnz = int(g.vseg[-1]), int(g.offsets[-1])
        else:
            h = Leiden(g.offsets, g.indices, g.weights, tuning=None)
            n, nnz = g.n, g.nnz
        t0 = time.perf_counter()
        best, ms0, ms1, trials = tune_handle(h, mode, args.runs, args.rounds)
        h.close()
        maxdeg = int(np.diff(g.offsets).max()) if n else 0
        e = {"gpu": gpu, **graph_class(n, nnz, maxdeg), **best, "graph": name, "mode": args.mode,
             "ms_default": ms0, "ms_tuned": ms1, "trials": len(trials), "tune_s": time.perf_counter() - t0}
        entries.append(e)
        print(json.dumps(e), flush=True)
    merge_cache(args.out, entries)


if __name__ == "__main__":
    main()
