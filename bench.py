#!/usr/bin/env python3
"""Leiden edges/s on one GB300.

One step is one leiden_run (every phase of the method: local-moving,
refinement, aggregation over all passes, final labels and modularity) on the
largest single-GPU workload: an R-MAT graph of scale 25 (33.5M vertices),
edge factor 56, (a, b, c) = (0.57, 0.19, 0.19), symmetrised, duplicates and
self-loops removed, unit weights (3,554,875,526 directed CSR entries; the
stand-in for the paper's sk-2005 web graph, Section 5.2 and Table 2). Its
edge list is drawn on the host and turned into the CSR on the GPU by
leiden_csr_from_edges. value = directed CSR entries / step time, with the
input resident in HBM. Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload rmat|road|sbm]

With N > 1 (torchrun, one process per GPU) every rank solves its own replica
of the workload: the method has no data-parallel split of one graph, so the
multi-GPU form is independent replicas ("scaling": "weak").

The same line carries the road-network workload ("road"): a 5000 x 5000
lattice with 10% of its edges dropped, 1% diagonal shortcuts and integer
weights in [1, 10] (25M vertices, ~91M entries), timed the same way, with its
own roofline, its CPU baseline (one oracle run on the full graph) and the
paper's variants on it ("variants"): the Louvain method (no refinement),
refine-based super-vertex labels and the randomized refinement, each with its
time, modularity and fraction of disconnected communities.

The batched form ("batched"): 4096 seeded SBM graphs (vertex counts
log-uniform in [100, 100000], 4-64 blocks, mean degree 8-32, p_out/p_in =
0.02; ~61M vertices, ~1.2e9 entries) packed as one segmented CSR and solved by
leiden_batch_run, in graphs/s, next to a per-graph loop of plain leiden_run
calls timed on a sample of the same graphs. With N > 1 the graphs are dealt
to ranks longest-first by entry count, each to the rank with the least work
so far.

The served form ("served"): a Poisson stream of seeded SBM (1k-4M vertices)
and R-MAT (scale 14-22, edge factor 16) graphs from host memory, served by
the continuous-batching server (leiden_server_*) and, on the same arrival
times, by a plain server that runs one leiden_run at a time. The offered rate
is set to 90% of the plain server's measured service rate; p50/p99 latency
(arrival to result on the host), graphs/s and the mean modularity of both are
reported. Rank 0 only.

"roofline" rates the dominant kernel class against the measured HBM copy
bandwidth: its algorithmic bytes (counted by the kernels in the first timed
step) over its CUDA-event time. "by_phase" and "overall" give the same for
each phase and for all profiled launches, and the profiled bytes over the
whole step. "e2e" runs the C ABI from page-locked host buffers (the copies in
and out inside the timed region; an unweighted graph goes without its weight
array) and splits a step into create, run and destroy. "cpu_baseline" is the oracle (sequential, one host core) on a
bounded sample of the same R-MAT recipe (scale 20). An optional part that
fails is reported as {"error": ...} in its place.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Leiden edges/s on 1 GB300 (% HBM roofline); batched graphs/s, p99 latency"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "roofline_traffic.json")
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat", choices=["rmat", "road", "sbm"])
    ap.add_argument("--side", type=int, default=5000, help="road lattice side")
    ap.add_argument("--rmat-scale", type=int, default=25)
    ap.add_argument("--mode", default="async", choices=["async", "det"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-road", action="store_true", help="skip the road object (when the headline is not road)")
    ap.add_argument("--cpu-scale", type=int, default=20, help="R-MAT scale of the CPU-baseline sample")
    ap.add_argument("--ref-scale", type=int, default=18, help="R-MAT scale of each reference-arm step")
    ap.add_argument("--ref-side", type=int, default=1500, help="road side of each reference-arm step (--workload road)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched form")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-sample", type=int, default=128, help="graphs of the per-graph loop")
    ap.add_argument("--no-serve", action="store_true", help="skip the served form")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the Louvain and refine-based-label comparison on the road graph")
    ap.add_argument("--serve-requests", type=int, default=200, help="measured requests of the served form")
    ap.add_argument("--serve-warmup", type=int, default=20, help="requests before the measured ones (not counted)")
    ap.add_argument("--serve-pool", type=int, default=24, help="distinct graphs the requests cycle through")
    ap.add_argument("--serve-load", type=float, default=0.9, help="offered rate / plain server's service rate")
    return ap.parse_args()


def variants_form(h, off, idx, mode, flags, stream, runs=5):
    """The paper's comparisons on the bench graph (outside the timed region):
    the Louvain variant (no refinement, Section 5: Leiden was 13% slower
    and Louvain left 4.0% of its communities disconnected) and refine-based
    super-vertex labels (Section 4.1: about the same time and modularity as
    move-based ones) and, in the asynchronous mode, the randomized refinement
    of the original method (Section 4.1: the greedy one was faster and better).
    Median of `runs` device-timed runs each."""
    import statistics

    import torch

    import paper_2312_13936_gb300 as lg
    out = {}
    variants = [("leiden", 0), ("louvain", lg.FLAG_LOUVAIN), ("refine_labels", lg.FLAG_REFINE_LABELS)]
    if mode == lg.LEIDEN_ASYNC:  # the randomized refinement has no deterministic mode
        variants.append(("random_refine", lg.FLAG_RANDOM_REFINE))
    for name, f in variants:
        h.run(mode=mode, flags=flags | f)
        ts, qs = [], []
        for _ in range(runs):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            memb, q, st = h.run(mode=mode, flags=flags | f)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            qs.append(q)
        bad = lg.disconnected(off, idx, memb)
        out[name] = {"ms": statistics.median(ts), "modularity": statistics.median(qs), "communities": st.communities,
                     "disconnected": bad, "disconnected_frac": bad / max(1, st.communities), "passes": st.passes}
    out["leiden_over_louvain_time"] = out["leiden"]["ms"] / out["louvain"]["ms"]
    return out


RMAT_ABC = (0.57, 0.19, 0.19)


def rmat_name(scale):
    return (f"R-MAT scale {scale}, edge factor 56, (0.57,0.19,0.19,0.05), symmetrised, duplicates and self-loops "
            f"removed, unit weights, seed 3")


def road_name(side):
    return (f"road lattice {side}x{side}, 10% edges dropped, 1% diagonal shortcuts, integer weights 1-10, seed 2")


def workload(args, dev):
    """The headline graph on the device: (name, n, nnz, off, idx, w as CUDA
    tensors). R-MAT: the edge list is drawn on the host and its CSR built on
    the GPU (leiden_csr_from_edges: reverse entries added, duplicates merged
    to weight 1, self-loops dropped); the others are generated on the host."""
    import torch

    import gen
    import paper_2312_13936_gb300 as lg
    if args.workload == "rmat":
        u, v = gen.rmat_edges(args.rmat_scale, 56, *RMAT_ABC, seed=3)
        du, dv = torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev)
        del u, v
        off, idx, w = lg.csr_from_edges(1 << args.rmat_scale, du, dv, None, drop_self_loops=True, combine="max")
        del du, dv
        torch.cuda.synchronize()
        return rmat_name(args.rmat_scale), 1 << args.rmat_scale, int(idx.numel()), off, idx, w
    if args.workload == "road":
        g, name = gen.road(args.side, 0.10, 0.01, 1, 10, seed=2), road_name(args.side)
    else:
        g, name = gen.sbm_workload(), "SBM 10,000 vertices, 50 blocks, p_in 0.05, p_out 0.0005, seed 1"
    return (name, g.n, g.nnz) + tuple(torch.as_tensor(a).to(dev) for a in (g.offsets, g.indices, g.weights))


class Clocks:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_sweep.cu", "k_aggregate.cu", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_2312_13936_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(cls_name, workload_name):
    """DRAM bytes per launch of a kernel class from the committed ncu
    summary, if it was captured on the current kernel sources and this
    workload; else None. Also returns the capture of a smaller case of the
    same recipe (its DRAM and algorithmic bytes per launch), when the
    workload itself is too large to capture, as a second value."""
    try:
        with open(TRAFFIC) as f:
            t = json.load(f)
        if t.get("source_hash") != kernel_source_hash():
            return None, None
        exact, sample = None, None
        for c in t.get("captures", []):
            cl = c.get("classes", {}).get(cls_name)
            if not cl:
                continue
            if c.get("workload") == workload_name:
                exact = cl.get("dram_bytes_per_launch")
            elif c.get("stands_for") == workload_name:
                sample = {"workload": c["workload"], "dram_bytes_per_launch": cl.get("dram_bytes_per_launch"),
                          "algorithmic_bytes_per_launch": cl.get("algorithmic_bytes_per_launch"),
                          "ratio": cl.get("ratio")}
        return exact, sample
    except Exception:
        return None, None


def phase_roofline(prof, peak, step_ms):
    """HBM roofline per phase and overall from a profiled run.

    prof maps (phase, bin) to {"launches", "ms", "bytes"}: the algorithmic
    bytes of the sweep and aggregation launches and their CUDA-event time.
    A phase's achieved bandwidth is its bytes over its launches' time. Overall
    is the same over all profiled launches ("profiled"), and the same bytes
    over the whole step ("step"), whose time also holds the schedule, setup
    and modularity kernels that count no bytes: a lower bound."""
    by_phase = {}
    for (phase, _), a in prof.items():
        e = by_phase.setdefault(phase, {"bytes": 0.0, "ms": 0.0, "launches": 0})
        e["bytes"] += a["bytes"]
        e["ms"] += a["ms"]
        e["launches"] += a["launches"]
    for e in by_phase.values():
        e["achieved"] = e["bytes"] / (e["ms"] / 1e3) / 1e9 if e["ms"] > 0 else 0.0
        e["frac"] = e["achieved"] / peak
    tb = sum(e["bytes"] for e in by_phase.values())
    tms = sum(e["ms"] for e in by_phase.values())
    over = {"bytes": tb, "profiled_ms": tms, "step_ms": step_ms}
    over["achieved_profiled"] = tb / (tms / 1e3) / 1e9 if tms > 0 else 0.0
    over["frac_profiled"] = over["achieved_profiled"] / peak
    over["achieved_step"] = tb / (step_ms / 1e3) / 1e9 if step_ms > 0 else 0.0
    over["frac_step"] = over["achieved_step"] / peak
    return by_phase, over


def optional_leg(fn, *args):
    """One optional part of the JSON line. A failure takes the part's place as
    {"error": ...}, with the traceback on stderr, so the headline still prints."""
    try:
        return fn(*args)
    except Exception as e:
        import traceback
        traceback.print_exc()
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def reduce_stats(stats, nmax, world):
    """All-reduce a 1-D tensor over the ranks: its first nmax entries (times)
    take the maximum over ranks, the others the sum. No collective for one rank."""
    if world > 1:
        import torch.distributed as dist
        mx = stats[:nmax].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(stats, op=dist.ReduceOp.SUM)
        stats[:nmax] = mx
    return stats


def batched_form(args, rank, world, mode, flags):
    """graphs/s of one leiden_batch_run over this rank's share of the batch,
    and of a per-graph loop of plain leiden_run calls on a sample of it."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import gen
    import paper_2312_13936_gb300 as lg
    b = gen.sbm_batch(args.batch_graphs, seed=4)
    G = b.num_graphs
    ids = lg.shard.lpt_shares(lg.shard.graph_entries(b), world)[rank]
    h = lg.LeidenBatch(*lg.shard.pack_share(b, ids))
    h.run(mode=mode, flags=flags)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for _ in range(args.batch_steps):
        memb, q, st = h.run(mode=mode, flags=flags)
    t1.record(s)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.batch_steps
    passes, comm = h.info()
    h.close()
    # per-graph loop of plain launches on a sample of the same graphs
    S = max(1, min(args.batch_sample, len(ids)))
    pick = np.linspace(0, len(ids) - 1, S).astype(int)
    dev = torch.device("cuda", torch.cuda.current_device())
    hs = []
    for k in pick:
        gk = b.graph(int(ids[k]))
        hs.append(lg.Leiden(torch.as_tensor(gk.offsets).to(dev), torch.as_tensor(gk.indices).to(dev),
                            torch.as_tensor(gk.weights).to(dev)))
    for hh in hs[:4]:
        hh.run(mode=mode, flags=flags)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ql = [hh.run(mode=mode, flags=flags)[1] for hh in hs]
    torch.cuda.synchronize()
    tl = time.perf_counter() - t
    for hh in hs:
        hh.close()
    stats = torch.tensor([ms, tl / S, float(q.sum()), float(len(q)), float(np.sum(ql)), float(np.sum(q[pick])),
                          float(S)], dtype=torch.float64, device=dev)
    ms, per_graph_s, qsum, qn, qls, qbs, ns = reduce_stats(stats, 2, world).tolist()
    return {
        "workload": (f"{G} SBM graphs, vertices log-uniform in [100, 100000], 4-64 blocks, mean degree 8-32, "
                     f"p_out/p_in 0.02, unit weights, seed 4; one segmented CSR per rank, "
                     f"graphs dealt to ranks longest-first by entries"),
        "graphs": G, "vertices": b.n, "entries": b.nnz, "mode": "async" if mode == lg.LEIDEN_ASYNC else "det",
        "graphs_per_s": G / (ms / 1e3), "ms_per_batch": ms, "edges_per_s": b.nnz / (ms / 1e3),
        "steps": args.batch_steps, "union_passes_rank0": st.passes, "max_graph_passes_rank0": int(passes.max()),
        "loop_graphs_per_s": world / per_graph_s, "loop_sample_graphs": int(ns),
        "speedup_vs_loop": (G / (ms / 1e3)) / (world / per_graph_s),
        "modularity_mean": qsum / qn, "modularity_mean_sample_batch": qbs / ns,
        "modularity_mean_sample_loop": qls / ns,
    }


def serve_pool(count, seed=5):
    """count seeded graphs: half SBM (n log-uniform in [1k, 4M], 4-64 blocks,
    mean degree 8-32, p_out/p_in 0.02), half R-MAT (scale 14-22, edge factor
    16, (0.57, 0.19, 0.19, 0.05)), unit weights."""
    import numpy as np

    import gen
    rng = np.random.default_rng(seed)
    pool, kinds = [], []
    for k in range(count):
        if k % 2 == 0:
            p = gen.sbm_batch_params(1, seed=seed * 1000 + k, nmin=1000, nmax=4_000_000)
            pool.append(gen.sbm(int(p["n"][0]), int(p["blocks"][0]), float(p["p_in"][0]), float(p["p_out"][0]),
                                int(p["seeds"][0])))
            kinds.append("sbm")
        else:
            pool.append(gen.rmat(int(rng.integers(14, 23)), 16, 0.57, 0.19, 0.19, seed=seed * 1000 + k))
            kinds.append("rmat")
    return pool, kinds


def served_form(args, mode, flags):
    """Continuous-batching server against a plain one-at-a-time server on the
    same Poisson arrivals (times measured on the host, results on the host)."""
    import numpy as np
    import torch

    import paper_2312_13936_gb300 as lg
    pool, kinds = serve_pool(args.serve_pool)
    W, R = args.serve_warmup, args.serve_requests
    T = W + R  # the first W arrivals warm the server up and are not counted
    stream = torch.cuda.current_stream()
    sp = lg._VP(stream.cuda_stream)

    def plain_one(g):
        h = lg.leiden_create(g.n, g.nnz, g.offsets.ctypes.data_as(lg._VP), g.indices.ctypes.data_as(lg._VP),
                             g.weights.ctypes.data_as(lg._VP), lg.LEIDEN_HOST, 0, sp)
        out = np.zeros(max(g.n, 1), np.int32)
        p = lg.leiden_params_default()
        p.mode = mode
        p.flags = flags
        q, st = lg.leiden_run(h, p, out.ctypes.data_as(lg._VP), lg.LEIDEN_HOST)
        lg.leiden_destroy(h)
        return q
    # service rate of the plain server (every pool graph once, after a warm-up)
    for g in pool[:2]:
        plain_one(g)
    t = time.perf_counter()
    for g in pool:
        plain_one(g)
    service = (time.perf_counter() - t) / len(pool)
    rate = args.serve_load / service
    rng = np.random.default_rng(55)
    arrive = np.cumsum(rng.exponential(1.0 / rate, T))
    order = rng.integers(0, len(pool), T)  # each request draws its graph from the pool

    def summary(lat, t_end, qs):
        lat = np.asarray(lat)  # of the measured requests, from the first one's arrival
        return {"graphs_per_s": R / (t_end - arrive[W]), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "modularity_mean": float(np.mean(qs))}

    # plain server: first come, first served, one leiden_run at a time
    lat, qs = [], []
    t0 = time.perf_counter()
    for k in range(T):
        now = time.perf_counter() - t0
        if now < arrive[k]:
            time.sleep(arrive[k] - now)
        q = plain_one(pool[order[k]])
        if k >= W:
            qs.append(q)
            lat.append(time.perf_counter() - t0 - arrive[k])
    plain = summary(lat, time.perf_counter() - t0, qs)
    # continuous batching
    cap_v = max(g.n for g in pool) * 4
    cap_e = max(g.nnz for g in pool) * 4
    srv = lg.LeidenServer(cap_v, cap_e, max_graphs=256, mode=mode)
    max_steps = 100_000  # every loop below ends: graphs finish within MAX_PASSES steps of admission

    def drain(count):
        got = 0
        for _ in range(max_steps):
            if got >= count:
                return
            srv.step()
            got += len(srv.results())
        raise RuntimeError("server made no progress")
    for g in pool[:2]:  # warm-up
        srv.submit(g.offsets, g.indices, g.weights)
    drain(2)
    lat, qs, steps = {}, {}, 0
    ids = {}
    t0 = time.perf_counter()
    k = 0
    while len(lat) < T:
        if steps > max_steps:
            raise RuntimeError("server made no progress")
        now = time.perf_counter() - t0
        while k < T and arrive[k] <= now:
            g = pool[order[k]]
            ids[srv.submit(g.offsets, g.indices, g.weights)] = k
            k += 1
        info = srv.info()
        if info["in_flight"] == 0 and info["waiting"] == 0 and info["finished"] == 0:
            if k >= T:
                raise RuntimeError("requests lost by the server")
            time.sleep(max(0.0, arrive[k] - (time.perf_counter() - t0)))
            continue
        if info["in_flight"] or info["waiting"]:
            srv.step()
            steps += 1
        for rid, memb, q, passes, comm in srv.results():
            j = ids.pop(rid)
            lat[j] = time.perf_counter() - t0 - arrive[j]
            qs[j] = q
    cb = summary([lat[j] for j in range(W, T)], time.perf_counter() - t0, [qs[j] for j in range(W, T)])
    cb["steps"] = steps
    # saturated: every graph of two rounds of the pool waiting at once
    S = 2 * len(pool)
    t = time.perf_counter()
    for k in range(S):
        g = pool[k % len(pool)]
        srv.submit(g.offsets, g.indices, g.weights)
    drain(S)
    sat_cb = S / (time.perf_counter() - t)
    srv.close()
    t = time.perf_counter()
    for k in range(S):
        plain_one(pool[k % len(pool)])
    sat_plain = S / (time.perf_counter() - t)
    return {
        "workload": (f"Poisson arrivals of {R} requests after {W} warm-up requests, each drawing one of "
                     f"{len(pool)} seeded graphs (SBM n in [1k, 4M] log-uniform, R-MAT scale 14-22 edge factor 16; "
                     f"{sum(g.nnz for g in pool) / 1e6:.0f}M entries in the pool), unit weights, from host memory"),
        "mode": "async" if mode == lg.LEIDEN_ASYNC else "det",
        "offered_rate_per_s": rate, "load_vs_plain": args.serve_load, "plain_service_ms": service * 1e3,
        "continuous": cb, "plain": plain,
        "saturated": {"graphs": S, "continuous_graphs_per_s": sat_cb, "plain_graphs_per_s": sat_plain,
                      "ratio": sat_cb / sat_plain},
    }


def cpu_baseline(kind, size):
    """The oracle (SEQ mode, sequential, one host core) on one bounded sample
    of a recipe: R-MAT of the given scale, or the road lattice of the given
    side."""
    import gen
    import oracle
    if kind == "rmat":
        g = gen.rmat(size, 56, *RMAT_ABC, seed=3)
        what = rmat_name(size)
    else:
        g = gen.road(size, 0.10, 0.01, 1, 10, seed=2)
        what = road_name(size)
    t = time.perf_counter()
    r = oracle.leiden(g, mode=oracle.SEQ)
    dt = time.perf_counter() - t
    assert r.status == 0
    return {"value": g.nnz / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": (f"one sequential oracle run (SEQ mode) on {what}: {g.n} vertices, {g.nnz} directed "
                       f"entries, {dt:.1f} s on 1 host core of {os.cpu_count()}"),
            "modularity": r.modularity}


def run_reference(args, rank):
    """Reference arm: the CPU oracle timed on host cores, same metric and unit,
    each step one run on a bounded sample of the GPU arm's workload."""
    if rank != 0:
        return
    import gen
    import oracle
    if args.workload == "road":
        g = gen.road(args.ref_side, 0.10, 0.01, 1, 10, seed=2)
        wl = f"{road_name(args.ref_side)} (bounded sample of the {args.side}x{args.side} workload)"
    else:
        g = gen.rmat(args.ref_scale, 56, *RMAT_ABC, seed=3)
        wl = f"{rmat_name(args.ref_scale)} (bounded sample of the scale-{args.rmat_scale} workload)"
    for _ in range(args.warmup):
        oracle.leiden(g, mode=oracle.SEQ)
    t = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.leiden(g, mode=oracle.SEQ)
    dt = time.perf_counter() - t
    value = args.steps * g.nnz / dt
    sample = (f"each step one sequential oracle run (SEQ mode) on {wl}: {g.n} vertices, {g.nnz} directed entries, "
              f"1 host core of {os.cpu_count()}")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "edges/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_ORACLE,
        "data": "synthetic", "config": {"workload": wl, "modularity": r.modularity},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def tuning_report(h, mode, flags, runs=3):
    """The launch shape the handle took (the autotuner cache's entry for this
    GPU and graph class, else the defaults) and the median device time of a
    run with it and with the defaults (outside the timed region)."""
    import statistics as st_

    import paper_2312_13936_gb300 as lg
    shape = h.tuning()
    default = lg.leiden_tuning_default().as_dict()

    def med():
        return st_.median(h.run(mode=mode, flags=flags)[2].ms_total for _ in range(runs))
    tuned_ms = med()
    default_ms = tuned_ms
    if shape != default:
        h.set_tuning(**default)
        default_ms = med()
        h.set_tuning(**shape)
    return {"shape": shape, "from_cache": shape != default, "tuned_ms": tuned_ms, "default_ms": default_ms,
            "cache": "paper_2312_13936_gb300/tuning_cache.json"}


def timed_runs(h, mode, flags, steps, warmup, stream, world, dev, clocks=None):
    """W untimed runs, then K runs between barriers and synchronisations,
    timed with CUDA events on the run's stream (max over ranks); the first
    timed run is profiled (events around every sweep and aggregation launch,
    work counters in the kernels). Returns (ms for the K runs, stats of the
    last run, membership, modularities, profile, kernel launches)."""
    import torch
    import torch.distributed as dist

    import paper_2312_13936_gb300 as lg
    for _ in range(warmup):
        h.run(mode=mode, flags=flags)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    prof, launches, qs = {}, 0, []
    for i in range(steps):
        memb, q, st = h.run(mode=mode, flags=flags | (lg.FLAG_PROFILE if i == 0 else 0))
        qs.append(q)
        launches += st.kernel_launches
        if i == 0:
            for k, v in h.profile().items():
                prof[k] = {"launches": v["launches"], "ms": v["ms"], "bytes": v["bytes"]}
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    if world > 1:
        ms = float(reduce_stats(torch.tensor([ms], device=dev), 1, world).item())
        dist.barrier()
    return ms, st, memb, qs, prof, launches, ck


def roofline_of(prof, peak, peak_kind, wname, step_ms):
    """Roofline object of the dominant kernel class of a profiled run."""
    top = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    if not top:
        return None
    (phase, binname), a = top
    achieved = a["bytes"] / (a["ms"] / 1e3) / 1e9
    cls = f"{phase}/{binname}"
    total_ms = sum(v["ms"] for v in prof.values())
    traffic, sample = traffic_for(cls, wname)
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "traffic": traffic, "kernel": cls, "peak_source": f"{peak_kind} hbm_gbs",
         "bytes_per_launch": a["bytes"] / a["launches"], "ms_per_launch": a["ms"] / a["launches"],
         "share_of_profiled_ms": a["ms"] / total_ms}
    if sample:
        r["traffic_smaller_case"] = sample
    r["by_phase"], r["overall"] = phase_roofline(prof, peak, step_ms)
    return r


def road_form(args, mode, flags, stream, world, dev, peak, peak_kind):
    """The road workload as a second object: device-timed edges/s, roofline,
    modularity and connectivity, the paper's variants on it, and the
    oracle's CPU baseline on the full graph."""
    import torch

    import gen
    import paper_2312_13936_gb300 as lg
    g = gen.road(args.side, 0.10, 0.01, 1, 10, seed=2)
    name = road_name(args.side)
    off, idx, w = (torch.as_tensor(a).to(dev) for a in (g.offsets, g.indices, g.weights))
    h = lg.Leiden(off, idx, w)
    ms, st, memb, qs, prof, launches, _ = timed_runs(h, mode, flags, args.steps, args.warmup, stream, world, dev)
    out = {"workload": name, "n": g.n, "nnz": g.nnz, "value": world * args.steps * g.nnz / (ms / 1e3),
           "unit": "edges/s", "ms_per_step": ms / args.steps, "modularity": statistics.median(qs),
           "disconnected_communities": lg.disconnected(off, idx, memb), "passes": st.passes,
           "phase_ms": {"move": st.ms_move, "refine": st.ms_refine, "aggregate": st.ms_aggregate,
                        "other": st.ms_other},
           "gpu_launches": launches,
           "roofline": roofline_of(prof, peak, peak_kind, name, ms / args.steps),
           "kernel_classes": {f"{k[0]}/{k[1]}": v for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}
    if world == 1:
        out["tuning"] = optional_leg(tuning_report, h, mode, flags)
    if not args.no_variants and world == 1:
        out["variants"] = optional_leg(variants_form, h, off, idx, mode, flags, stream)
    h.close()
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = optional_leg(cpu_baseline, "road", args.side)
    return out


DTYPE = ("fp32 edge weights, per-edge sums and move keys; fp64 community totals, 2m and modularity "
         "(asynchronous mode); int64 sums and 128-bit keys (deterministic mode)")
DTYPE_ORACLE = "f64 (the oracle's sequential mode)"


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2312_13936_gb300 as lg
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    t_build = time.perf_counter()
    wname, n, nnz, off, idx, w = workload(args, dev)
    t_build = time.perf_counter() - t_build
    mode = lg.LEIDEN_ASYNC if args.mode == "async" else lg.LEIDEN_DETERMINISTIC
    base_flags = 0
    stream = torch.cuda.current_stream()
    h = lg.Leiden(off, idx, w)
    peak, peak_kind = hbm_peak()

    # ---- timed region (device time, CUDA events on the run's stream)
    clocks = Clocks(local)
    ms, st, memb, qs, prof, launches, ck = timed_runs(h, mode, base_flags, args.steps, args.warmup, stream, world,
                                                      dev, clocks)
    value = world * args.steps * nnz / (ms / 1e3)
    # every community connected? (Algorithm 5 on the GPU, outside the timed region)
    disconnected = lg.disconnected(off, idx, memb)
    tuning = optional_leg(tuning_report, h, mode, base_flags) if world == 1 else None
    h.close()
    graph_bytes = 8 * (n + 1) + 8 * nnz

    # ---- end to end through the C ABI with host buffers (H2D and D2H inside)
    def e2e_leg():
        import ctypes
        vp = ctypes.c_void_p
        # the user's buffers, staged once in page-locked host memory (outside
        # the timed region), as a caller that streams graphs would keep them;
        # an unweighted graph (every weight 1) is passed without weights, as
        # its user holds none (the library then takes unit weights)
        unweighted = nnz > 0 and bool(torch.all(w == 1).item())
        arrays = (off, idx) if unweighted else (off, idx, w)
        try:
            hbuf = [torch.empty(t.numel(), dtype=t.dtype, pin_memory=True) for t in arrays]
            hout = torch.empty(max(n, 1), dtype=torch.int32, pin_memory=True)
            pinned = True
        except RuntimeError:
            hbuf = [torch.empty(t.numel(), dtype=t.dtype) for t in arrays]
            hout = torch.empty(max(n, 1), dtype=torch.int32)
            pinned = False
        for hb, t in zip(hbuf, arrays):
            hb.copy_(t)
        hw = vp(None) if unweighted else vp(hbuf[2].data_ptr())
        P = lg.leiden_params_default()
        P.mode = mode
        P.flags = base_flags
        split = [0.0, 0.0, 0.0]  # create (H2D + device setup), run (+ D2H of the result), destroy

        def one():
            t0 = time.perf_counter()
            hh = lg.leiden_create(n, nnz, vp(hbuf[0].data_ptr()), vp(hbuf[1].data_ptr()), hw,
                                  lg.LEIDEN_HOST, 0, vp(stream.cuda_stream))
            stream.synchronize()
            t1 = time.perf_counter()
            lg.leiden_run(hh, P, vp(hout.data_ptr()), lg.LEIDEN_HOST)
            t2 = time.perf_counter()
            lg.leiden_destroy(hh)
            t3 = time.perf_counter()
            for k, dt in enumerate((t1 - t0, t2 - t1, t3 - t2)):
                split[k] += dt
        one()
        split[:] = [0.0, 0.0, 0.0]
        ne = max(2, args.steps // 4)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ne):
            one()
        te = time.perf_counter() - t0
        if world > 1:
            te = float(reduce_stats(torch.tensor([te], device=dev), 1, world).item())
        return {"value": world * ne * nnz / te, "unit": "edges/s",
                "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in hbuf),
                "d2h_bytes_per_step": n * 4 + 8, "pinned": pinned,
                "weights": "none passed (unit weights)" if unweighted else "passed",
                "steps": ne, "ms_per_step": te * 1e3 / ne,
                "create_ms": split[0] * 1e3 / ne, "run_ms": split[1] * 1e3 / ne,
                "destroy_ms": split[2] * 1e3 / ne}

    # legs with collectives run bare under several ranks: a rank that stopped
    # on its own error would leave the others waiting
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg() if world > 1 else optional_leg(e2e_leg)
    del off, idx, w
    torch.cuda.empty_cache()
    road = None
    if args.workload != "road" and not args.no_road:
        road = (road_form(args, mode, base_flags, stream, world, dev, peak, peak_kind) if world > 1
                else optional_leg(road_form, args, mode, base_flags, stream, world, dev, peak, peak_kind))
    batched = None
    if not args.no_batch:
        batched = (batched_form(args, rank, world, mode, base_flags) if world > 1
                   else optional_leg(batched_form, args, rank, world, mode, base_flags))

    if rank != 0:
        dist.destroy_process_group()
        return
    roofline = roofline_of(prof, peak, peak_kind, wname, ms / args.steps)
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = (optional_leg(cpu_baseline, "rmat", args.cpu_scale) if args.workload == "rmat"
               else optional_leg(cpu_baseline, "road", min(args.side, 5000)) if args.workload == "road" else None)
    served = None if (args.no_serve or world > 1) else optional_leg(served_form, args, mode, base_flags)
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": wname, "n": n, "nnz": nnz, "mode": args.mode,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (CSR %.2f GB)" % (graph_bytes / 1e9),
                   "build_s": t_build,
                   "modularity": statistics.median(qs), "disconnected_communities": disconnected,
                   "passes": st.passes,
                   "move_sweeps": st.move_iterations, "refine_sweeps": st.refine_iterations,
                   "phase_ms": {"move": st.ms_move, "refine": st.ms_refine, "aggregate": st.ms_aggregate,
                                "other": st.ms_other}},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": launches,
        "tuning": tuning,
        "road": road,
        "batched": batched,
        "served": served,
        "kernel_classes": {f"{k[0]}/{k[1]}": v for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
