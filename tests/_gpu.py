"""GPU-test helpers: run the library through the C ABI and compare its
per-pass trace with the oracle's."""
import numpy as np

import gen
import oracle
import paper_2312_13936_gb300 as lg

TRACE_ITEMS = (lg.TRACE_INIT, lg.TRACE_MOVE, lg.TRACE_REFINE, lg.TRACE_COUNTS, lg.TRACE_RENUMBER, lg.TRACE_DENDRO)


def run_gpu(g, mode, trace=False, **kw):
    h = lg.Leiden(g.offsets, g.indices, g.weights)
    try:
        memb, q, st = h.run(mode=mode, trace=trace, **kw)
        tr = {}
        if trace:
            for p in range(st.passes):
                for w in TRACE_ITEMS + (lg.TRACE_AGG_OFF, lg.TRACE_AGG_DEG, lg.TRACE_AGG_IDX, lg.TRACE_AGG_W):
                    try:
                        tr.setdefault(p, {})[w] = h.trace(p, w)
                    except lg.LeidenError:
                        pass
        return memb.cpu().numpy(), q, st, tr
    finally:
        h.close()


def rows(off, deg, idx, w):
    """holey CSR rows as stored: the (target, weight) pairs of each row's fill,
    in their stored order (the slots after a row's fill are unused)"""
    out = []
    for c in range(len(deg)):
        a = int(off[c])
        out.append(list(zip(idx[a:a + deg[c]].tolist(), w[a:a + deg[c]].tolist())))
    return out


def compare_traces(gpu_tr, ora_tr):
    """Bit-exact per-phase comparison of a deterministic run; returns a list of
    mismatch descriptions. Aggregated rows are compared as stored: both
    sides write them in ascending target order (reading R10)."""
    bad = []
    if sorted(gpu_tr) != sorted(ora_tr):
        bad.append(f"passes differ: gpu {sorted(gpu_tr)} oracle {sorted(ora_tr)}")
    for p in sorted(set(gpu_tr) & set(ora_tr)):
        G, O = gpu_tr[p], ora_tr[p]
        for w in TRACE_ITEMS:
            if (w in G) != (w in O):
                bad.append(f"pass {p} item {w}: recorded on one side only")
            elif w in G and not np.array_equal(G[w], O[w]):
                d = np.nonzero(np.asarray(G[w]) != np.asarray(O[w]))[0] if len(G[w]) == len(O[w]) else []
                bad.append(f"pass {p} item {w}: differs ({len(d)} entries, first {d[:5]})")
        if lg.TRACE_AGG_OFF in O:
            if lg.TRACE_AGG_OFF not in G:
                bad.append(f"pass {p}: aggregated graph missing on GPU")
                continue
            if not np.array_equal(G[lg.TRACE_AGG_OFF], O[oracle.T_AGG_OFF]):
                bad.append(f"pass {p}: aggregated offsets differ")
            if not np.array_equal(G[lg.TRACE_AGG_DEG], O[oracle.T_AGG_DEG]):
                bad.append(f"pass {p}: aggregated degrees differ")
            else:
                rg = rows(G[6], G[7], G[8], G[9])
                ro = rows(O[6], O[7], O[8], O[9])
                nd = sum(1 for a, b in zip(rg, ro) if a != b)
                if nd:
                    bad.append(f"pass {p}: {nd} aggregated rows differ")
    return bad


# Asynchronous results are draws of a randomized heuristic (the paper's
# asynchronous execution introduces variability, Section 4.1), and the
# oracle's sequential order is one arbitrary order among many. Per graph,
# the asynchronous mode is therefore held to its expected modularity -- the
# mean over SEEDS runs with different schedule seeds -- against the lower
# of the oracle's identity-order run and its mean over ORDERS random vertex
# relabellings, within the stated 0.005.
SEEDS = 8
ORDERS = 8


def relabel(g, seed):
    """g with its vertices renumbered by a seeded random permutation."""
    perm = np.random.default_rng(seed).permutation(g.n)
    deg = np.diff(g.offsets)
    rows_ = np.repeat(np.arange(g.n), deg)
    keep = rows_ <= g.indices
    return gen.from_edges(g.n, perm[rows_[keep]], perm[g.indices[keep]], g.weights[keep])


def seq_reference(g, flags=0, orders=ORDERS, se=0.001, max_orders=64):
    """min(oracle SEQ run, mean of oracle SEQ over random relabellings).

    The mean is estimated to a standard error of `se`: at least `orders`
    relabellings, more (up to `max_orders`) while the sample's standard
    error is larger -- small sparse graphs spread by up to 0.018 (standard
    deviation) under relabelling, where eight orders leave the reference
    itself uncertain by more than the tolerance."""
    q0 = oracle.leiden(g, mode=oracle.SEQ, flags=flags).modularity
    if g.n == 0:
        return q0
    run = lambda k: oracle.leiden(relabel(g, 1000 + k), mode=oracle.SEQ, flags=flags).modularity
    qs = [run(k) for k in range(orders)]
    while len(qs) < max_orders and np.std(qs, ddof=1) / np.sqrt(len(qs)) > se:
        qs.append(run(len(qs)))
    return min(q0, float(np.mean(qs)))
