"""Small helpers shared by the tests: dense reference forms and seeded inputs."""
import numpy as np

import gen


def dense(g):
    """Dense weighted adjacency A (A_ii = self-loop weight, stored once)."""
    A = np.zeros((g.n, g.n))
    for i in range(g.n):
        for e in range(g.offsets[i], g.offsets[i + 1]):
            A[i, g.indices[e]] += g.weights[e]
    return A


def q_dense(A, memb, gamma=1.0):
    """Eq. 1, first form, with the null-model term over all vertex pairs:
    Q = 1/2m sum_ij [A_ij - gamma K_i K_j / 2m] delta(C_i, C_j)."""
    K = A.sum(axis=1)
    two_m = K.sum()
    if two_m == 0:
        return 0.0
    same = memb[:, None] == memb[None, :]
    return float(((A - gamma * np.outer(K, K) / two_m) * same).sum() / two_m)


def q_times_4m2_exact(A, memb):
    """(2m)^2 * Q exactly, in Python integers, for integer weights (gamma = 1):
    (2m)^2 Q = sum_c [2m sigma_c - Sigma_c^2]."""
    Ai = A.astype(np.int64)
    K = Ai.sum(axis=1)
    two_m = int(K.sum())
    tot = 0
    for c in np.unique(memb):
        sel = memb == c
        sigma = int(Ai[np.ix_(sel, sel)].sum())
        Sig = int(K[sel].sum())
        tot += two_m * sigma - Sig * Sig
    return tot


def random_graph_with_loops(n, p, seed, wmax=5):
    """G(n,p) with integer weights plus random self-loops (aggregated style)."""
    rng = np.random.default_rng(seed)
    base = gen.gnp(n, p, seed=seed, wmax=wmax)
    deg = np.diff(base.offsets)
    rows = np.repeat(np.arange(n), deg)
    keep = rows < base.indices
    u = list(rows[keep])
    v = list(base.indices[keep])
    w = list(base.weights[keep])
    for i in range(n):
        if rng.random() < 0.3:
            u.append(i)
            v.append(i)
            w.append(float(rng.integers(1, wmax + 1)))
    return gen.from_edges(n, u, v, w)


def ari(a, b):
    """Adjusted Rand index of two labelings (Hubert & Arabie 1985)."""
    a = np.unique(a, return_inverse=True)[1]
    b = np.unique(b, return_inverse=True)[1]
    n = len(a)
    cont = np.zeros((a.max() + 1, b.max() + 1), np.int64)
    np.add.at(cont, (a, b), 1)
    comb = lambda x: x * (x - 1) / 2.0
    sum_ij = comb(cont).sum()
    sa = comb(cont.sum(1)).sum()
    sb = comb(cont.sum(0)).sum()
    exp = sa * sb / comb(n)
    mx = (sa + sb) / 2.0
    return float((sum_ij - exp) / (mx - exp))
