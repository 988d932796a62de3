"""Independent checkers for the tests: brute-force cuts, closed-form graph families,
CSR invariants.  None of this calls the oracle or the GPU library."""
from __future__ import annotations

import itertools
import random

import numpy as np

import graphgen as gg


def edges_of(offsets, adj, w):
    """Undirected edge list (u < v) with parallel entries summed."""
    acc = {}
    n = len(offsets) - 1
    for v in range(n):
        for e in range(int(offsets[v]), int(offsets[v + 1])):
            u = int(adj[e])
            if v < u:
                acc[(v, u)] = acc.get((v, u), 0) + int(w[e])
    return acc


def cut_weight(offsets, adj, w, side: np.ndarray) -> int:
    """Capacity of the cut (side, V minus side), Sec. 3 definition."""
    n = len(offsets) - 1
    src = np.repeat(np.arange(n), np.diff(np.asarray(offsets)))
    cross = side[src] != side[np.asarray(adj)]
    return int(np.asarray(w, dtype=np.int64)[cross].sum()) // 2


def brute_lambda(offsets, adj, w) -> int:
    """Minimum over all 2^(n-1) - 1 bipartitions (vertex n-1 fixed on side 0)."""
    n = len(offsets) - 1
    assert 2 <= n <= 22
    E = edges_of(offsets, adj, w)
    if not E:
        return 0
    us = np.array([k[0] for k in E], dtype=np.int64)
    vs = np.array([k[1] for k in E], dtype=np.int64)
    ws = np.array(list(E.values()), dtype=np.int64)
    best = None
    total = 1 << (n - 1)
    step = 1 << 16
    for start in range(1, total, step):
        masks = np.arange(start, min(total, start + step), dtype=np.int64)
        su = (masks[:, None] >> us[None, :]) & 1
        sv = (masks[:, None] >> vs[None, :]) & 1
        cw = ((su != sv) * ws[None, :]).sum(axis=1)
        m = int(cw.min())
        best = m if best is None else min(best, m)
    return best


def stoer_wagner(offsets, adj, w) -> int:
    """Exact minimum cut by networkx's Stoer-Wagner (a library routine)."""
    import networkx as nx
    G = nx.Graph()
    n = len(offsets) - 1
    G.add_nodes_from(range(n))
    for (u, v), wt in edges_of(offsets, adj, w).items():
        G.add_edge(u, v, weight=wt)
    if not nx.is_connected(G):
        return 0
    val, _ = nx.stoer_wagner(G)
    return int(val)


# ------------------------------------------------------------- graph families
def cycle(n, wt=1):
    return gg.from_edges(n, [(i, (i + 1) % n, wt) for i in range(n)], f"C{n}")


def path(ws):
    n = len(ws) + 1
    return gg.from_edges(n, [(i, i + 1, int(ws[i])) for i in range(n - 1)], "path")


def complete(n, wt=1):
    return gg.from_edges(n, [(i, j, wt) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def complete_bipartite(a, b):
    return gg.from_edges(a + b, [(i, a + j, 1) for i in range(a) for j in range(b)], f"K{a},{b}")


def hypercube(d):
    n = 1 << d
    return gg.from_edges(n, [(v, v ^ (1 << k), 1) for v in range(n) for k in range(d) if v < v ^ (1 << k)], f"Q{d}")


def grid(p, q):
    idx = lambda i, j: i * q + j
    E = []
    for i in range(p):
        for j in range(q):
            if i + 1 < p:
                E.append((idx(i, j), idx(i + 1, j), 1))
            if j + 1 < q:
                E.append((idx(i, j), idx(i, j + 1), 1))
    return gg.from_edges(p * q, E, f"grid{p}x{q}")


def two_cliques(k, j):
    """Two K_k joined by j disjoint unit edges (j < k - 1): lambda = j."""
    E = [(a, b, 1) for a in range(k) for b in range(a + 1, k)]
    E += [(k + a, k + b, 1) for a in range(k) for b in range(a + 1, k)]
    E += [(i, k + i, 1) for i in range(j)]
    return gg.from_edges(2 * k, E, f"2K{k}+{j}")


def pr2_counterexample():
    """Triangles {0,1,2} and {3,4,5} of weight 10, vertex 6 tied to 0 and 3 with
    weight 1: lambda = 1 while the minimum degree is 2, and both edges at vertex 6
    pass Padberg-Rinaldi condition 2."""
    E = [(0, 1, 10), (1, 2, 10), (0, 2, 10), (3, 4, 10), (4, 5, 10), (3, 5, 10), (6, 0, 1), (6, 3, 1)]
    return gg.from_edges(7, E, "pr2-counterexample")


def random_graph(n, p, seed, wmax=5, connected=True):
    rnd = random.Random(seed)
    E = []
    for a, b in itertools.combinations(range(n), 2):
        if rnd.random() < p:
            E.append((a, b, rnd.randint(1, wmax)))
    if connected:
        perm = list(range(n))
        rnd.shuffle(perm)
        for i in range(1, n):
            E.append((perm[i - 1], perm[i], rnd.randint(1, wmax)))
    return gg.from_edges(n, E, f"rand(n={n},p={p},seed={seed})")


def check_csr(offsets, adj, w, merged=True):
    """Symmetric, no self-loops; if merged: lists strictly ascending (no duplicates)."""
    offsets = np.asarray(offsets)
    adj = np.asarray(adj)
    w = np.asarray(w)
    n = len(offsets) - 1
    assert offsets[0] == 0 and np.all(np.diff(offsets) >= 0) and offsets[-1] == len(adj)
    src = np.repeat(np.arange(n), np.diff(offsets))
    assert np.all(src != adj), "self-loop"
    assert np.all(w > 0)
    a = np.lexsort((w, adj, src))
    b = np.lexsort((w, src, adj))
    assert np.array_equal(src[a], adj[b]) and np.array_equal(adj[a], src[b]) and np.array_equal(w[a], w[b]), "asymmetric"
    if merged:
        same = src[1:] == src[:-1]
        assert np.all(adj[1:][same] > adj[:-1][same]), "lists not strictly ascending"
