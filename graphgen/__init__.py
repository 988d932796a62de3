"""Seeded synthetic graph generators (inputs only; none of the method's arithmetic).

Shared by the CPU oracle's tests, the GPU parity tests and ``bench.py``.  Every
graph is returned as an undirected CSR: ``offsets`` int64[n+1], ``adj`` int32[nnz]
(both directions of every edge present) and ``w`` int32[nnz].

Workload families follow the paper's instances: random hyperbolic graphs with
power-law exponent 5 (Appendix C, "Random Hyperbolic Graphs"), k-cores restricted to
their largest connected component (Appendix C, "Real-world Graphs"), Erdos-Renyi
blocks with weights uniform in [1, 100] (Appendix C, "Clustered Erdos-Renyi Graphs").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the generator library in place (plain g++, no fused multiply-add so
    that every host architecture draws the same graph)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            vp, i64, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.gg_rhg.restype = vp
            lib.gg_rhg.argtypes = [i64, f64, f64, u64]
            lib.gg_er.restype = vp
            lib.gg_er.argtypes = [i64, f64, u64, i32, i32]
            lib.gg_planted.restype = vp
            lib.gg_planted.argtypes = [i64, i64, f64, i64, u64, i32, i32]
            lib.gg_core_lcc.restype = vp
            lib.gg_core_lcc.argtypes = [vp, vp, vp, i64, i64, i32]
            lib.gg_pair_weights.restype = None
            lib.gg_pair_weights.argtypes = [vp, vp, vp, i64, u64, i32, i32]
            lib.gg_rhg_radius.restype = f64
            lib.gg_rhg_radius.argtypes = [i64, f64, f64]
            lib.gg_info.restype = None
            lib.gg_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            lib.gg_uniform.restype = None
            lib.gg_uniform.argtypes = [u64, u64, i64, vp]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected CSR with int32 ids and int32 weights."""
    offsets: np.ndarray  # int64 [n+1]
    adj: np.ndarray      # int32 [nnz]
    w: np.ndarray        # int32 [nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.adj.shape[0])

    @property
    def m(self) -> int:
        """Undirected edge count (the paper's m)."""
        return self.nnz // 2


def _take(h, name: str) -> Graph:
    lib = _load()
    n = ctypes.c_int64()
    nnz = ctypes.c_int64()
    lib.gg_info(h, ctypes.byref(n), ctypes.byref(nnz))
    off = np.empty(n.value + 1, dtype=np.int64)
    adj = np.empty(nnz.value, dtype=np.int32)
    w = np.empty(nnz.value, dtype=np.int32)
    lib.gg_copy(h, off.ctypes.data, adj.ctypes.data, w.ctypes.data)
    lib.gg_free(h)
    return Graph(off, adj, w, name)


def rhg(n: int, avg_deg: float, seed: int, gamma: float = 5.0) -> Graph:
    """Random hyperbolic graph (threshold model), unit weights, ids in angular order."""
    return _take(_load().gg_rhg(n, float(avg_deg), float(gamma), seed & (2**64 - 1)),
                 f"rhg(n={n},deg={avg_deg},gamma={gamma},seed={seed})")


def rhg_radius(n: int, avg_deg: float, gamma: float = 5.0) -> float:
    return float(_load().gg_rhg_radius(n, float(avg_deg), float(gamma)))


def er(n: int, avg_deg: float, seed: int, wlo: int = 1, whi: int = 1) -> Graph:
    """Erdos-Renyi G(n, p) with p = avg_deg / (n - 1); weights uniform in [wlo, whi]."""
    return _take(_load().gg_er(n, float(avg_deg), seed & (2**64 - 1), wlo, whi),
                 f"er(n={n},deg={avg_deg},seed={seed})")


def planted(blocks: int, block_n: int, avg_deg: float, bridges: int, seed: int,
            wlo: int = 1, whi: int = 100) -> Graph:
    """`blocks` ER blocks of `block_n` vertices joined by `bridges` random edges."""
    return _take(_load().gg_planted(blocks, block_n, float(avg_deg), bridges, seed & (2**64 - 1), wlo, whi),
                 f"planted({blocks}x{block_n},deg={avg_deg},bridges={bridges},seed={seed})")


def clustered_er(n: int, density: float, k: int, seed: int) -> Graph:
    """The clustered Erdos-Renyi family of the paper's experiments (Sec. 5, "clustered
    Erdos-Renyi graphs"): G(n, p) with p = density / 100, weights uniform in [1, 100],
    the weight of an edge inside one of the k clusters (contiguous id ranges) multiplied
    by n, so that the minimum cut separates clusters with high probability."""
    g = er(n, density / 100.0 * (n - 1), seed, 1, 100)
    part = (np.arange(g.n, dtype=np.int64) * k) // max(g.n, 1)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    w = g.w.astype(np.int64)
    w[part[src] == part[g.adj]] *= n
    assert w.max() < 2**31
    return Graph(g.offsets, g.adj, w.astype(np.int32), f"clustered_er(n={n},d={density}%,k={k},seed={seed})")


def core_lcc(g: Graph, k: int, lcc: bool = True) -> Graph:
    """k-core (peel degree < k) followed by the largest connected component."""
    h = _load().gg_core_lcc(g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, g.n, k, int(lcc))
    out = _take(h, f"{g.name}|core{k}{'|lcc' if lcc else ''}")
    return out


def with_pair_weights(g: Graph, seed: int, lo: int, hi: int) -> Graph:
    """Copy of `g` whose weights are uniform in [lo, hi], equal in both directions."""
    w = g.w.copy()
    _load().gg_pair_weights(g.offsets.ctypes.data, g.adj.ctypes.data, w.ctypes.data, g.n,
                            seed & (2**64 - 1), lo, hi)
    return Graph(g.offsets, g.adj, w, f"{g.name}|w[{lo},{hi}]")


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gg_uniform(seed & (2**64 - 1), stream, count, out.ctypes.data)
    return out


def from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR from an undirected edge list [(u, v, w), ...]; both directions stored,
    neighbour lists sorted by (id, weight)."""
    lists = [[] for _ in range(n)]
    for u, v, wt in edges:
        lists[u].append((v, wt))
        lists[v].append((u, wt))
    off = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        off[v + 1] = off[v] + len(lists[v])
    adj = np.empty(off[-1], dtype=np.int32)
    w = np.empty(off[-1], dtype=np.int32)
    for v in range(n):
        lst = sorted(lists[v])
        for k, (u, wt) in enumerate(lst):
            adj[off[v] + k] = u
            w[off[v] + k] = wt
    return Graph(off, adj, w, name)


# ----------------------------------------------------------------- workloads
def workload_rhg_small(seed: int = 1) -> Graph:
    """RHG n=2^14, average degree 32, exponent 5, unit weights, largest component."""
    return core_lcc(rhg(1 << 14, 32, seed), 0, True)


def workload_rhg_large(seed: int = 1, n: int = 1 << 22) -> Graph:
    """RHG n=2^22, average degree 64, exponent 5, unit weights, 16-core, largest
    component."""
    return core_lcc(rhg(n, 64, seed), 16, True)


def workload_planted(seed: int = 1, blocks: int = 8, block_n: int = 1 << 20) -> Graph:
    """8 ER blocks of 2^20 vertices (average degree 48) plus 64 bridges, weights
    uniform in [1, 100]."""
    return planted(blocks, block_n, 48, 64, seed, 1, 100)


def batch_specs(count: int, seed: int, lo_exp: int = 6, hi_exp: int = 14):
    """Per-graph recipe of the batched workload: n = floor(2^U(lo,hi)); a seeded coin
    picks RHG (average degree U[16, 64]) or ER (average degree U[8, 32]); the degree
    is clamped to (n - 1) / 2; weights uniform in [1, 10]."""
    u = uniform(seed, 7, 4 * count)
    specs = []
    for i in range(count):
        n = int(2.0 ** (lo_exp + (hi_exp - lo_exp) * u[4 * i]))
        kind = "rhg" if u[4 * i + 1] < 0.5 else "er"
        deg = 16 + 48 * u[4 * i + 2] if kind == "rhg" else 8 + 24 * u[4 * i + 2]
        deg = min(deg, (n - 1) / 2.0)
        specs.append((kind, n, deg, (seed * 1000003 + i) & (2**63 - 1)))
    return specs


def batch_graph(spec) -> Graph:
    kind, n, deg, s = spec
    g = rhg(n, deg, s) if kind == "rhg" else er(n, deg, s)
    g = core_lcc(g, 0, True)
    return with_pair_weights(g, s ^ 0x5EED, 1, 10)
