"""CPU oracle for the VieCut minimum-cut method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` import this module.  The GPU library never calls it and shares no code
with it.  The arithmetic lives in ``oracle.cpp`` (plain single-threaded C++, every
function citing the paper's passage); this file only builds it and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STEP_KINDS = {0: "initial", 1: "lp", 2: "pr_a", 3: "pr_b", 4: "noi"}


class OrcStep(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("lambda_hat", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compiles the oracle with plain g++ (single-threaded, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _declare_viecut(lib):
    vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    lib.orc_viecut.restype = ctypes.c_int
    lib.orc_viecut.argtypes = [i64, vp, vp, vp, i32, u64, i32, i64, i32, vp, vp, vp, i64, vp, i32, i32, i32]


def load_variant(path: str):
    """Loads another build of oracle.cpp (tests only: a copy with a planted mistake)
    for ``viecut(..., _lib=...)``."""
    lib = ctypes.CDLL(path)
    _declare_viecut(lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            lib.orc_mix64.restype = u64
            lib.orc_mix64.argtypes = [u64]
            lib.orc_level_key.restype = u64
            lib.orc_level_key.argtypes = [u64, i64]
            lib.orc_degrees.restype = None
            lib.orc_degrees.argtypes = [i64, vp, vp, vp, vp]
            lib.orc_lp_round.restype = None
            lib.orc_lp_round.argtypes = [i64, vp, vp, vp, vp, u64, vp]
            lib.orc_lp_level.restype = i32
            lib.orc_lp_level.argtypes = [i64, vp, vp, vp, u64, i32, i32, vp, i32]
            lib.orc_lp_round_async.restype = None
            lib.orc_lp_round_async.argtypes = [i64, vp, vp, vp, vp, u64, i32, i64, i64, i32]
            lib.orc_contract.restype = i64
            lib.orc_contract.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            for name in ("orc_pr_pass_a", "orc_pr_pass_b", "orc_noi_round"):
                f = getattr(lib, name)
                f.restype = i64
                f.argtypes = [i64, vp, vp, vp, i64, vp]
            _declare_viecut(lib)
            lib.orc_correct.restype = i64
            lib.orc_correct.argtypes = [i64, vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


@dataclass
class CsrGraph:
    """CSR with int64 weights (the form every coarse graph takes)."""
    offsets: np.ndarray
    adj: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.adj.shape[0])


def as_csr64(offsets, adj, w) -> CsrGraph:
    return CsrGraph(np.ascontiguousarray(offsets, np.int64), np.ascontiguousarray(adj, np.int32),
                    np.ascontiguousarray(w, np.int64))


def mix64(z: int) -> int:
    return int(_load().orc_mix64(z & (2**64 - 1)))


def level_key(seed: int, level: int) -> int:
    return int(_load().orc_level_key(seed & (2**64 - 1), level))


def degrees(g: CsrGraph) -> np.ndarray:
    d = np.empty(g.n, np.int64)
    _load().orc_degrees(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, d.ctypes.data)
    return d


def lp_round(g: CsrGraph, labels, key: int) -> np.ndarray:
    lab, p = _c(labels, np.int32)
    out = np.empty(g.n, np.int32)
    _load().orc_lp_round(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, p,
                         key & (2**64 - 1), out.ctypes.data)
    return out


def lp_level(g: CsrGraph, key: int, lp_iters: int, converge: bool, lp_async: int = 0):
    """The rounds of one level from the identity labelling: (final labels, rounds run).
    lp_async: 0 synchronous, 1 asynchronous [R11], 2 asynchronous with the first round's
    restriction."""
    out = np.empty(g.n, np.int32)
    r = _load().orc_lp_level(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, key & (2**64 - 1),
                             lp_iters, 1 if converge else 0, out.ctypes.data, int(lp_async))
    return out, int(r)


def lp_round_async(g: CsrGraph, labels, key: int, rnd: int, blk: int = 128, waves: int = 8,
                   restrict_first: bool = False) -> np.ndarray:
    """One asynchronous round [R11] from `labels` (blocks of blk ids in `waves` waves)."""
    lab = np.array(labels, dtype=np.int32)
    _load().orc_lp_round_async(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, lab.ctypes.data,
                               key & (2**64 - 1), rnd, blk, waves, 1 if restrict_first else 0)
    return lab


def contract(g: CsrGraph, labels):
    """Returns (coarse graph, cid)."""
    lab, p = _c(labels, np.int32)
    cid = np.empty(g.n, np.int32)
    cn = ctypes.c_int64()
    coff = np.empty(g.n + 1, np.int64)
    cadj = np.empty(max(g.nnz, 1), np.int32)
    cw = np.empty(max(g.nnz, 1), np.int64)
    nnz = _load().orc_contract(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, p,
                               cid.ctypes.data, ctypes.byref(cn), coff.ctypes.data, cadj.ctypes.data,
                               cw.ctypes.data)
    h = CsrGraph(coff[: cn.value + 1].copy(), cadj[:nnz].copy(), cw[:nnz].copy())
    return h, cid


def correct(g: CsrGraph, labels):
    """The correcting step [R10] on a clustering: returns (cluster ids, their count)."""
    lab, p = _c(labels, np.int32)
    cid = np.empty(g.n, np.int32)
    k = _load().orc_correct(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data, p, cid.ctypes.data)
    return cid, int(k)


def _labels_call(name, g: CsrGraph, lambda_hat: int):
    out = np.empty(g.n, np.int32)
    cnt = getattr(_load(), name)(g.n, g.offsets.ctypes.data, g.adj.ctypes.data, g.w.ctypes.data,
                                 int(lambda_hat), out.ctypes.data)
    return out, int(cnt)


def pr_pass_a(g: CsrGraph, lambda_hat: int):
    """(labels = union-find roots, number of unions)."""
    return _labels_call("orc_pr_pass_a", g, lambda_hat)


def pr_pass_b(g: CsrGraph, lambda_hat: int):
    return _labels_call("orc_pr_pass_b", g, lambda_hat)


def noi_round(g: CsrGraph, lambda_hat: int):
    return _labels_call("orc_noi_round", g, lambda_hat)


@dataclass
class Result:
    cut: int
    side_bits: np.ndarray           # uint64 [ceil(n/64)]
    trace: list = field(default_factory=list)  # [(kind, level, n, nnz, lambda_hat)]

    def side(self, n: int) -> np.ndarray:
        """Boolean membership of each original vertex in the returned side."""
        bits = np.unpackbits(self.side_bits.view(np.uint8), bitorder="little")[:n]
        return bits.astype(bool)


def viecut(offsets, adj, w, seed: int = 1, lp_iters: int = 2, n0: int = 10000,
           pr_runs_max: int = 8, trace_cap: int = 4096, correct: bool = False, converge: bool = False,
           lp_async: int = 0, _lib=None) -> Result:
    """The whole deterministic method.  `w` may be int32 or int64.  correct: the
    correcting step on every label-propagation clustering (reading [R10]).  converge:
    at most lp_iters rounds per level, ending after a round in which at most 1/10000 of
    the vertices changed their label (the VieCut25 configuration, App. D).  lp_async: 1
    asynchronous rounds in shuffled 128-vertex blocks and eight waves [R11], 2 the same
    with the first round's restriction.  `_lib`
    (tests only) runs another build of oracle.cpp with the same entry points, e.g. one
    with a mistake planted to show that a pin catches it."""
    off, po = _c(offsets, np.int64)
    a, pa = _c(adj, np.int32)
    w = np.asarray(w)
    wbytes = 8 if w.dtype == np.int64 else 4
    ww, pw = _c(w, np.int64 if wbytes == 8 else np.int32)
    n = off.shape[0] - 1
    cut = ctypes.c_int64()
    bits = np.zeros((n + 63) // 64, np.uint64)
    tr = (OrcStep * trace_cap)()
    tl = ctypes.c_int64()
    lib = _lib if _lib is not None else _load()
    rc = lib.orc_viecut(n, po, pa, pw, wbytes, seed & (2**64 - 1), lp_iters, n0, pr_runs_max,
                            ctypes.byref(cut), bits.ctypes.data, tr, trace_cap, ctypes.byref(tl),
                            1 if correct else 0, 1 if converge else 0, int(lp_async))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    steps = [(tr[k].kind, tr[k].level, tr[k].n, tr[k].nnz, tr[k].lambda_hat)
             for k in range(min(tl.value, trace_cap))]
    return Result(int(cut.value), bits, steps)
