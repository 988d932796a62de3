"""GB300 (sm_103a) implementation of VieCut, the inexact minimum-cut method of
"Practical Minimum Cut Algorithms" (Henzinger, Noe, Schulz, Strash; arXiv 1708.06127).

This module is a thin ctypes binding of the C ABI declared in ``include/viecut.h``:
the functions keep the C names and only marshal arguments.  Every step of the
method runs in the CUDA kernels of ``libviecut.so``; there is no CPU fallback.  If the
library is missing the import of any entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libviecut.so")
_lock = threading.Lock()
_lib = None

VIECUT_OK = 0
VIECUT_EINVAL = -1
VIECUT_ENOMEM = -2
VIECUT_ECUDA = -3
VIECUT_ETIMEOUT = -4
VIECUT_ECANCELLED = -5
VIECUT_EBUSY = -6

STEP_KINDS = {0: "initial", 1: "lp", 2: "pr_a", 3: "pr_b", 4: "noi"}


class ViecutError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"viecut error {code}: {msg}")
        self.code = code


class viecut_opts(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int64), ("pr_runs_max", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("validate", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("lp_group", ctypes.c_int32), ("emit_group", ctypes.c_int32), ("correct", ctypes.c_int32),
                ("lp_converge", ctypes.c_int32), ("lp_async", ctypes.c_int32)]


class viecut_stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_lp", ctypes.c_double), ("ms_contract", ctypes.c_double),
                ("ms_pr", ctypes.c_double), ("ms_noi", ctypes.c_double), ("ms_other", ctypes.c_double),
                ("ms_lp_kernel", ctypes.c_double), ("lp_launches", ctypes.c_int64), ("lp_nnz", ctypes.c_int64),
                ("lp_n", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("levels", ctypes.c_int64),
                ("trace_len", ctypes.c_int64), ("lp_bytes", ctypes.c_int64),
                ("first_group", ctypes.c_int32), ("emit_group", ctypes.c_int32),
                ("ms_contract_kernel", ctypes.c_double), ("ms_premerge_kernel", ctypes.c_double),
                ("contractions", ctypes.c_int64), ("contract_bytes", ctypes.c_int64),
                ("premerge_bytes", ctypes.c_int64)]


class viecut_graph_desc(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("adj", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("m", ctypes.c_int64)]


class viecut_batch_stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("super_steps", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("graphs", ctypes.c_int64), ("vertices", ctypes.c_int64), ("entries", ctypes.c_int64)]


class viecut_server_opts(ctypes.Structure):
    _fields_ = [("base", viecut_opts), ("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("lp_iters", ctypes.c_int32), ("solo_min_n", ctypes.c_int64), ("solo_lanes", ctypes.c_int32),
                ("solo_exact", ctypes.c_int32)]


class viecut_server_stats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("max_resident", ctypes.c_int64), ("super_steps", ctypes.c_int64), ("joins", ctypes.c_int64),
                ("budget_used", ctypes.c_int64), ("solo_completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("failed", ctypes.c_int64)]


class viecut_request_info(ctypes.Structure):
    _fields_ = [("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("lane", ctypes.c_int32), ("pad", ctypes.c_int32), ("n", ctypes.c_int64), ("m", ctypes.c_int64)]


class viecut_step(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("lambda_hat", ctypes.c_int64)]


# (name, restype, argtypes) of every entry point declared in include/viecut.h
_vp, _i64, _i32, _u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
_pvp = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = [
    ("viecut_struct_sizes", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("viecut_opts_init", ctypes.c_int, [_vp]),
    ("viecut_create", ctypes.c_int, [_pvp, _vp, _vp, _i64, _i64, _vp, _vp]),
    ("viecut_create_device", ctypes.c_int, [_pvp, _vp, _vp, _i64, _i64, _vp, _vp]),
    ("viecut_run", ctypes.c_int, [_vp, _u64, _i32, _vp, _vp]),
    ("viecut_load", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _vp]),
    ("viecut_solve", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _vp, _u64, _i32, _vp, _vp]),
    ("viecut_run_device", ctypes.c_int, [_vp, _u64, _i32, _vp, _vp]),
    ("viecut_get_stats", ctypes.c_int, [_vp, _vp]),
    ("viecut_get_trace", ctypes.c_int, [_vp, _vp, _i64, _vp]),
    ("viecut_destroy", ctypes.c_int, [_vp]),
    ("viecut_last_error", ctypes.c_char_p, []),
    ("viecut_launch_count", ctypes.c_int64, []),
    ("viecut_debug_fail_device_allocs", ctypes.c_int, [_i64, _i64]),
    ("viecut_graph_upload", ctypes.c_int, [_pvp, _vp, _vp, _vp, _i64, _i64, _i32]),
    ("viecut_graph_shape", ctypes.c_int, [_vp, _vp, _vp]),
    ("viecut_graph_download", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("viecut_graph_free", ctypes.c_int, [_vp]),
    ("viecut_step_degrees", ctypes.c_int, [_vp, _vp]),
    ("viecut_step_lp", ctypes.c_int, [_vp, _vp, _u64, _i32, _vp]),
    ("viecut_step_contract", ctypes.c_int, [_vp, _vp, _pvp, _vp]),
    ("viecut_step_pr_a", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("viecut_step_pr_b", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("viecut_step_noi_round", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("viecut_noi_round_noalloc", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    ("viecut_batch_create", ctypes.c_int, [_pvp, _vp, _i32, _vp]),
    ("viecut_batch_run", ctypes.c_int, [_vp, _u64, _i32, _vp, _vp]),
    ("viecut_batch_side_words", ctypes.c_int, [_vp, _vp]),
    ("viecut_batch_get_trace", ctypes.c_int, [_vp, _i32, _vp, _i64, _vp]),
    ("viecut_batch_get_stats", ctypes.c_int, [_vp, _vp]),
    ("viecut_batch_destroy", ctypes.c_int, [_vp]),
    ("viecut_server_opts_init", ctypes.c_int, [_vp]),
    ("viecut_server_start", ctypes.c_int, [_pvp, _vp]),
    ("viecut_server_submit", ctypes.c_int, [_vp, _vp, _u64, _vp]),
    ("viecut_server_poll", ctypes.c_int, [_vp, _u64, _vp, _vp, _vp]),
    ("viecut_server_poll_info", ctypes.c_int, [_vp, _u64, _vp, _vp, _vp]),
    ("viecut_server_wait", ctypes.c_int, [_vp, _u64, ctypes.c_double, _vp, _vp, _vp]),
    ("viecut_server_cancel", ctypes.c_int, [_vp, _u64]),
    ("viecut_server_get_stats", ctypes.c_int, [_vp, _vp]),
    ("viecut_server_stop", ctypes.c_int, [_vp]),
]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded libviecut.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with paper_1708_06127_gb300.build() "
                                  "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != VIECUT_OK:
        raise ViecutError(rc, lib().viecut_last_error().decode())


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def viecut_opts_init(**kw) -> viecut_opts:
    o = viecut_opts()
    _check(lib().viecut_opts_init(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def viecut_create(offsets, adj, n: int, m: int, weights, opts: viecut_opts | None = None):
    h = ctypes.c_void_p()
    _check(lib().viecut_create(ctypes.byref(h), _ptr(offsets), _ptr(adj), n, m, _ptr(weights),
                               ctypes.byref(opts) if opts is not None else None))
    return h


def viecut_create_device(d_offsets, d_adj, n: int, m: int, d_weights, opts: viecut_opts | None = None):
    h = ctypes.c_void_p()
    _check(lib().viecut_create_device(ctypes.byref(h), _ptr(d_offsets), _ptr(d_adj), n, m, _ptr(d_weights),
                                      ctypes.byref(opts) if opts is not None else None))
    return h


def viecut_load(h, offsets, adj, n: int, m: int, weights) -> None:
    _check(lib().viecut_load(h, _ptr(offsets), _ptr(adj), n, m, _ptr(weights)))


def viecut_solve(h, offsets, adj, n: int, m: int, weights, seed: int, lp_iters: int, side_bits=None) -> int:
    cut = ctypes.c_int64()
    _check(lib().viecut_solve(h, _ptr(offsets), _ptr(adj), n, m, _ptr(weights), seed & (2**64 - 1), lp_iters,
                              ctypes.byref(cut), _ptr(side_bits)))
    return int(cut.value)


def viecut_run(h, seed: int, lp_iters: int, side_bits=None) -> int:
    cut = ctypes.c_int64()
    _check(lib().viecut_run(h, seed & (2**64 - 1), lp_iters, ctypes.byref(cut), _ptr(side_bits)))
    return int(cut.value)


def viecut_run_device(h, seed: int, lp_iters: int, d_cut, d_side_bits=None):
    _check(lib().viecut_run_device(h, seed & (2**64 - 1), lp_iters, _ptr(d_cut), _ptr(d_side_bits)))


def viecut_get_stats(h) -> dict:
    s = viecut_stats()
    _check(lib().viecut_get_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in viecut_stats._fields_}


def viecut_get_trace(h) -> list:
    cap = 4096
    buf = (viecut_step * cap)()
    ln = ctypes.c_int64()
    _check(lib().viecut_get_trace(h, buf, cap, ctypes.byref(ln)))
    return [(buf[i].kind, buf[i].level, buf[i].n, buf[i].nnz, buf[i].lambda_hat) for i in range(min(cap, ln.value))]


def viecut_destroy(h):
    if h:
        _check(lib().viecut_destroy(h))


def viecut_launch_count() -> int:
    return int(lib().viecut_launch_count())


def viecut_debug_fail_device_allocs(after: int, count: int) -> None:
    """Test hook: after `after` more device allocations, `count` fail with VIECUT_ENOMEM."""
    _check(lib().viecut_debug_fail_device_allocs(int(after), int(count)))


# ----------------------------------------------------------------- step API
def viecut_graph_upload(offsets, adj, weights, device: int = 0):
    off = np.ascontiguousarray(offsets, np.int64)
    a = np.ascontiguousarray(adj, np.int32)
    w = np.ascontiguousarray(weights, np.int64)
    g = ctypes.c_void_p()
    _check(lib().viecut_graph_upload(ctypes.byref(g), off.ctypes.data, a.ctypes.data, w.ctypes.data,
                                     off.shape[0] - 1, a.shape[0], device))
    return g


def viecut_graph_shape(g):
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().viecut_graph_shape(g, ctypes.byref(n), ctypes.byref(nnz)))
    return int(n.value), int(nnz.value)


def viecut_graph_download(g):
    n, nnz = viecut_graph_shape(g)
    off = np.empty(n + 1, np.int64)
    adj = np.empty(max(nnz, 1), np.int32)
    w = np.empty(max(nnz, 1), np.int64)
    _check(lib().viecut_graph_download(g, off.ctypes.data, adj.ctypes.data, w.ctypes.data))
    return off, adj[:nnz], w[:nnz]


def viecut_graph_free(g):
    if g:
        _check(lib().viecut_graph_free(g))


def viecut_step_degrees(g) -> np.ndarray:
    n, _ = viecut_graph_shape(g)
    d = np.empty(n, np.int64)
    _check(lib().viecut_step_degrees(g, d.ctypes.data))
    return d


def viecut_step_lp(g, lab_in, key: int, rounds: int) -> np.ndarray:
    n, _ = viecut_graph_shape(g)
    out = np.empty((rounds, n), np.int32)
    li = None if lab_in is None else np.ascontiguousarray(lab_in, np.int32)
    _check(lib().viecut_step_lp(g, None if li is None else li.ctypes.data, key & (2**64 - 1), rounds, out.ctypes.data))
    return out


def viecut_step_contract(g, labels):
    n, _ = viecut_graph_shape(g)
    lab = np.ascontiguousarray(labels, np.int32)
    cid = np.empty(n, np.int32)
    out = ctypes.c_void_p()
    _check(lib().viecut_step_contract(g, lab.ctypes.data, ctypes.byref(out), cid.ctypes.data))
    return out, cid


def _step_labels(name, g, lambda_hat):
    n, _ = viecut_graph_shape(g)
    lab = np.empty(n, np.int32)
    ch = ctypes.c_int32()
    _check(getattr(lib(), name)(g, int(lambda_hat), lab.ctypes.data, ctypes.byref(ch)))
    return lab, int(ch.value)


def viecut_step_pr_a(g, lambda_hat):
    return _step_labels("viecut_step_pr_a", g, lambda_hat)


def viecut_step_pr_b(g, lambda_hat):
    return _step_labels("viecut_step_pr_b", g, lambda_hat)


def viecut_step_noi_round(g, lambda_hat):
    return _step_labels("viecut_step_noi_round", g, lambda_hat)


def viecut_noi_round_noalloc(d_offsets, d_adj, d_weights, n: int, lambda_hat: int, d_labels, d_changed,
                             stream=None):
    """Allocation-free exact-step round on device tensors (see include/viecut.h)."""
    _check(lib().viecut_noi_round_noalloc(_ptr(d_offsets), _ptr(d_adj), _ptr(d_weights), n, int(lambda_hat),
                                          _ptr(d_labels), _ptr(d_changed), stream))


# ----------------------------------------------------------------- batches
def viecut_batch_create(graphs, opts: viecut_opts | None = None):
    """graphs: sequence of (offsets int64, adj int32, weights int32) host arrays."""
    descs = (viecut_graph_desc * len(graphs))()
    keep = []
    for i, (off, adj, w) in enumerate(graphs):
        off = np.ascontiguousarray(off, np.int64)
        adj = np.ascontiguousarray(adj, np.int32)
        w = np.ascontiguousarray(w, np.int32)
        keep.append((off, adj, w))
        descs[i] = viecut_graph_desc(off.ctypes.data, adj.ctypes.data, w.ctypes.data, off.shape[0] - 1, adj.shape[0])
    b = ctypes.c_void_p()
    _check(lib().viecut_batch_create(ctypes.byref(b), descs, len(graphs), ctypes.byref(opts) if opts else None))
    return b


def viecut_batch_side_words(b) -> int:
    w = ctypes.c_int64()
    _check(lib().viecut_batch_side_words(b, ctypes.byref(w)))
    return int(w.value)


def viecut_batch_run(b, k: int, seed: int, lp_iters: int, side_bits=None) -> np.ndarray:
    cuts = np.empty(k, np.int64)
    _check(lib().viecut_batch_run(b, seed & (2**64 - 1), lp_iters, cuts.ctypes.data, _ptr(side_bits)))
    return cuts


def viecut_batch_get_trace(b, g: int) -> list:
    cap = 4096
    buf = (viecut_step * cap)()
    ln = ctypes.c_int64()
    _check(lib().viecut_batch_get_trace(b, g, buf, cap, ctypes.byref(ln)))
    return [(buf[i].kind, buf[i].level, buf[i].n, buf[i].nnz, buf[i].lambda_hat) for i in range(min(cap, ln.value))]


def viecut_batch_get_stats(b) -> dict:
    st = viecut_batch_stats()
    _check(lib().viecut_batch_get_stats(b, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in viecut_batch_stats._fields_}


def viecut_batch_destroy(b):
    if b:
        _check(lib().viecut_batch_destroy(b))


class Batch:
    """Owns a batch of graphs; ``run`` returns (cut values, list of side bitmaps)."""

    def __init__(self, graphs, n0: int = 10000, pr_runs_max: int = 8, device: int = 0, stream=None,
                 validate: int = 1):
        self.ns = [int(np.asarray(g[0]).shape[0] - 1) for g in graphs]
        o = viecut_opts_init(n0=n0, pr_runs_max=pr_runs_max, device=device, stream=stream, validate=validate)
        self.b = viecut_batch_create(graphs, o)
        self.words = viecut_batch_side_words(self.b)

    def run(self, seed: int = 1, lp_iters: int = 2):
        bits = np.zeros(max(1, self.words), np.uint64)
        cuts = viecut_batch_run(self.b, len(self.ns), seed, lp_iters, bits)
        out, at = [], 0
        for n in self.ns:
            w = (n + 63) // 64
            out.append(bits[at:at + w].copy())
            at += w
        return cuts, out

    def trace(self, g: int) -> list:
        return viecut_batch_get_trace(self.b, g)

    def stats(self) -> dict:
        return viecut_batch_get_stats(self.b)

    def close(self):
        if self.b:
            viecut_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- serving
def viecut_server_opts_init(**kw) -> viecut_server_opts:
    o = viecut_server_opts()
    _check(lib().viecut_server_opts_init(ctypes.byref(o)))
    for k, v in kw.items():
        if k in ("n0", "pr_runs_max", "device", "stream", "lp_group", "emit_group", "correct", "lp_converge",
                 "lp_async"):
            setattr(o.base, k, v)
        else:
            setattr(o, k, v)
    return o


def viecut_server_start(opts: viecut_server_opts | None = None):
    s = ctypes.c_void_p()
    _check(lib().viecut_server_start(ctypes.byref(s), ctypes.byref(opts) if opts else None))
    return s


def viecut_server_submit(s, offsets, adj, weights, seed: int) -> int:
    off = np.ascontiguousarray(offsets, np.int64)
    a = np.ascontiguousarray(adj, np.int32)
    w = np.ascontiguousarray(weights, np.int32)
    d = viecut_graph_desc(off.ctypes.data, a.ctypes.data, w.ctypes.data, off.shape[0] - 1, a.shape[0])
    t = ctypes.c_uint64()
    _check(lib().viecut_server_submit(s, ctypes.byref(d), seed & (2**64 - 1), ctypes.byref(t)))
    return int(t.value)


def viecut_server_poll(s, ticket: int, n: int):
    """None while the request runs, else (cut, side bitmap, latency in ms)."""
    cut = ctypes.c_int64()
    lat = ctypes.c_double()
    bits = np.zeros(max(1, (n + 63) // 64), np.uint64)
    rc = lib().viecut_server_poll(s, ticket, ctypes.byref(cut), bits.ctypes.data, ctypes.byref(lat))
    if rc == VIECUT_EBUSY:
        return None
    _check(rc)
    return int(cut.value), bits, float(lat.value)


def _info_dict(info: viecut_request_info) -> dict:
    return {k: getattr(info, k) for k, _ in viecut_request_info._fields_ if k != "pad"}


def viecut_server_poll_info(s, ticket: int, n: int):
    """None while the request runs, else (cut, side bitmap, timing dict)."""
    cut = ctypes.c_int64()
    info = viecut_request_info()
    bits = np.zeros(max(1, (n + 63) // 64), np.uint64)
    rc = lib().viecut_server_poll_info(s, ticket, ctypes.byref(cut), bits.ctypes.data, ctypes.byref(info))
    if rc == VIECUT_EBUSY:
        return None
    _check(rc)
    return int(cut.value), bits, _info_dict(info)


def viecut_server_wait(s, ticket: int, n: int, timeout_ms: float):
    """(cut, side bitmap, timing dict); raises ViecutError (VIECUT_ETIMEOUT) when the request
    has not finished within timeout_ms."""
    cut = ctypes.c_int64()
    info = viecut_request_info()
    bits = np.zeros(max(1, (n + 63) // 64), np.uint64)
    _check(lib().viecut_server_wait(s, ticket, float(timeout_ms), ctypes.byref(cut), bits.ctypes.data,
                                    ctypes.byref(info)))
    return int(cut.value), bits, _info_dict(info)


def viecut_server_cancel(s, ticket: int) -> None:
    _check(lib().viecut_server_cancel(s, ticket))


def viecut_server_get_stats(s) -> dict:
    st = viecut_server_stats()
    _check(lib().viecut_server_get_stats(s, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in viecut_server_stats._fields_}


def viecut_server_stop(s):
    if s:
        _check(lib().viecut_server_stop(s))


class Server:
    """Continuous-batching min-cut server on one GPU."""

    def __init__(self, hbm_budget_bytes: int = 120 << 30, max_slots: int = 1024, lp_iters: int = 2,
                 n0: int = 10000, pr_runs_max: int = 8, device: int = 0, solo_min_n: int = 1 << 16,
                 solo_lanes: int = 8, solo_exact: bool = True):
        o = viecut_server_opts_init(hbm_budget_bytes=hbm_budget_bytes, max_slots=max_slots, lp_iters=lp_iters,
                                    n0=n0, pr_runs_max=pr_runs_max, device=device, solo_min_n=solo_min_n,
                                    solo_lanes=solo_lanes, solo_exact=int(solo_exact))
        self.s = viecut_server_start(o)
        self.sizes = {}

    def submit(self, offsets, adj, weights, seed: int = 1) -> int:
        t = viecut_server_submit(self.s, offsets, adj, weights, seed)
        self.sizes[t] = int(np.asarray(offsets).shape[0] - 1)
        return t

    def poll(self, ticket: int):
        try:
            r = viecut_server_poll(self.s, ticket, self.sizes[ticket])
        except ViecutError:
            self.sizes.pop(ticket, None)  # a refused request is answered once
            raise
        if r is not None:
            del self.sizes[ticket]
        return r

    def poll_info(self, ticket: int):
        """None while the request runs, else (cut, side bitmap, timing dict)."""
        try:
            r = viecut_server_poll_info(self.s, ticket, self.sizes[ticket])
        except ViecutError:
            self.sizes.pop(ticket, None)  # answered once (refused, cancelled, failed)
            raise
        if r is not None:
            del self.sizes[ticket]
        return r

    def wait(self, ticket: int, timeout: float = 600.0):
        """(cut, side bitmap, latency in ms), waiting on the host at most `timeout` seconds
        (ViecutError with VIECUT_ETIMEOUT after it; the ticket stays valid)."""
        try:
            cut, bits, info = viecut_server_wait(self.s, ticket, self.sizes[ticket], 1000.0 * timeout)
        except ViecutError as e:
            if e.code != VIECUT_ETIMEOUT:
                self.sizes.pop(ticket, None)
            raise
        del self.sizes[ticket]
        return cut, bits, info["latency_ms"]

    def cancel(self, ticket: int) -> None:
        viecut_server_cancel(self.s, ticket)

    def stats(self) -> dict:
        return viecut_server_get_stats(self.s)

    def close(self):
        if self.s:
            viecut_server_stop(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- convenience
class MinCut:
    """Owns a handle over one graph; ``run`` returns (cut value, side bitmap)."""

    def __init__(self, offsets, adj, weights, n0: int = 10000, pr_runs_max: int = 8, device: int = 0,
                 stream=None, validate: int = 1, timing: bool = False, on_device: bool = False,
                 lp_group: int = 0, emit_group: int = 0, correct: bool = False, lp_converge: bool = False,
                 lp_async: int = 0):
        n = int(offsets.shape[0] - 1)
        m = int(adj.shape[0])
        o = viecut_opts_init(n0=n0, pr_runs_max=pr_runs_max, device=device, stream=stream,
                             validate=validate, timing=int(timing), lp_group=lp_group, emit_group=emit_group,
                             correct=int(correct), lp_converge=int(lp_converge), lp_async=int(lp_async))
        self.n, self.m = n, m
        self._keep = (offsets, adj, weights)
        self.h = (viecut_create_device if on_device else viecut_create)(offsets, adj, n, m, weights, o)

    def load(self, offsets, adj, weights):
        """Rebinds the handle to another host graph, reusing its device buffers."""
        n = int(offsets.shape[0] - 1)
        m = int(adj.shape[0])
        viecut_load(self.h, offsets, adj, n, m, weights)
        self.n, self.m = n, m
        self._keep = (offsets, adj, weights)

    def solve(self, offsets, adj, weights, seed: int = 1, lp_iters: int = 2):
        """Loads another host graph and runs on it in one call."""
        n = int(offsets.shape[0] - 1)
        m = int(adj.shape[0])
        bits = np.zeros((n + 63) // 64, np.uint64)
        cut = viecut_solve(self.h, offsets, adj, n, m, weights, seed, lp_iters, bits)
        self.n, self.m = n, m
        self._keep = (offsets, adj, weights)
        return cut, bits

    def run(self, seed: int = 1, lp_iters: int = 2):
        bits = np.zeros((self.n + 63) // 64, np.uint64)
        cut = viecut_run(self.h, seed, lp_iters, bits)
        return cut, bits

    def stats(self) -> dict:
        return viecut_get_stats(self.h)

    def trace(self) -> list:
        return viecut_get_trace(self.h)

    def close(self):
        if self.h:
            viecut_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exact_min_cut(offsets, adj, weights, device: int = 0, on_device: bool = False):
    """Exact minimum cut by the rounds of Nagamochi, Ono and Ibaraki alone (Sec. 3): the
    method with n0 at least the vertex count, so no label-propagation level runs and the
    exact step starts on the input graph.  Returns (cut value, side bitmap)."""
    n = int(offsets.shape[0] - 1)
    with MinCut(offsets, adj, weights, n0=max(n, 2), device=device, on_device=on_device) as mc:
        return mc.run(1, 0)
