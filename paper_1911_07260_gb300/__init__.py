"""Ordered shortest paths on GB300: Python binding of ``libog.so``.

This module only marshals arguments to the C ABI declared in ``include/og.h``; every
step of the computation runs in the library's CUDA kernels.  There is no CPU fallback:
if ``libog.so`` is missing, every call raises.

Buffers may be numpy arrays (host) or torch CUDA tensors (device); the library detects
which.  ``stream`` defaults to torch's current CUDA stream when torch is in use.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libog.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "og.h")
_lib = None

OK, E_INVALID, E_OOM, E_CUDA, E_OVERFLOW, E_TIMEOUT, E_BUSY, E_ARENA, E_INTERNAL = range(9)
Q_SSSP, Q_PPSP, Q_ASTAR, Q_WBFS, Q_BF = 0, 1, 2, 3, 4
FUSION_OFF = 0xFFFFFFFE
FUSION_UNBOUNDED = 0xFFFFFFFF
ENGINE_DEFAULT, ENGINE_ROUNDS, ENGINE_ASYNC = 0, 1, 2
PRECHECK_ON, PRECHECK_OFF = 1, 2
LAYOUT_CSR, LAYOUT_ELL = 1, 2
PREFETCH_ON, PREFETCH_OFF = 1, 2
ORDER_AUTO, ORDER_HOT_FIRST, ORDER_USER = 0, 1, 2
KCORE_LAZY, KCORE_EAGER = 0, 1
UPDATE_EAGER, UPDATE_LAZY = 1, 2
UNREACHED = 0xFFFFFFFF


class OgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)}"
        if code in (E_CUDA, E_INTERNAL, E_TIMEOUT):
            msg += f" ({last_cuda_error()})"
        super().__init__(msg)


class Config(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_uint32), ("fusion_threshold", ctypes.c_uint32),
                ("expand_tile", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("ring_buckets", ctypes.c_uint32), ("engine", ctypes.c_uint32),
                ("precheck", ctypes.c_uint32), ("layout", ctypes.c_uint32),
                ("prefetch", ctypes.c_uint32), ("hub_degree", ctypes.c_uint32),
                ("bucket_update", ctypes.c_uint32), ("pull_divisor", ctypes.c_uint32),
                ("spin_limit_ns", ctypes.c_uint64), ("arena_entries", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("rounds", "fused_iters", "items", "stale", "relax", "improved",
                 "local_inserts", "global_inserts", "overflow_inserts", "redistributions",
                 "restarts", "kernel_ns", "flushes", "t_frontier_ns", "t_fused_ns",
                 "t_barrier_ns", "t_hub_ns")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Query(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("src", ctypes.c_uint32), ("dst", ctypes.c_uint32),
                ("delta", ctypes.c_uint32)]


def lib():
    """The loaded ``libog.so`` (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1911_07260_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        P = ctypes.POINTER
        sig = {
            "og_graph_upload": (i32, [vp, vp, vp, u32, u64, vp, P(vp)]),
            "og_graph_set_coords": (i32, [vp, vp, vp]),
            "og_graph_set_order": (i32, [vp, u32, vp]),
            "og_graph_get_order": (i32, [vp, P(u32), P(u32)]),
            "og_hot_first_order": (i32, [vp, u32, vp, P(u64)]),
            "og_graph_info": (i32, [vp, P(u32), P(u64), P(u32), P(u32)]),
            "og_graph_set_config": (i32, [vp, P(Config)]),
            "og_graph_get_config": (i32, [vp, P(Config)]),
            "og_graph_free": (None, [vp]),
            "og_config_default": (None, [P(Config)]),
            "og_sssp_delta": (i32, [vp, u32, u32, vp, vp]),
            "og_sssp_bellman_ford": (i32, [vp, u32, vp, P(Stats), vp]),
            "og_kcore": (i32, [vp, u32, P(Config), vp, P(Stats), vp]),
            "og_setcover": (i32, [vp, u32, vp, P(Config), vp, P(Stats), vp]),
            "og_wbfs": (i32, [vp, u32, vp, vp]),
            "og_ppsp": (i32, [vp, u32, u32, u32, P(u32), vp]),
            "og_astar": (i32, [vp, u32, u32, vp, u32, P(u32), vp]),
            "og_query_run": (i32, [vp, P(Query), P(Config), vp, P(u32), P(Stats), vp]),
            "og_batch_run": (i32, [vp, P(Query), u32, P(Config), vp, vp, P(Stats), vp]),
            "og_server_create": (i32, [vp, u32, P(Config), vp, P(vp)]),
            "og_server_submit": (i32, [vp, P(Query), u64]),
            "og_server_step": (i32, [vp, u32, P(u32)]),
            "og_server_poll": (i32, [vp, vp, vp, u32, P(u32)]),
            "og_server_slots": (i32, [vp, P(u32), P(u32)]),
            "og_server_free": (None, [vp]),
            "og_autotune": (i32, [vp, u32, vp, vp, u32, u32, u32, P(Config)]),
            "og_autotune_batch": (i32, [vp, vp, u32, u32, u32, P(Config)]),
            "og_strerror": (ctypes.c_char_p, [i32]),
            "og_last_cuda_error": (ctypes.c_char_p, []),
            "og_version": (i32, []),
            "og_sssp_delta_noalloc": (i32, [vp, vp, u32, u64, u32, u32, vp, vp]),
            "og_launch_status": (i32, [u32, u32, u32, u32, u32]),
            "og_probe_chain": (i32, [u32, u64, u64, u32, u32, u32, u32, P(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols(path: str = HEADER_PATH) -> list[str]:
    """Function names declared in include/og.h."""
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(og_\w+)\s*\(", text, re.M)))


def strerror(code: int) -> str:
    try:
        return lib().og_strerror(code).decode()
    except RuntimeError:
        return f"error {code}"


def last_cuda_error() -> str:
    return lib().og_last_cuda_error().decode()


def _check(code: int, where: str):
    if code != OK:
        raise OgError(code, where)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def config(**kw) -> Config:
    """A Config with every field 0 (= graph / library default) except those given."""
    c = Config()
    for k, v in kw.items():
        setattr(c, k, int(v))
    return c


class Graph:
    """A CSR graph resident on the device (``og_graph``)."""

    def __init__(self, offsets, nbr, w, stream=None):
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        nbr = np.ascontiguousarray(nbr, dtype=np.uint32)
        w = np.ascontiguousarray(w, dtype=np.uint32)
        n = offsets.shape[0] - 1
        h = ctypes.c_void_p()
        _check(lib().og_graph_upload(offsets.ctypes.data, nbr.ctypes.data if nbr.size else None,
                                     w.ctypes.data if w.size else None, n, nbr.shape[0],
                                     _stream(stream), ctypes.byref(h)), "og_graph_upload")
        self._h = h
        self.n = int(n)
        self.m = int(nbr.shape[0])

    @classmethod
    def from_csr(cls, g, stream=None, coords: bool = True):
        """Upload a ``graphgen.Graph``-like object (offsets, nbr, w, optional xy)."""
        obj = cls(g.offsets, g.nbr, g.w, stream)
        if coords and getattr(g, "xy", None) is not None:
            obj.set_coords(g.xy, stream)
        return obj

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("graph already freed")
        return self._h

    def set_coords(self, xy, stream=None):
        if isinstance(xy, np.ndarray):
            xy = np.ascontiguousarray(xy, dtype=np.float32)
        _check(lib().og_graph_set_coords(self.handle, _ptr(xy), _stream(stream)),
               "og_graph_set_coords")

    def set_order(self, order: int, stream=None):
        """Device vertex order: ORDER_AUTO, ORDER_HOT_FIRST or ORDER_USER (results keep
        the caller's ids in every order)."""
        _check(lib().og_graph_set_order(self.handle, order, _stream(stream)),
               "og_graph_set_order")

    def order(self) -> tuple:
        """(order in effect, vertices whose device id differs from their own)."""
        o, mv = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().og_graph_get_order(self.handle, ctypes.byref(o), ctypes.byref(mv)),
               "og_graph_get_order")
        return o.value, mv.value

    def info(self) -> dict:
        n, m, lo, hi = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().og_graph_info(self.handle, ctypes.byref(n), ctypes.byref(m),
                                   ctypes.byref(lo), ctypes.byref(hi)), "og_graph_info")
        return dict(n=n.value, m=m.value, min_w=lo.value, max_w=hi.value)

    def get_config(self) -> Config:
        c = Config()
        _check(lib().og_graph_get_config(self.handle, ctypes.byref(c)), "og_graph_get_config")
        return c

    def set_config(self, c: Config):
        _check(lib().og_graph_set_config(self.handle, ctypes.byref(c)), "og_graph_set_config")

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().og_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _alloc_dist(g: Graph, out, count: int = 1):
    if out is None:
        out = np.empty(count * g.n, np.uint32) if count > 1 else np.empty(g.n, np.uint32)
    return out


def sssp_delta(g: Graph, src: int, delta: int = 0, out=None, stream=None):
    """Delta-stepping SSSP with bucket fusion; returns ``out`` (uint32[n])."""
    out = _alloc_dist(g, out)
    _check(lib().og_sssp_delta(g.handle, src, delta, _ptr(out), _stream(stream)), "og_sssp_delta")
    return out


def bellman_ford(g: Graph, src: int, out=None, stream=None):
    """Unordered frontier-based Bellman-Ford; returns (``out`` uint32[n], Stats)."""
    out = _alloc_dist(g, out)
    st = Stats()
    _check(lib().og_sssp_bellman_ford(g.handle, src, _ptr(out), ctypes.byref(st), _stream(stream)),
           "og_sssp_bellman_ford")
    return out, st


def kcore(g: Graph, mode: int = KCORE_LAZY, cfg=None, out=None, stream=None):
    """Coreness of every vertex by peeling; returns (``out`` uint32[n], Stats)."""
    out = _alloc_dist(g, out)
    st = Stats()
    _check(lib().og_kcore(g.handle, mode, ctypes.byref(cfg) if cfg else None, _ptr(out),
                          ctypes.byref(st), _stream(stream)), "og_kcore")
    return out, st


def setcover(g: Graph, eps_ppm: int = 10000, priority=None, cfg=None, out=None, stream=None):
    """Approximate set cover of the sets S_v = adjacency of v; ``priority`` is a
    permutation of 0..n-1 (uint32, host array or device tensor; None = identity).
    Returns (``out`` uint32[n]: step in which each set joined, 0 = never; Stats)."""
    out = _alloc_dist(g, out)
    if isinstance(priority, np.ndarray):
        priority = np.ascontiguousarray(priority, dtype=np.uint32)
    st = Stats()
    _check(lib().og_setcover(g.handle, eps_ppm, _ptr(priority), ctypes.byref(cfg) if cfg else None,
                             _ptr(out), ctypes.byref(st), _stream(stream)), "og_setcover")
    return out, st


def wbfs(g: Graph, src: int, out=None, stream=None):
    """Weighted BFS (Delta = 1); returns ``out`` (uint32[n])."""
    out = _alloc_dist(g, out)
    _check(lib().og_wbfs(g.handle, src, _ptr(out), _stream(stream)), "og_wbfs")
    return out


def ppsp(g: Graph, src: int, dst: int, delta: int = 0, stream=None) -> int:
    d = ctypes.c_uint32()
    _check(lib().og_ppsp(g.handle, src, dst, delta, ctypes.byref(d), _stream(stream)), "og_ppsp")
    return int(d.value)


def astar(g: Graph, src: int, dst: int, delta: int = 0, coords=None, stream=None) -> int:
    d = ctypes.c_uint32()
    if isinstance(coords, np.ndarray):
        coords = np.ascontiguousarray(coords, dtype=np.float32)
    _check(lib().og_astar(g.handle, src, dst, _ptr(coords), delta, ctypes.byref(d),
                          _stream(stream)), "og_astar")
    return int(d.value)


def query_run(g: Graph, kind: int, src: int, dst: int = 0, delta: int = 0, cfg=None,
              out=None, stream=None):
    """Any query kind with an explicit schedule; returns (dist_out, d, Stats)."""
    q = Query(kind, src, dst, delta)
    st = Stats()
    d = ctypes.c_uint32()
    if out is None and kind in (Q_SSSP, Q_WBFS, Q_BF):
        out = np.empty(g.n, np.uint32)
    _check(lib().og_query_run(g.handle, ctypes.byref(q), ctypes.byref(cfg) if cfg else None,
                              _ptr(out), ctypes.byref(d), ctypes.byref(st), _stream(stream)),
           "og_query_run")
    return out, int(d.value), st


def batch_run(g: Graph, queries, cfg=None, out=None, want_dist: bool = True, stream=None):
    """Runs queries [(kind, src, dst, delta), ...] in one persistent launch.
    Returns (dist_out or None, d_out uint32[nq], Stats)."""
    nq = len(queries)
    arr = (Query * nq)(*[Query(*map(int, q)) for q in queries])
    if out is None and want_dist:
        out = np.empty(nq * g.n, np.uint32)
    d = np.zeros(nq, np.uint32)
    st = Stats()
    _check(lib().og_batch_run(g.handle, arr, nq, ctypes.byref(cfg) if cfg else None, _ptr(out),
                              d.ctypes.data, ctypes.byref(st), _stream(stream)), "og_batch_run")
    return out, d, st


class Server:
    """Continuous-batching query server (``og_server``)."""

    def __init__(self, g: Graph, max_slots: int = 0, cfg=None, stream=None):
        h = ctypes.c_void_p()
        _check(lib().og_server_create(g.handle, max_slots, ctypes.byref(cfg) if cfg else None,
                                      _stream(stream), ctypes.byref(h)), "og_server_create")
        self._h = h
        self.graph = g
        ms, nf = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().og_server_slots(h, ctypes.byref(ms), ctypes.byref(nf)), "og_server_slots")
        self.max_slots = ms.value

    def free_slots(self) -> int:
        ms, nf = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().og_server_slots(self._h, ctypes.byref(ms), ctypes.byref(nf)),
               "og_server_slots")
        return nf.value

    def submit(self, kind: int, src: int, dst: int, tag: int, delta: int = 0) -> bool:
        """Admits a query; False if every slot is busy."""
        q = Query(kind, src, dst, delta)
        r = lib().og_server_submit(self._h, ctypes.byref(q), tag)
        if r == E_BUSY:
            return False
        _check(r, "og_server_submit")
        return True

    def step(self, budget_us: int = 0) -> int:
        """One launch over the admitted queries, at most budget_us (0 = to completion);
        returns how many are still running."""
        n = ctypes.c_uint32()
        _check(lib().og_server_step(self._h, budget_us, ctypes.byref(n)), "og_server_step")
        return n.value

    def poll(self, cap: int = 4096):
        tags = np.zeros(cap, np.uint64)
        d = np.zeros(cap, np.uint32)
        n = ctypes.c_uint32()
        _check(lib().og_server_poll(self._h, tags.ctypes.data, d.ctypes.data, cap,
                                    ctypes.byref(n)), "og_server_poll")
        return tags[:n.value], d[:n.value]

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().og_server_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hot_first_order(degrees):
    """(device_to_user uint32[n], hot_edges): the hot-first order for these out-degrees,
    computed on the host (``og_hot_first_order``)."""
    deg = np.ascontiguousarray(degrees, dtype=np.uint32)
    out = np.empty(deg.shape[0], np.uint32)
    he = ctypes.c_uint64()
    _check(lib().og_hot_first_order(deg.ctypes.data if deg.size else None, deg.shape[0],
                                    out.ctypes.data if out.size else None, ctypes.byref(he)),
           "og_hot_first_order")
    return out, int(he.value)


def autotune(g: Graph, kind: int, srcs, dsts=None, delta_lo: int = 0, delta_hi: int = 0) -> Config:
    srcs = np.ascontiguousarray(srcs, dtype=np.uint32)
    dd = None if dsts is None else np.ascontiguousarray(dsts, dtype=np.uint32)
    c = Config()
    _check(lib().og_autotune(g.handle, kind, srcs.ctypes.data, None if dd is None else dd.ctypes.data,
                             srcs.shape[0], delta_lo, delta_hi, ctypes.byref(c)), "og_autotune")
    return c


def autotune_batch(g: Graph, queries, delta_lo: int = 0, delta_hi: int = 0) -> Config:
    """Tunes the schedule on a whole batch [(kind, src, dst, delta), ...]."""
    nq = len(queries)
    arr = (Query * nq)(*[Query(*map(int, q)) for q in queries])
    c = Config()
    _check(lib().og_autotune_batch(g.handle, arr, nq, delta_lo, delta_hi, ctypes.byref(c)),
           "og_autotune_batch")
    return c


def sssp_delta_noalloc(offsets, edges, n: int, m: int, src: int, delta: int, out,
                       stream=None):
    """Allocation-free SSSP: offsets (device uint32[n+1]), edges (device uint32[2m],
    interleaved neighbor/weight pairs) and out (device uint32[n]) are the caller's; the
    library's scratch is a fixed static device array (graphs of up to 2^20 vertices)."""
    _check(lib().og_sssp_delta_noalloc(_ptr(offsets), _ptr(edges), n, m, src, delta, _ptr(out),
                                       _stream(stream)), "og_sssp_delta_noalloc")
    return out


def launch_status(err: int, bad_code: int = 0, bad_val: int = 0, bad_aux: int = 0,
                  arena_out: bool = False) -> int:
    """Status the round-engine entry points derive from a launch's error word (no GPU
    needed): OG_E_INTERNAL > OG_E_TIMEOUT > OG_E_ARENA > OG_E_OVERFLOW > OG_OK."""
    return int(lib().og_launch_status(err, bad_code, bad_val, bad_aux, 1 if arena_out else 0))


def probe_chain(mode: int, nbytes: int, ctas: int, threads: int, hops: int,
                footprint: int = 0, chains: int = 1) -> float:
    """ns per dependent access: mode 0 L2 loads, 1 atomicMin round trips, 2 L1 loads;
    footprint (default: the whole array) = bytes of 128-byte lines the chains visit,
    spread evenly over the nbytes array; chains = independent chains per thread."""
    v = ctypes.c_double(0.0)
    _check(lib().og_probe_chain(mode, nbytes, footprint or nbytes, ctas, threads, chains,
                                hops, ctypes.byref(v)), "og_probe_chain")
    return float(v.value)


def version() -> int:
    return int(lib().og_version())
