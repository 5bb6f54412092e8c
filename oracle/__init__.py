"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It computes the plain definition of shortest-path distances
(``oracle.c``: Dijkstra, BFS, Bellman-Ford, certificate check) and
k-core coreness by peeling and a linear-time certificate of coreness, approximate set
cover by bucketed nearly independent steps and a certificate for set covers, and shares
no code with
the CUDA path in ``paper_1911_07260_gb300``.

Each wrapper takes a ``graphgen.Graph`` (CSR: uint64 offsets, uint32 neighbours,
uint32 weights) and returns uint32 distances with 0xFFFFFFFF = unreachable.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

UNREACHED = 0xFFFFFFFF
SATURATED = 0xFFFFFFFE
OK, OVERFLOW, INVALID, NOMEM = 0, 1, -1, -2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (plain C, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, u32 = ctypes.c_void_p, ctypes.c_uint32
        L.or_dijkstra.restype = ctypes.c_int
        L.or_dijkstra.argtypes = [u32, vp, vp, vp, u32, u32, vp]
        L.or_bfs.restype = ctypes.c_int
        L.or_bfs.argtypes = [u32, vp, vp, u32, vp]
        L.or_bellman_ford.restype = ctypes.c_int
        L.or_bellman_ford.argtypes = [u32, vp, vp, vp, u32, vp]
        L.or_check_sssp.restype = ctypes.c_int
        L.or_check_sssp.argtypes = [u32, vp, vp, vp, u32, vp, vp]
        L.or_kcore.restype = ctypes.c_int
        L.or_kcore.argtypes = [u32, vp, vp, vp]
        L.or_setcover.restype = ctypes.c_int
        L.or_setcover.argtypes = [u32, vp, vp, u32, vp, vp, vp]
        L.or_check_kcore.restype = ctypes.c_int
        L.or_check_kcore.argtypes = [u32, vp, vp, vp, vp]
        L.or_check_setcover.restype = ctypes.c_int
        L.or_check_setcover.argtypes = [u32, vp, vp, u32, vp, ctypes.c_uint64, vp]
        _lib = L
    return _lib


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
    nbr = np.ascontiguousarray(g.nbr, dtype=np.uint32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    return off, nbr, w


def _status(st: int, allow_overflow: bool) -> int:
    if st == INVALID:
        raise OracleError("invalid arguments")
    if st == NOMEM:
        raise OracleError("out of host memory")
    if st == OVERFLOW and not allow_overflow:
        raise OracleError("a finite distance does not fit in uint32 (>= 0xFFFFFFFE)")
    return st


def dijkstra(g, src: int, target: int | None = None, allow_overflow: bool = False) -> np.ndarray:
    """All distances from ``src`` (or, with ``target``, a run that stops once the target
    is settled; only ``result[target]`` is then final)."""
    off, nbr, w = _csr(g)
    out = np.empty(g.n, np.uint32)
    st = _load().or_dijkstra(g.n, off.ctypes.data, nbr.ctypes.data, w.ctypes.data, int(src),
                             UNREACHED if target is None else int(target), out.ctypes.data)
    _status(st, allow_overflow)
    return out


def ppsp(g, src: int, target: int) -> int:
    """Shortest-path distance from ``src`` to ``target`` (0xFFFFFFFF if unreachable)."""
    return int(dijkstra(g, src, target)[target])


def bfs(g, src: int) -> np.ndarray:
    """Hop counts from ``src``."""
    off, nbr, _ = _csr(g)
    out = np.empty(g.n, np.uint32)
    _status(_load().or_bfs(g.n, off.ctypes.data, nbr.ctypes.data, int(src), out.ctypes.data),
            False)
    return out


def bellman_ford(g, src: int, allow_overflow: bool = False) -> np.ndarray:
    """All distances from ``src`` by repeated full relaxation passes."""
    off, nbr, w = _csr(g)
    out = np.empty(g.n, np.uint32)
    st = _load().or_bellman_ford(g.n, off.ctypes.data, nbr.ctypes.data, w.ctypes.data,
                                 int(src), out.ctypes.data)
    _status(st, allow_overflow)
    return out


def check_sssp(g, src: int, dist: np.ndarray) -> tuple[int, int]:
    """Certificate check; returns (code, vertex): code 0 = valid (see oracle.c)."""
    off, nbr, w = _csr(g)
    d = np.ascontiguousarray(dist, dtype=np.uint32)
    bad = ctypes.c_uint32(0)
    code = _load().or_check_sssp(g.n, off.ctypes.data, nbr.ctypes.data, w.ctypes.data,
                                 int(src), d.ctypes.data, ctypes.byref(bad))
    if code == INVALID:
        raise OracleError("invalid arguments")
    return int(code), int(bad.value)


def kcore(g) -> np.ndarray:
    """Coreness of every vertex (peeling; degrees count CSR entries)."""
    off, nbr, _ = _csr(g)
    out = np.empty(g.n, np.uint32)
    _status(_load().or_kcore(g.n, off.ctypes.data, nbr.ctypes.data, out.ctypes.data), False)
    return out


def check_kcore(g, core) -> tuple[int, int]:
    """Certificate of a coreness vector (``oracle.c``, ``or_check_kcore``), O(n + m).
    Returns (code, vertex): 0 = what ``kcore`` computes; 1 = a vertex keeps fewer than
    core[v] of its entries once every entry w -> v with core[w] < core[v] is taken away
    (its value is too high; on a symmetric graph: fewer than core[v] neighbours of value
    >= core[v]); 2 = a vertex of some level cannot be extracted at that level (a value
    too low somewhere)."""
    off, nbr, _ = _csr(g)
    c = np.ascontiguousarray(core, dtype=np.uint32)
    if c.shape != (g.n,):
        raise OracleError("one coreness per vertex")
    bad = ctypes.c_uint32(0)
    code = _load().or_check_kcore(g.n, off.ctypes.data, nbr.ctypes.data, c.ctypes.data,
                                  ctypes.byref(bad))
    _status(code if code < 0 else 0, False)
    return int(code), int(bad.value)


def setcover(g, pri, eps_ppm: int = 10000) -> tuple[np.ndarray, int]:
    """Approximate unweighted set cover of the sets S_v = adjacency of v (``oracle.c``,
    ``or_setcover``).  ``pri`` is a permutation of 0..n-1 (the sets' priorities).
    Returns (step at which each set joined the cover, 0 = never; number of steps)."""
    off, nbr, _ = _csr(g)
    p = np.ascontiguousarray(pri, dtype=np.uint32)
    if p.shape != (g.n,):
        raise OracleError("priorities must have one entry per vertex")
    out = np.empty(g.n, np.uint32)
    steps = ctypes.c_uint64(0)
    _status(_load().or_setcover(g.n, off.ctypes.data, nbr.ctypes.data, int(eps_ppm),
                                p.ctypes.data, out.ctypes.data, ctypes.byref(steps)), False)
    return out, int(steps.value)


def check_setcover(g, step_out, steps: int, eps_ppm: int = 10000) -> tuple[int, int]:
    """Certificate of a set cover given as join steps (``oracle.c``,
    ``or_check_setcover``).  Returns (code, where): 0 = certified; 1 = an element of the
    universe stays uncovered (where = element); 2 = a set joined with too few new
    elements (where = set); 3 = the sets of a step overlap too much (where = step);
    4 = a step number beyond ``steps`` (where = set)."""
    off, nbr, _ = _csr(g)
    s = np.ascontiguousarray(step_out, dtype=np.uint32)
    bad = ctypes.c_uint32(0)
    code = _load().or_check_setcover(g.n, off.ctypes.data, nbr.ctypes.data, int(eps_ppm),
                                     s.ctypes.data, int(steps), ctypes.byref(bad))
    _status(code if code < 0 else 0, False)
    return int(code), int(bad.value)
