"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only lays out graphs and queries (vertices, edges, weights, coordinates,
sources and targets, set priorities); it holds none of the shortest-path, k-core or
set cover arithmetic.  The large families
(grid, road-like grid, R-MAT) are built by ``graphgen.cpp`` (compiled by :func:`build`);
small irregular test graphs are built here with numpy.  All draws are seeded.

Workload recipes (the paper's own datasets -- RoadUSA, Germany, Massachusetts, social
and web graphs, the table of datasets in Section 6 -- are not available;
these synthetic graphs stand in for them):

* ``grid(256, 256, 1, 1000, seed=1)``: 4-neighbour grid, weights uniform in [1, 1000).
* ``road(side, 0.15, 0.02, seed=1)``: road-like grid (15% of grid edges dropped, 2% of
  unit cells get one diagonal, largest component kept, weight
  ``max(round(100*len*U[1,1.5)), ceil(100*len))``) with float32 integral coordinates.
* ``rmat(24, 16, .57, .19, .19, wlo, whi, seed=1)``: R-MAT, ids shuffled, self loops and
  duplicates dropped, symmetrised.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so in place (host code, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, u32, u64, f64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        L.gg_grid.restype = vp
        L.gg_grid.argtypes = [u32, u32, u32, u32, u64]
        L.gg_road.restype = vp
        L.gg_road.argtypes = [u32, f64, f64, u64]
        L.gg_rmat.restype = vp
        L.gg_rmat.argtypes = [u32, u32, f64, f64, f64, u32, u32, u64]
        L.gg_n.restype = u32
        L.gg_n.argtypes = [vp]
        L.gg_m.restype = u64
        L.gg_m.argtypes = [vp]
        L.gg_has_xy.restype = ctypes.c_int
        L.gg_has_xy.argtypes = [vp]
        L.gg_side_rows.restype = u32
        L.gg_side_rows.argtypes = [vp]
        L.gg_side_cols.restype = u32
        L.gg_side_cols.argtypes = [vp]
        L.gg_copy.restype = None
        L.gg_copy.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gg_free.restype = None
        L.gg_free.argtypes = [vp]
        L.gg_reweight.restype = None
        L.gg_reweight.argtypes = [u32, vp, vp, vp, u32, u32, u64]
        _lib = L
    return _lib


@dataclass
class Graph:
    """CSR graph: ``offsets`` uint64[n+1], ``nbr`` uint32[m], ``w`` uint32[m].

    ``xy`` is float32[n, 2] (x = column, y = row) for grid-shaped graphs, else None.
    ``grid2id`` maps a grid position ``row*cols+col`` to a vertex id (-1 if absent).
    """
    name: str
    offsets: np.ndarray
    nbr: np.ndarray
    w: np.ndarray
    xy: np.ndarray | None = None
    grid2id: np.ndarray | None = None
    rows: int = 0
    cols: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.nbr.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def _take(h, name: str, meta: dict) -> Graph:
    L = _load()
    if not h:
        raise ValueError(f"graph generator rejected its arguments ({name})")
    try:
        n, m = L.gg_n(h), L.gg_m(h)
        off = np.empty(n + 1, np.uint64)
        nbr = np.empty(m, np.uint32)
        w = np.empty(m, np.uint32)
        rows, cols = L.gg_side_rows(h), L.gg_side_cols(h)
        xy = np.empty((n, 2), np.float32) if L.gg_has_xy(h) else None
        g2 = np.empty(rows * cols, np.int32) if rows * cols > 0 else None
        L.gg_copy(h, off.ctypes.data, nbr.ctypes.data, w.ctypes.data,
                  xy.ctypes.data if xy is not None else None,
                  g2.ctypes.data if g2 is not None else None)
    finally:
        L.gg_free(h)
    return Graph(name, off, nbr, w, xy, g2, rows, cols, meta)


def grid(rows: int, cols: int, wlo: int = 1, whi: int = 1000, seed: int = 1) -> Graph:
    """4-neighbour grid, both directions stored, weights uniform in [wlo, whi)."""
    return _take(_load().gg_grid(rows, cols, wlo, whi, seed), f"grid{rows}x{cols}",
                 dict(kind="grid", rows=rows, cols=cols, wlo=wlo, whi=whi, seed=seed))


def road(side: int, drop_p: float = 0.15, diag_p: float = 0.02, seed: int = 1) -> Graph:
    """Road-like grid with integral float32 coordinates (see module docstring)."""
    return _take(_load().gg_road(side, drop_p, diag_p, seed), f"road{side}",
                 dict(kind="road", side=side, drop_p=drop_p, diag_p=diag_p, seed=seed))


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, wlo: int = 1, whi: int = 1 << 16, seed: int = 1) -> Graph:
    """R-MAT graph, symmetrised and cleaned; weights uniform in [wlo, whi)."""
    return _take(_load().gg_rmat(scale, edgefactor, a, b, c, wlo, whi, seed),
                 f"rmat{scale}", dict(kind="rmat", scale=scale, edgefactor=edgefactor,
                                      a=a, b=b, c=c, wlo=wlo, whi=whi, seed=seed))


def with_weights(g: Graph, wlo: int, whi: int, seed: int) -> Graph:
    """Same topology, new weights uniform in [wlo, whi), drawn from the unordered
    endpoint pair (so both directions of a symmetric edge agree)."""
    L = _load()
    w = np.empty(g.m, np.uint32)
    L.gg_reweight(g.n, g.offsets.ctypes.data, g.nbr.ctypes.data, w.ctypes.data,
                  wlo, whi, seed)
    return Graph(g.name + f"_w{wlo}_{whi}", g.offsets, g.nbr, w, g.xy, g.grid2id,
                 g.rows, g.cols, dict(g.meta, wlo=wlo, whi=whi, wseed=seed))


def from_edges(n: int, src, dst, w, name: str = "edges", xy=None) -> Graph:
    """Directed CSR from edge arrays (kept as given: multi-edges and self loops stay).
    Adjacency order: by source, then by destination, then by weight."""
    src = np.asarray(src, np.uint64)
    dst = np.asarray(dst, np.uint32)
    w = np.asarray(w, np.uint32)
    order = np.lexsort((w, dst, src))
    src, dst, w = src[order], dst[order], w[order]
    off = np.zeros(n + 1, np.uint64)
    np.add.at(off, (src + 1).astype(np.int64), 1)
    off = np.cumsum(off).astype(np.uint64)
    return Graph(name, off, dst.copy(), w.copy(),
                 None if xy is None else np.asarray(xy, np.float32), None, 0, 0,
                 dict(kind="edges"))


def random_graph(n: int, m: int, wlo: int = 0, whi: int = 10, seed: int = 0,
                 symmetric: bool = False, self_loops: bool = True) -> Graph:
    """Small random (multi)graph for tests: m directed edge draws, endpoints uniform."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m)
    d = rng.integers(0, n, m)
    if not self_loops:
        keep = s != d
        s, d = s[keep], d[keep]
    w = rng.integers(wlo, whi, s.shape[0])
    if symmetric:
        s, d, w = np.concatenate([s, d]), np.concatenate([d, s]), np.concatenate([w, w])
    return from_edges(n, s, d, w, name=f"rand{n}_{m}_{seed}")


def path_graph(weights) -> Graph:
    """Directed path 0 -> 1 -> ... -> k with the given weights."""
    weights = np.asarray(weights, np.uint32)
    k = weights.shape[0]
    return from_edges(k + 1, np.arange(k), np.arange(1, k + 1), weights, name=f"path{k}")


def sample_sources(g: Graph, count: int, seed: int = 2) -> np.ndarray:
    """Uniform random vertices with at least one out-edge (without replacement when
    possible)."""
    rng = np.random.default_rng(seed)
    cand = np.nonzero(np.diff(g.offsets) > 0)[0]
    if cand.size == 0:
        raise ValueError("graph has no vertex with an out-edge")
    return cand[rng.choice(cand.size, size=count, replace=cand.size < count)].astype(np.uint32)


def priorities(n: int, seed: int = 3) -> np.ndarray:
    """A seeded uniformly random permutation of 0..n-1 (the set priorities of approximate
    set cover, drawn once and passed to both the oracle and the CUDA path)."""
    return np.random.default_rng(seed).permutation(n).astype(np.uint32)


def sample_pairs_grid_steps(g: Graph, count: int, kmin: int, kmax: int, seed: int = 2,
                            log_uniform: bool = False) -> np.ndarray:
    """(source, target) pairs on a grid-shaped graph: the target sits k grid steps (L1
    distance on the grid) from the source, k ~ U{kmin..kmax} or log-uniform; a draw that
    lands off the grid or outside the kept component is redrawn."""
    if g.grid2id is None:
        raise ValueError("graph has no grid layout")
    rng = np.random.default_rng(seed)
    rows, cols = g.rows, g.cols
    pos = np.full(g.n, -1, np.int64)
    ids = np.nonzero(g.grid2id >= 0)[0]
    pos[g.grid2id[ids]] = ids
    out = np.empty((count, 2), np.uint32)
    i = 0
    while i < count:
        s = int(rng.integers(0, g.n))
        if log_uniform:
            k = int(round(np.exp(rng.uniform(np.log(kmin), np.log(kmax)))))
        else:
            k = int(rng.integers(kmin, kmax + 1))
        dx = int(rng.integers(-k, k + 1))
        dy = (k - abs(dx)) * (1 if rng.integers(0, 2) else -1)
        r, c = divmod(int(pos[s]), cols)
        r2, c2 = r + dy, c + dx
        if not (0 <= r2 < rows and 0 <= c2 < cols):
            continue
        t = int(g.grid2id[r2 * cols + c2])
        if t < 0 or t == s:
            continue
        out[i] = (s, t)
        i += 1
    return out
