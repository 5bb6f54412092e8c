"""Properties of the seeded synthetic inputs (CPU only)."""
import math

import numpy as np
import pytest


def _src_of(g):
    return np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets).astype(np.int64))


def _symmetric_weights(g):
    s = _src_of(g)
    d = g.nbr.astype(np.int64)
    fwd = dict(zip(zip(s.tolist(), d.tolist()), g.w.tolist()))
    return all(fwd.get((v, u)) == w for (u, v), w in fwd.items())


def test_grid_shape_and_weights(gg):
    g = gg.grid(256, 256, 1, 1000, seed=1)
    assert g.n == 65536 and g.m == 261120
    assert g.w.min() >= 1 and g.w.max() <= 999
    assert np.all(np.diff(g.offsets.astype(np.int64)) >= 2)
    small = gg.grid(9, 7, 1, 1000, seed=1)
    assert _symmetric_weights(small)


def test_generators_are_deterministic(gg):
    a, b = gg.road(64, seed=1), gg.road(64, seed=1)
    c = gg.road(64, seed=2)
    for x, y in [(a.offsets, b.offsets), (a.nbr, b.nbr), (a.w, b.w), (a.xy, b.xy)]:
        np.testing.assert_array_equal(x, y)
    assert not (a.m == c.m and np.array_equal(a.w[:100], c.w[:100]))
    r1, r2 = gg.rmat(10, seed=4), gg.rmat(10, seed=4)
    np.testing.assert_array_equal(r1.nbr, r2.nbr)
    np.testing.assert_array_equal(r1.w, r2.w)


def test_road_properties(gg, orc):
    g = gg.road(120, 0.15, 0.02, seed=1)
    assert _symmetric_weights(g)
    # largest component only: everything reachable from vertex 0
    assert (orc.bfs(g, 0) != 0xFFFFFFFF).all()
    s = _src_of(g)
    dx = np.abs(g.xy[s, 0] - g.xy[g.nbr, 0])
    dy = np.abs(g.xy[s, 1] - g.xy[g.nbr, 1])
    grid_edge = (dx + dy) == 1
    diag = (dx == 1) & (dy == 1)
    assert np.all(grid_edge | diag)
    assert g.w[grid_edge].min() >= 100 and g.w[grid_edge].max() <= 150
    assert g.w[diag].min() >= 142 and g.w[diag].max() <= 212
    # about 85% of grid edges and 2% of cells survive
    assert 0.80 < grid_edge.sum() / 2 / (2 * 120 * 119) < 0.90
    assert 0.01 < diag.sum() / 2 / (119 * 119) < 0.03
    # relabelling is row-major
    key = g.xy[:, 1].astype(np.int64) * 120 + g.xy[:, 0].astype(np.int64)
    assert np.all(np.diff(key) > 0)


def _h(xy, t):
    """floor(100 * Euclidean distance) for integral coordinates, exactly."""
    d2 = ((xy[:, 0] - xy[t, 0]).astype(np.int64) ** 2 +
          (xy[:, 1] - xy[t, 1]).astype(np.int64) ** 2)
    return np.array([math.isqrt(10000 * int(x)) for x in d2], np.int64)


def test_road_heuristic_is_consistent(gg):
    """With w >= ceil(100 * length) every edge satisfies h(u) <= w(u, v) + h(v), so the
    A* heuristic floor(100 * Euclid) is consistent (hence admissible)."""
    g = gg.road(80, seed=7)
    s = _src_of(g)
    for t in [0, g.n // 2, g.n - 1]:
        h = _h(g.xy, t)
        assert np.all(h[s] <= g.w.astype(np.int64) + h[g.nbr])
        assert h[t] == 0


def test_rmat_cleaned_and_symmetric(gg):
    g = gg.rmat(11, 16, 0.57, 0.19, 0.19, 1, 24, seed=1)
    s = _src_of(g)
    assert not np.any(s == g.nbr)                       # no self loops
    key = s * g.n + g.nbr
    assert np.unique(key).size == key.size              # no duplicates
    assert _symmetric_weights(g)
    assert g.w.min() >= 1 and g.w.max() <= 23
    deg = g.degrees()
    assert deg.max() > 20 * max(1.0, deg[deg > 0].mean())   # skewed degrees
    g2 = gg.with_weights(g, 1, 1 << 16, seed=3)
    assert _symmetric_weights(g2) and g2.w.max() > 1000


def test_grid_step_pairs(gg):
    g = gg.road(200, seed=1)
    pairs = gg.sample_pairs_grid_steps(g, 50, 10, 100, seed=2)
    l1 = (np.abs(g.xy[pairs[:, 0]] - g.xy[pairs[:, 1]])).sum(axis=1)
    assert l1.min() >= 10 and l1.max() <= 100
    src = gg.sample_sources(g, 8, seed=2)
    assert src.dtype == np.uint32 and len(set(src.tolist())) == 8


def test_priorities_are_seeded_permutations(gg):
    for n in (1, 7, 1000):
        p = gg.priorities(n, seed=5)
        assert p.dtype == np.uint32 and sorted(p.tolist()) == list(range(n))
        np.testing.assert_array_equal(p, gg.priorities(n, seed=5))
    assert not np.array_equal(gg.priorities(1000, seed=5), gg.priorities(1000, seed=6))


def test_rmat_structure_does_not_depend_on_the_weight_range(gg):
    """The full-size k-core and set cover tests take the R-MAT SSSP graph for the bench's
    k-core / set cover graph (same generator and seed, weights in [1, 2)): the two share
    offsets and neighbours, only the weights differ."""
    a = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
    b = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 1 << 16, seed=1)
    c = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 24, seed=1)
    for x in (b, c):
        np.testing.assert_array_equal(a.offsets, x.offsets)
        np.testing.assert_array_equal(a.nbr, x.nbr)
    assert int(a.w.max()) == 1 and int(b.w.max()) > 24 and int(c.w.max()) < 24
