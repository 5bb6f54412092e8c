"""The hot-first vertex order's permutation, computed by the library on the host
(`og_hot_first_order`, no device call), against its definition written out here: the
n/8 vertices of largest out-degree (ties: the smaller id) take device ids 0 .. n/8 - 1 in
that order, the other vertices below n/8 take the ids the hot ones left (both in
increasing order), every other vertex keeps its id."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def og():
    import paper_1911_07260_gb300 as og
    from paper_1911_07260_gb300 import build
    build.build()
    return og


def _expected(deg):
    n = len(deg)
    k = n // 8
    order = sorted(range(n), key=lambda v: (-int(deg[v]), v))
    hot = order[:k]
    hotset = set(hot)
    pi = list(range(n))
    for i, v in enumerate(hot):
        pi[i] = v
    freed = sorted(h for h in hot if h >= k)
    displaced = sorted(v for v in range(k) if v not in hotset)
    assert len(freed) == len(displaced)
    for h, c in zip(freed, displaced):
        pi[h] = c
    return np.array(pi, np.uint32), int(sum(int(deg[v]) for v in hot))


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (8, 2), (9, 3), (64, 4), (1000, 5),
                                    (4099, 6)])
def test_matches_the_definition(og, n, seed):
    rng = np.random.default_rng(seed)
    # many ties (small degrees) and a heavy tail
    deg = np.minimum(rng.zipf(1.6, n), 5000).astype(np.uint32)
    deg[rng.random(n) < 0.2] = 0
    got, hot_edges = og.hot_first_order(deg)
    ref, ref_edges = _expected(deg)
    np.testing.assert_array_equal(got, ref)
    assert hot_edges == ref_edges
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))  # a permutation


def test_already_hot_first_moves_nothing(og):
    deg = np.array(list(range(800, 0, -1)), np.uint32)  # descending: ids are the order
    got, hot_edges = og.hot_first_order(deg)
    np.testing.assert_array_equal(got, np.arange(800, dtype=np.uint32))
    assert hot_edges == int(deg[:100].sum())


def test_the_upload_rule_tells_power_law_from_road(og, gg):
    """The upload packs a graph whose hottest eighth holds half of the edges or more:
    R-MAT does, the road-like grid does not."""
    for g, skewed in ((gg.rmat(14, 16, 0.57, 0.19, 0.19, 1, 2, seed=1), True),
                      (gg.road(150, seed=1), False)):
        deg = np.diff(g.offsets).astype(np.uint32)
        _, hot_edges = og.hot_first_order(deg)
        assert (2 * hot_edges >= g.m) == skewed


def test_rejects_empty_input(og):
    with pytest.raises(og.OgError) as e:
        og.hot_first_order(np.zeros(0, np.uint32))
    assert e.value.code == og.E_INVALID
