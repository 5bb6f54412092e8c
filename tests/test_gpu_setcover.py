"""GPU parity for approximate set cover: the CUDA path (through the C ABI) against the CPU
oracle, bit-exact.

The method is deterministic given the graph, eps and the priorities (every step's claims
resolve to the smallest priority, and a step's decisions read only the state at its
start), so the step in which each set joins the cover must match the oracle exactly,
for every launch shape (CTAs per SM, large-set threshold).
"""
import itertools

import numpy as np
import pytest

from tests.golden import fixtures

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def og():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1911_07260_gb300 as og
    from paper_1911_07260_gb300 import build
    build.build()
    torch.cuda.init()
    return og


def _graph(gg, n, pairs):
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    return gg.from_edges(n, pairs[:, 0], pairs[:, 1], np.ones(len(pairs), np.uint32))


def _sym(gg, n, pairs):
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    return _graph(gg, n, np.concatenate([pairs, pairs[:, ::-1]]))


def _cliques(sizes):
    pairs, base = [], 0
    for k in sizes:
        pairs += [(base + a, base + b) for a, b in itertools.combinations(range(k), 2)]
        base += k + 2
    return base, pairs


def _graphs(gg):
    rng = np.random.default_rng(5)
    out = [("grid64", gg.grid(64, 64, 1, 2, seed=1)),
           ("road300", gg.road(300, 0.15, 0.02, seed=1)),
           ("rmat13", gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 2, seed=6)),
           ("star", _sym(gg, 3001, [(0, i) for i in range(1, 3001)]))]
    n, p = _cliques([3, 7, 40, 90])
    out.append(("cliques", _sym(gg, n, p)))
    # a directed multigraph: repeated entries, self loops, vertices only some sets hold
    m = 20000
    a = rng.integers(0, 3000, m)
    b = np.where(rng.random(m) < 0.3, rng.integers(0, 50, m), rng.integers(0, 3000, m))
    out.append(("multi", _graph(gg, 3000, np.stack([a, b], 1))))
    return out


@pytest.mark.parametrize("eps", [0, 10000, 250000, 1000000])
def test_setcover_matches_oracle(og, orc, gg, eps):
    """Grid, road-like grid, R-MAT (sets above and below the large-set threshold), a star
    of 3000 leaves, cliques, a directed multigraph: every set's join step and the number
    of steps equal the oracle's, with random priorities."""
    for name, g in _graphs(gg):
        pri = gg.priorities(g.n, seed=len(name))
        ref, steps = orc.setcover(g, pri, eps)
        got, st = og.setcover(og.Graph.from_csr(g), eps, pri)
        np.testing.assert_array_equal(got, ref, err_msg=name)
        assert st.rounds == steps, name
        assert st.improved == int((ref > 0).sum()), name


def test_setcover_hand_worked_fixtures(og, gg):
    for f in fixtures.load_setcover():
        g = _graph(gg, f["n"], f["edges"])
        got, st = og.setcover(og.Graph.from_csr(g), f["eps_ppm"], np.array(f["pri"]))
        assert got.tolist() == f["expect"], f["name"]
        assert st.rounds == f["steps"], f["name"]


@pytest.mark.parametrize("hub", [16, 32, 100, 1 << 26])
@pytest.mark.parametrize("bps", [1, 2, 4])
def test_setcover_launch_shapes_identical(og, orc, gg, hub, bps):
    """Every large-set threshold (16: most R-MAT sets split over the grid; 2^26: every
    set handled 32 to a warp) and CTAs per SM give the oracle's cover."""
    g = gg.rmat(14, 16, 0.57, 0.19, 0.19, 1, 2, seed=7)
    pri = gg.priorities(g.n, seed=11)
    ref, steps = orc.setcover(g, pri, 10000)
    got, st = og.setcover(og.Graph.from_csr(g), 10000, pri,
                          cfg=og.config(hub_degree=hub, blocks_per_sm=bps))
    np.testing.assert_array_equal(got, ref)
    assert st.rounds == steps


def test_setcover_identity_priorities_and_device_buffers(og, orc, gg):
    """NULL priorities are the identity; device priorities and a device output give the
    host result."""
    import torch
    g = gg.rmat(12, 8, 0.57, 0.19, 0.19, 1, 2, seed=3)
    G = og.Graph.from_csr(g)
    ref, _ = orc.setcover(g, np.arange(g.n), 10000)
    got, _ = og.setcover(G, 10000, None)
    np.testing.assert_array_equal(got, ref)
    pri = gg.priorities(g.n, seed=4)
    ref2, _ = orc.setcover(g, pri, 10000)
    dpri = torch.from_numpy(pri.view(np.int32)).cuda()
    dout = torch.empty(g.n, dtype=torch.int32, device="cuda")
    og.setcover(G, 10000, dpri, out=dout)
    np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref2)


def test_setcover_many_bands_and_empty_graphs(og, orc, gg):
    """eps = 0 makes one bucket per residual size: a star of 5000 leaves beside cliques
    and paths spans hundreds of bands, most of them empty.  A graph without edges covers
    nothing in no steps."""
    n, p = _cliques([5, 33, 200])
    p = p + [(n + 1, n + 1 + i) for i in range(1, 5001)]
    p = p + [(n + 6000 + i, n + 6001 + i) for i in range(50)]
    g = _sym(gg, n + 6100, p)
    pri = gg.priorities(g.n, seed=9)
    for eps in (0, 1000):
        ref, steps = orc.setcover(g, pri, eps)
        got, st = og.setcover(og.Graph.from_csr(g), eps, pri)
        np.testing.assert_array_equal(got, ref)
        assert st.rounds == steps
    e = gg.from_edges(7, [], [], [])
    got, st = og.setcover(og.Graph.from_csr(e), 10000, np.arange(7))
    assert got.tolist() == [0] * 7 and st.rounds == 0


def test_setcover_rejects_bad_arguments(og, gg):
    g = _sym(gg, 5, [(0, 1), (1, 2), (3, 4)])
    G = og.Graph.from_csr(g)
    for pri in (np.array([0, 1, 2, 2, 4]), np.array([0, 1, 2, 3, 5])):
        with pytest.raises(og.OgError) as e:
            og.setcover(G, 10000, pri)
        assert e.value.code == og.E_INVALID
    with pytest.raises(og.OgError) as e:
        og.setcover(G, 1000001, np.arange(5))
    assert e.value.code == og.E_INVALID
    # the graph stays usable after a rejected call
    got, _ = og.setcover(G, 10000, np.arange(5))
    assert set(np.nonzero(got)[0].tolist()) >= {1}
