"""GPU parity in the hot-first vertex order: every entry point keeps the caller's ids.

The library may store a graph with its highest-degree vertices moved to the low device
ids (a layout choice for the L2, decided at upload for large power-law graphs and
settable per graph).  Whatever the order, sources, targets, coordinates and priorities
go in with the caller's ids and distances, coreness and join steps come back in the
caller's order, so every result below is compared with the oracle on the graph as
given, bit-exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


@pytest.fixture(scope="module")
def og():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1911_07260_gb300 as og
    from paper_1911_07260_gb300 import build
    build.build()
    torch.cuda.init()
    return og


def _graphs(gg):
    return [("rmat12", gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=5)),
            ("rmat13_w2", gg.rmat(13, 8, 0.57, 0.19, 0.19, 1, 2, seed=9)),
            ("road150", gg.road(150, seed=5)),
            ("multi", gg.random_graph(3000, 40000, 0, 50, seed=4))]


def _hot(og, g):
    G = og.Graph.from_csr(g)
    G.set_order(og.ORDER_HOT_FIRST)
    order, moved = G.order()
    assert order == og.ORDER_HOT_FIRST and moved > 0
    return G


def test_order_query_kinds_match_oracle(og, orc, gg):
    """SSSP, wBFS, Bellman-Ford, PPSP through both engines, single and batched, host and
    device outputs: the caller's ids in, the caller's order out."""
    import torch
    for name, g in _graphs(gg):
        G = _hot(og, g)
        rng = np.random.default_rng(len(name))
        srcs = [int(x) for x in rng.integers(0, g.n, 4)]
        for s in srcs:
            ref = orc.dijkstra(g, s)
            np.testing.assert_array_equal(og.sssp_delta(G, s, 64), ref, err_msg=name)
            np.testing.assert_array_equal(og.bellman_ford(G, s)[0], ref, err_msg=name)
            d = torch.empty(g.n, dtype=torch.int32, device="cuda")
            og.sssp_delta(G, s, 7, out=d)
            np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), ref, err_msg=name)
            t = int(rng.integers(0, g.n))
            assert og.ppsp(G, s, t, 64) == orc.ppsp(g, s, t), name
        if g.w.min() > 0:
            np.testing.assert_array_equal(og.wbfs(G, srcs[0]),
                                          orc.dijkstra(g, srcs[0]), err_msg=name)
        qs = [(og.Q_SSSP, s, 0, 0) for s in srcs] + [(og.Q_PPSP, srcs[0], srcs[1], 0)]
        for engine in (1, 2):
            out, dres, _ = og.batch_run(G, qs, cfg=og.config(engine=engine))
            out = out.reshape(len(qs), g.n)
            for i, s in enumerate(srcs):
                np.testing.assert_array_equal(out[i], orc.dijkstra(g, s), err_msg=name)
            assert dres[-1] == orc.ppsp(g, srcs[0], srcs[1]), name


def test_order_batch_of_many_rows(og, orc, gg):
    """A batch of 40 queries (its rows go back to the caller's order 16 at a time), host
    and device outputs, every row against the oracle."""
    import torch
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=5)
    G = _hot(og, g)
    rng = np.random.default_rng(40)
    srcs = [int(x) for x in rng.integers(0, g.n, 40)]
    qs = [(og.Q_SSSP, s, 0, 64) for s in srcs]
    ref = np.stack([orc.dijkstra(g, s) for s in srcs])
    out, _, _ = og.batch_run(G, qs)
    np.testing.assert_array_equal(out.reshape(len(qs), g.n), ref)
    d = torch.empty(len(qs) * g.n, dtype=torch.int32, device="cuda")
    og.batch_run(G, qs, out=d)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32).reshape(len(qs), g.n), ref)


def test_order_astar_coordinates_stay_in_caller_order(og, orc, gg):
    """A* reads coordinates per vertex: set before or after the reorder, they stay
    attached to the caller's vertices."""
    g = gg.road(120, seed=3)
    pairs = gg.sample_pairs_grid_steps(g, 12, 5, 200, seed=8, log_uniform=True)
    G1 = og.Graph.from_csr(g)          # coordinates uploaded in the user's order
    G1.set_order(og.ORDER_HOT_FIRST)   # ... and moved with the vertices
    G2 = og.Graph.from_csr(g, coords=False)
    G2.set_order(og.ORDER_HOT_FIRST)
    G2.set_coords(g.xy)                # coordinates uploaded after the reorder
    for s, t in pairs.tolist():
        ref = orc.ppsp(g, s, t)
        assert og.astar(G1, s, t, 300) == ref
        assert og.astar(G2, s, t, 300) == ref


@pytest.mark.parametrize("mode", [0, 1])
def test_order_kcore_matches_oracle(og, orc, gg, mode):
    import torch
    for name, g in _graphs(gg)[:2]:
        G = _hot(og, g)
        ref = orc.kcore(g)
        got, _ = og.kcore(G, mode)
        np.testing.assert_array_equal(got, ref, err_msg=name)
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        og.kcore(G, mode, out=d)
        np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), ref, err_msg=name)


def test_order_setcover_priorities_and_identity(og, orc, gg):
    """Set cover: host, device and identity priorities are the caller's; join steps come
    back per set in the caller's order; a repeated priority is still rejected."""
    import torch
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 2, seed=7)
    G = _hot(og, g)
    pri = gg.priorities(g.n, seed=3)
    ref, steps = orc.setcover(g, pri, 10000)
    got, st = og.setcover(G, 10000, pri)
    np.testing.assert_array_equal(got, ref)
    assert st.rounds == steps
    dpri = torch.from_numpy(pri.view(np.int32)).cuda()
    before = dpri.clone()
    dout = torch.empty(g.n, dtype=torch.int32, device="cuda")
    og.setcover(G, 10000, dpri, out=dout)
    np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref)
    assert torch.equal(dpri, before), "the caller's priorities were written"
    ref_id, _ = orc.setcover(g, np.arange(g.n), 10000)
    got_id, _ = og.setcover(G, 10000, None)
    np.testing.assert_array_equal(got_id, ref_id)
    bad = pri.copy()
    bad[1] = bad[0]
    with pytest.raises(og.OgError) as e:
        og.setcover(G, 10000, bad)
    assert e.value.code == og.E_INVALID


def test_order_server_and_busy(og, orc, gg):
    """Served queries take the caller's ids; the order cannot change under a server."""
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=5)
    G = _hot(og, g)
    srv = og.Server(G, max_slots=8, cfg=og.config(delta=64))
    rng = np.random.default_rng(2)
    pairs = rng.integers(0, g.n, (20, 2)).tolist()
    got, pending = {}, list(enumerate(pairs))
    while pending or len(got) < len(pairs):
        while pending and srv.submit(og.Q_PPSP, pending[0][1][0], pending[0][1][1],
                                     tag=pending[0][0]):
            pending.pop(0)
        srv.step(budget_us=100)
        tags, d = srv.poll()
        got.update(zip(tags.tolist(), d.tolist()))
    for i, (s, t) in enumerate(pairs):
        assert got[i] == orc.ppsp(g, s, t), i
    with pytest.raises(og.OgError) as e:
        G.set_order(og.ORDER_USER)
    assert e.value.code == og.E_BUSY
    srv.free()
    G.set_order(og.ORDER_USER)
    assert G.order() == (og.ORDER_USER, 0)


def test_order_round_trip_and_auto(og, orc, gg):
    """Hot-first and back gives the caller's order again; automatic order keeps a small
    graph as given and packs a large power-law one."""
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=5)
    G = og.Graph.from_csr(g)
    assert G.order() == (og.ORDER_USER, 0)         # below the automatic size
    G.set_order(og.ORDER_HOT_FIRST)
    G.set_order(og.ORDER_HOT_FIRST)                # idempotent
    _, moved = G.order()
    G.set_order(og.ORDER_USER)
    assert G.order() == (og.ORDER_USER, 0)
    np.testing.assert_array_equal(og.sssp_delta(G, 3, 64), orc.dijkstra(g, 3))
    G.set_order(og.ORDER_AUTO)                     # still below the automatic size
    assert G.order() == (og.ORDER_USER, 0)
    with pytest.raises(og.OgError):
        G.set_order(7)
    big = gg.rmat(20, 16, 0.57, 0.19, 0.19, 1, 2, seed=1)
    B = og.Graph.from_csr(big)
    order, moved = B.order()
    assert order == og.ORDER_HOT_FIRST and 0 < moved <= 2 * (big.n // 8)
    src = int(gg.sample_sources(big, 1, seed=3)[0])
    assert orc.check_sssp(big, src, og.sssp_delta(B, src, 64)) == (0, 0)
    road = gg.road(1200, seed=2)                   # > 2^20 vertices, no skew
    R = og.Graph.from_csr(road)
    assert R.order() == (og.ORDER_USER, 0)
