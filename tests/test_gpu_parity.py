"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Distances are integers, so every comparison is exact equality.  Where several schedules
are legal (Delta, fusion threshold, tile, ring size, CTAs per SM) they must all give the
same distances (Section 3.3: fusion never reorders priorities; Section 2: coarsening only
changes the schedule).
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


@pytest.fixture(scope="module")
def grid256(gg, og):
    g = gg.grid(256, 256, 1, 1000, seed=1)
    return g, og.Graph.from_csr(g)


def _dev(n):
    import torch
    return torch.empty(n, dtype=torch.int32, device="cuda")


def _np(t):
    return t.cpu().numpy().view(np.uint32)


def test_grid256_delta1000_bit_exact(og, orc, grid256):
    g, G = grid256
    ref = orc.dijkstra(g, 0)
    got = og.sssp_delta(G, 0, 1000)
    np.testing.assert_array_equal(got, ref)
    # device output buffer gives the same answer
    d = _dev(g.n)
    og.sssp_delta(G, 0, 1000, out=d)
    np.testing.assert_array_equal(_np(d), ref)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("delta", [1, 2, 7, 1000, 1 << 20, 1 << 31])
@pytest.mark.parametrize("fusion", [0xFFFFFFFE, 1, 64, 0xFFFFFFFF])
def test_schedule_sweep_identical(og, orc, grid256, delta, fusion, engine):
    g, G = grid256
    src = 31337
    ref = orc.dijkstra(g, src)
    cfg = og.config(delta=delta, fusion_threshold=fusion, engine=engine)
    got, _, st = og.query_run(G, og.Q_SSSP, src, cfg=cfg)
    np.testing.assert_array_equal(got, ref)
    assert st.rounds >= 1 and st.relax >= g.m // 2


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("tile,ring,bps", [(32, 2, 1), (256, 4, 2), (2048, 64, 0), (96, 2, 3)])
def test_tile_ring_occupancy_sweep(og, orc, grid256, tile, ring, bps, engine):
    g, G = grid256
    ref = orc.dijkstra(g, 65535)
    cfg = og.config(delta=37, expand_tile=tile, ring_buckets=ring, blocks_per_sm=bps,
                    engine=engine)
    got, _, st = og.query_run(G, og.Q_SSSP, 65535, cfg=cfg)
    np.testing.assert_array_equal(got, ref)
    if ring == 2:
        assert st.overflow_inserts > 0 and st.redistributions > 0


@pytest.mark.parametrize("seed", range(40))
def test_random_small_graphs(og, orc, gg, seed):
    """Ragged shapes: zero weights, self loops, parallel edges, unreachable parts,
    isolated vertices, a hub of high degree."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 8 * n))
    g = gg.random_graph(n, m, wlo=0, whi=int(rng.choice([2, 30, 1000, 100000])), seed=seed,
                        symmetric=bool(seed % 3 == 0))
    if seed % 5 == 0 and n > 10:  # add a hub with many out-edges
        s = np.concatenate([np.repeat(np.arange(n), np.diff(g.offsets).astype(np.int64)),
                            np.zeros(5 * n, np.int64)])
        d = np.concatenate([g.nbr, rng.integers(0, n, 5 * n)])
        w = np.concatenate([g.w, rng.integers(0, 50, 5 * n)])
        g = gg.from_edges(n, s, d, w)
    G = og.Graph.from_csr(g)
    for src in {0, int(rng.integers(0, n)), n - 1}:
        ref = orc.dijkstra(g, src)
        delta = int(rng.choice([1, 3, 64, 5000]))
        fusion = int(rng.choice([0xFFFFFFFE, 2, 128, 0xFFFFFFFF]))
        for engine in (1, 2):
            got, _, _ = og.query_run(G, og.Q_SSSP, src, cfg=og.config(
                delta=delta, fusion_threshold=fusion, engine=engine))
            np.testing.assert_array_equal(got, ref)


def test_single_vertex_and_edgeless(og, orc, gg):
    g = gg.from_edges(1, [], [], [])
    G = og.Graph.from_csr(g)
    assert og.sssp_delta(G, 0, 5).tolist() == [0]
    g = gg.from_edges(7, [3], [3], [4])  # only a self loop
    G = og.Graph.from_csr(g)
    assert og.sssp_delta(G, 3, 1).tolist() == [INF] * 3 + [0] + [INF] * 3


def test_wbfs_unit_weights_is_bfs(og, orc, gg):
    g = gg.random_graph(5000, 20000, wlo=1, whi=2, seed=11, symmetric=True)
    G = og.Graph.from_csr(g)
    for src in (0, 4999):
        np.testing.assert_array_equal(og.wbfs(G, src), orc.bfs(g, src))


def test_wbfs_rmat_small_weights(og, orc, gg):
    g = gg.rmat(14, 16, 0.57, 0.19, 0.19, 1, 24, seed=1)
    G = og.Graph.from_csr(g)
    for src in gg.sample_sources(g, 3, seed=2):
        np.testing.assert_array_equal(og.wbfs(G, int(src)), orc.dijkstra(g, int(src)))


def test_wbfs_rejects_zero_weight(og, gg):
    g = gg.path_graph([1, 0, 2])
    G = og.Graph.from_csr(g)
    with pytest.raises(og.OgError) as e:
        og.wbfs(G, 0)
    assert e.value.code == og.E_INVALID


def test_sssp_rmat_weights_up_to_2e16(og, orc, gg):
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 1 << 16, seed=3)
    G = og.Graph.from_csr(g)
    for src in gg.sample_sources(g, 2, seed=2):
        ref = orc.dijkstra(g, int(src))
        for delta in (256, 4096, 65536):
            np.testing.assert_array_equal(og.sssp_delta(G, int(src), delta), ref)


@pytest.fixture(scope="module")
def road300(gg, og):
    g = gg.road(300, seed=1)
    return g, og.Graph.from_csr(g)


def test_ppsp_and_astar_match_oracle(og, orc, gg, road300):
    g, G = road300
    pairs = gg.sample_pairs_grid_steps(g, 25, 1, 400, seed=5)
    for s, t in pairs.tolist():
        ref = orc.ppsp(g, s, t)
        for delta in (64, 1024, 16384):
            assert og.ppsp(G, s, t, delta) == ref
            assert og.astar(G, s, t, delta) == ref


def test_ppsp_edge_cases(og, orc, gg, road300):
    g, G = road300
    assert og.ppsp(G, 5, 5, 100) == 0
    assert og.astar(G, 5, 5, 100) == 0
    # unreachable target
    h = gg.from_edges(4, [0, 2], [1, 3], [5, 5])
    H = og.Graph.from_csr(h)
    assert og.ppsp(H, 0, 3, 4) == INF
    with pytest.raises(og.OgError):
        og.ppsp(H, 0, 99, 4)
    with pytest.raises(og.OgError):  # A* needs coordinates
        og.astar(H, 0, 1, 4)


def test_astar_with_fractional_coordinates(og, orc, gg):
    """Non-integral coordinates take the double-precision heuristic, reduced by one unit;
    with Euclidean-consistent weights the result stays exact."""
    rng = np.random.default_rng(3)
    n = 400
    xy = rng.uniform(0, 50, (n, 2)).astype(np.float32)
    s, d = rng.integers(0, n, 3000), rng.integers(0, n, 3000)
    keep = s != d
    s, d = s[keep], d[keep]
    length = np.sqrt(((xy[s].astype(np.float64) - xy[d]) ** 2).sum(1))
    w = np.ceil(100 * length).astype(np.uint32) + rng.integers(0, 30, s.size).astype(np.uint32)
    g = gg.from_edges(n, np.concatenate([s, d]), np.concatenate([d, s]),
                      np.concatenate([w, w]), xy=xy)
    G = og.Graph.from_csr(g)
    for src, dst in rng.integers(0, n, (20, 2)).tolist():
        assert og.astar(G, src, dst, 200) == orc.ppsp(g, src, dst)


def test_batch_equals_alone(og, orc, gg, road300):
    g, G = road300
    srcs = gg.sample_sources(g, 6, seed=9)
    pairs = gg.sample_pairs_grid_steps(g, 10, 10, 300, seed=9)
    queries = [(og.Q_SSSP, int(s), 0, 2048) for s in srcs]
    queries += [(og.Q_PPSP, int(a), int(b), 1024) for a, b in pairs[:5]]
    queries += [(og.Q_ASTAR, int(a), int(b), 512) for a, b in pairs[5:]]
    queries += [(og.Q_WBFS, int(srcs[0]), 0, 0)]
    out, d, st = og.batch_run(G, queries)
    out = out.reshape(len(queries), g.n)
    for i, (kind, s, t, delta) in enumerate(queries):
        if kind == og.Q_SSSP:
            np.testing.assert_array_equal(out[i], orc.dijkstra(g, s))
            np.testing.assert_array_equal(out[i], og.sssp_delta(G, s, delta))
        elif kind == og.Q_WBFS:
            np.testing.assert_array_equal(out[i], orc.dijkstra(g, s))
        else:
            assert d[i] == orc.ppsp(g, s, t)
    assert st.rounds > 0


def test_batch_device_output(og, orc, gg, road300):
    import torch
    g, G = road300
    srcs = [0, 100, 2000]
    buf = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    og.batch_run(G, [(og.Q_SSSP, s, 0, 0) for s in srcs], out=buf)
    got = _np(buf).reshape(len(srcs), g.n)
    for i, s in enumerate(srcs):
        np.testing.assert_array_equal(got[i], orc.dijkstra(g, s))


@pytest.mark.parametrize("engine", [1, 2])
def test_arena_regrowth_keeps_results_exact(og, orc, grid256, engine):
    g, G = grid256
    ref = orc.dijkstra(g, 123)
    cfg = og.config(delta=50, ring_buckets=2, arena_entries=300, engine=engine)
    got, _, st = og.query_run(G, og.Q_SSSP, 123, cfg=cfg)
    np.testing.assert_array_equal(got, ref)
    assert st.restarts >= 1


@pytest.mark.parametrize("engine", [1, 2])
def test_barrier_timeout_is_reported_and_context_survives(og, orc, grid256, engine):
    """A wait limit of 1 ns makes the bounded device waits give up (the grid barrier of
    the round engine, the idle wait of the barrier-free engine): the call returns
    OG_E_TIMEOUT instead of hanging, and the next call still works."""
    g, G = grid256
    with pytest.raises(og.OgError) as e:
        og.query_run(G, og.Q_SSSP, 0, cfg=og.config(delta=1000, spin_limit_ns=1,
                                                    engine=engine))
    assert e.value.code == og.E_TIMEOUT
    np.testing.assert_array_equal(og.sssp_delta(G, 0, 1000), orc.dijkstra(g, 0))


def test_distance_saturation_reported(og, gg):
    g = gg.path_graph([0xFFFFFFF0, 0x10, 0x10])
    G = og.Graph.from_csr(g)
    with pytest.raises(og.OgError) as e:
        og.sssp_delta(G, 0, 1 << 20)
    assert e.value.code == og.E_OVERFLOW


def test_invalid_arguments(og, gg, grid256):
    g, G = grid256
    with pytest.raises(og.OgError) as e:
        og.sssp_delta(G, g.n, 10)
    assert e.value.code == og.E_INVALID
    with pytest.raises(og.OgError):
        og.Graph(np.array([0, 2], np.uint64), np.array([0, 5], np.uint32),
                 np.array([1, 1], np.uint32))  # neighbor out of range
    with pytest.raises(og.OgError):
        og.Graph(np.array([0, 2, 1], np.uint64), np.array([0, 1], np.uint32),
                 np.array([1, 1], np.uint32))  # offsets not monotone


def test_fusion_cuts_rounds_on_road_graph(og, orc, road300):
    """Section 6.4 (the table of running times and rounds with and without bucket
    fusion): fusion processes the same bucket without a global round;
    the result is unchanged and the number of global rounds drops."""
    g, G = road300
    ref = orc.dijkstra(g, 0)
    rounds = dict(delta=2048, engine=og.ENGINE_ROUNDS)
    _, _, off = og.query_run(G, og.Q_SSSP, 0, cfg=og.config(fusion_threshold=0xFFFFFFFE, **rounds))
    got, _, on = og.query_run(G, og.Q_SSSP, 0, cfg=og.config(fusion_threshold=2048, **rounds))
    np.testing.assert_array_equal(got, ref)
    assert on.rounds * 3 < off.rounds, (on.rounds, off.rounds)
    assert on.fused_iters > 0 and off.fused_iters == 0


def test_async_engine_fusion_keeps_work_local(og, orc, road300):
    """Barrier-free engine: with fusion most inserts of the current bucket stay in the
    warp's local bucket; without it every insert goes through a global bucket."""
    g, G = road300
    ref = orc.dijkstra(g, 7)
    asy = dict(delta=2048, engine=og.ENGINE_ASYNC)
    got_off, _, off = og.query_run(G, og.Q_SSSP, 7, cfg=og.config(fusion_threshold=0xFFFFFFFE,
                                                                 **asy))
    got_on, _, on = og.query_run(G, og.Q_SSSP, 7, cfg=og.config(fusion_threshold=256, **asy))
    np.testing.assert_array_equal(got_off, ref)
    np.testing.assert_array_equal(got_on, ref)
    assert off.local_inserts == 0 and off.global_inserts >= g.n - 1
    assert on.local_inserts > 4 * on.global_inserts
    assert on.rounds == off.rounds  # one transition per non-empty bucket either way


def test_ppsp_dirty_ring_reuse(og, orc, gg, road300):
    """Early-exit queries leave entries behind; later calls on the same graph (same and
    different ring layouts) must still be exact."""
    g, G = road300
    pairs = gg.sample_pairs_grid_steps(g, 12, 5, 60, seed=21)
    for s, t in pairs.tolist():
        assert og.ppsp(G, s, t, 256) == orc.ppsp(g, s, t)
        np.testing.assert_array_equal(og.sssp_delta(G, s, 256), orc.dijkstra(g, s))
        np.testing.assert_array_equal(og.sssp_delta(G, t, 16), orc.dijkstra(g, t))


def test_server_mix_equals_alone(og, orc, gg, road300):
    """Continuous batching: queries admitted while others run, stepped with a small time
    budget so they overlap across launches; every result equals the same query run alone
    and the oracle."""
    g, G = road300
    pairs = gg.sample_pairs_grid_steps(g, 60, 5, 400, seed=33, log_uniform=True)
    srv = og.Server(G, max_slots=16, cfg=og.config(delta=512, fusion_threshold=64))
    expect, got = {}, {}
    pending = list(enumerate(pairs.tolist()))
    steps = 0
    while pending or len(got) < len(pairs):
        while pending:
            i, (s, t) = pending[0]
            kind = og.Q_ASTAR if i % 2 else og.Q_PPSP
            if not srv.submit(kind, s, t, tag=i):
                break
            pending.pop(0)
            expect[i] = (og.astar(G, s, t, 512) if kind == og.Q_ASTAR else og.ppsp(G, s, t, 512))
        srv.step(budget_us=50)
        steps += 1
        tags, d = srv.poll()
        for tg, dv in zip(tags.tolist(), d.tolist()):
            got[tg] = dv
        assert steps < 100000
    for i, (s, t) in enumerate(pairs.tolist()):
        assert got[i] == expect[i] == orc.ppsp(g, s, t), i
    assert srv.free_slots() == srv.max_slots
    srv.free()


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("precheck", [1, 2])
def test_precheck_on_off_identical(og, orc, gg, engine, precheck):
    """Reading dist[v] before the atomicMin only skips relaxations that cannot improve:
    distances are unchanged on a skewed and on a road-like graph."""
    for g in (gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=5), gg.road(150, seed=5)):
        G = og.Graph.from_csr(g)
        src = int(gg.sample_sources(g, 1, seed=3)[0])
        got, _, _ = og.query_run(G, og.Q_SSSP, src, cfg=og.config(
            delta=64, precheck=precheck, engine=engine, fusion_threshold=256))
        np.testing.assert_array_equal(got, orc.dijkstra(g, src))


@pytest.mark.parametrize("engine", [1, 2])
def test_csr_and_ell_layouts_identical(og, orc, gg, engine):
    """Graphs of degree <= 8 also get ELL rows (no offsets lookup); both layouts give the
    oracle's distances, for SSSP and for PPSP / A*."""
    g = gg.road(200, seed=11)
    G = og.Graph.from_csr(g)
    src = int(gg.sample_sources(g, 1, seed=4)[0])
    ref = orc.dijkstra(g, src)
    pairs = gg.sample_pairs_grid_steps(g, 6, 5, 150, seed=8)
    for layout in (og.LAYOUT_CSR, og.LAYOUT_ELL):
        cfg = og.config(delta=1024, layout=layout, engine=engine, fusion_threshold=128)
        got, _, _ = og.query_run(G, og.Q_SSSP, src, cfg=cfg)
        np.testing.assert_array_equal(got, ref)
        for s, t in pairs.tolist():
            for kind in (og.Q_PPSP, og.Q_ASTAR):
                _, d, _ = og.query_run(G, kind, s, t, cfg=cfg)
                assert d == orc.ppsp(g, s, t)


def test_hub_vertices_split_across_ctas(og, orc, gg):
    """Vertices with >= hub_degree out-edges (default 4096) are listed and expanded by all
    warps after the round (the BIG phase); a batch over a graph with several such hubs
    stays exact."""
    rng = np.random.default_rng(17)
    n = 60000
    s = [rng.integers(0, n, 120000)]
    d = [rng.integers(0, n, 120000)]
    for hub in (0, 7, 12345):
        s.append(np.full(50000, hub))
        d.append(rng.integers(0, n, 50000))
    s, d = np.concatenate(s), np.concatenate(d)
    w = rng.integers(1, 5000, s.size)
    g = gg.from_edges(n, s, d, w)
    assert np.diff(g.offsets).max() >= 32768
    G = og.Graph.from_csr(g)
    srcs = [0, 7, 999, 12345]
    out, _, _ = og.batch_run(G, [(og.Q_SSSP, x, 0, 256) for x in srcs])
    out = out.reshape(len(srcs), n)
    for i, x in enumerate(srcs):
        np.testing.assert_array_equal(out[i], orc.dijkstra(g, x))


@pytest.mark.parametrize("hub", [32, 200, 1024, 0xFFFFFFFF])
@pytest.mark.parametrize("fusion", [1024, 0xFFFFFFFE])
def test_hub_degree_sweep_rmat(og, orc, gg, hub, fusion):
    """The hub threshold only moves work between the CTA that meets a vertex and the BIG
    phase: every threshold (down to 32, where most edges of an R-MAT graph belong to hubs,
    up to none) and fusion on or off give the oracle's distances for a 4-query batch."""
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 1 << 16, seed=5)
    G = og.Graph.from_csr(g)
    srcs = [int(x) for x in gg.sample_sources(g, 4, seed=3)]
    for tile in (32, 384):
        cfg = og.config(engine=og.ENGINE_ROUNDS, hub_degree=hub, fusion_threshold=fusion,
                        expand_tile=tile)
        out, _, _ = og.batch_run(G, [(og.Q_SSSP, x, 0, 512) for x in srcs], cfg=cfg)
        out = out.reshape(len(srcs), g.n)
        for i, x in enumerate(srcs):
            np.testing.assert_array_equal(out[i], orc.dijkstra(g, x))


def test_autotune_batch_mixed_queries(og, orc, gg, road300):
    """The batch tuner times a mixed SSSP / PPSP / A* batch under its candidates; the
    schedule it returns keeps every query exact.  Bad arguments are rejected."""
    g, G = road300
    srcs = [int(x) for x in gg.sample_sources(g, 6, seed=11)]
    qs = [(og.Q_SSSP, srcs[0], 0, 0), (og.Q_SSSP, srcs[1], 0, 0),
          (og.Q_PPSP, srcs[2], srcs[3], 0), (og.Q_ASTAR, srcs[4], srcs[5], 0)]
    cfg = og.autotune_batch(G, qs, 1 << 8, 1 << 14)
    assert cfg.delta >= 1 and cfg.fusion_threshold > 0
    out, d, _ = og.batch_run(G, qs, cfg=cfg)
    out = out.reshape(len(qs), g.n)
    np.testing.assert_array_equal(out[0], orc.dijkstra(g, srcs[0]))
    np.testing.assert_array_equal(out[1], orc.dijkstra(g, srcs[1]))
    assert d[2] == orc.ppsp(g, srcs[2], srcs[3])
    assert d[3] == orc.ppsp(g, srcs[4], srcs[5])
    for bad in ([], [(og.Q_SSSP, g.n, 0, 0)], [(7, 0, 0, 0)], [(og.Q_PPSP, 0, g.n, 0)]):
        with pytest.raises(og.OgError) as e:
            og.autotune_batch(G, bad)
        assert e.value.code == og.E_INVALID
    G.set_config(og.Config())  # the fixture's graph goes back to library defaults


def test_bellman_ford_matches_oracle(og, orc, gg, grid256, road300):
    """The unordered Bellman-Ford baseline (OG_Q_BF) reaches the oracle's distances on the
    grid, the road-like graph, R-MAT with weights up to 2^16 and ragged random graphs
    with zero weights, self loops and unreachable parts."""
    cases = [(grid256[0], grid256[1], [0, 4321]), (road300[0], road300[1], None)]
    r = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1 << 16, seed=4)
    cases.append((r, og.Graph.from_csr(r), None))
    for seed in (3, 8):
        rg = gg.random_graph(1500, 6000, 0, 20, seed=seed)
        cases.append((rg, og.Graph.from_csr(rg), [0, 7]))
    for g, G, srcs in cases:
        srcs = srcs or [int(x) for x in gg.sample_sources(g, 2, seed=5)]
        for s in srcs:
            got, st = og.bellman_ford(G, s)
            ref = orc.dijkstra(g, s)
            np.testing.assert_array_equal(got, ref)
            np.testing.assert_array_equal(got, orc.bellman_ford(g, s))
            assert st.fused_iters == 0 and st.local_inserts == 0  # no fusion, no order


def test_bellman_ford_round_count_is_hop_depth(og, gg):
    """On a path of k edges round r settles vertex r, so Bellman-Ford needs at least k
    rounds (and one more to see the frontier empty), while Delta-stepping with one wide
    bucket and fusion settles the path in far fewer global rounds."""
    k = 500
    g = gg.path_graph([3] * k)
    G = og.Graph.from_csr(g)
    got, st = og.bellman_ford(G, 0)
    np.testing.assert_array_equal(got, np.arange(k + 1, dtype=np.uint32) * 3)
    assert k <= st.rounds <= k + 2
    cfg = og.config(delta=1 << 20, fusion_threshold=og.FUSION_UNBOUNDED, engine=og.ENGINE_ROUNDS)
    _, _, st2 = og.query_run(G, og.Q_SSSP, 0, cfg=cfg)
    assert st2.rounds < st.rounds // 10


def test_bellman_ford_in_batches_and_small_arenas(og, orc, gg, road300):
    """A batch mixing Bellman-Ford with ordered queries runs on the round engine even
    when the asynchronous engine is asked for; a two-bucket ring with a tiny arena forces
    the overflow pile and its redistribution; the server rejects the kind."""
    g, G = road300
    s = [int(x) for x in gg.sample_sources(g, 4, seed=9)]
    qs = [(og.Q_BF, s[0], 0, 0), (og.Q_SSSP, s[1], 0, 2048), (og.Q_PPSP, s[2], s[3], 2048),
          (og.Q_BF, s[3], 0, 0)]
    out, d, _ = og.batch_run(G, qs, cfg=og.config(engine=og.ENGINE_ASYNC))
    out = out.reshape(4, g.n)
    for i in (0, 1, 3):
        np.testing.assert_array_equal(out[i], orc.dijkstra(g, qs[i][1]))
    assert d[2] == orc.ppsp(g, s[2], s[3]) and d[0] == 0 and d[3] == 0
    cfg = og.config(ring_buckets=2, arena_entries=2000)
    got, _, st = og.query_run(G, og.Q_BF, s[0], cfg=cfg)
    np.testing.assert_array_equal(got, orc.dijkstra(g, s[0]))
    assert st.overflow_inserts > 0 or st.restarts > 0
    srv = og.Server(G, max_slots=4)
    with pytest.raises(og.OgError) as e:
        srv.submit(og.Q_BF, s[0], 0, tag=1)
    assert e.value.code == og.E_INVALID
    srv.free()


def _sym_pairs(gg, n, pairs):
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    s = np.concatenate([pairs[:, 0], pairs[:, 1]])
    d = np.concatenate([pairs[:, 1], pairs[:, 0]])
    return gg.from_edges(n, s, d, np.ones(s.size, np.uint32))


def _cliques(sizes, gap=3):
    """Disjoint cliques (coreness size - 1) plus `gap` isolated vertices after each."""
    pairs, base = [], 0
    for k in sizes:
        idx = np.arange(base, base + k)
        a, b = np.triu_indices(k, 1)
        pairs.append(np.stack([idx[a], idx[b]], 1))
        base += k + gap
    return base, np.concatenate(pairs)


@pytest.mark.parametrize("mode", [0, 1])
def test_kcore_matches_oracle(og, orc, gg, grid256, road300, mode):
    """Coreness, lazy (histogram) and eager, equals the oracle's peeling on the grid, the
    road-like graph, R-MAT (skewed, isolated vertices), random simple graphs, cliques and
    stars."""
    graphs = [grid256[0], road300[0], gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 2, seed=6)]
    rng = np.random.default_rng(4)
    for n, m in ((500, 3000), (2000, 30000)):
        p = rng.integers(0, n, (m, 2))
        p = np.unique(np.sort(p[p[:, 0] != p[:, 1]], 1), axis=0)
        graphs.append(_sym_pairs(gg, n, p))
    n, p = _cliques([1, 2, 5, 40])
    graphs.append(_sym_pairs(gg, n, p))
    graphs.append(_sym_pairs(gg, 50, [(0, i) for i in range(1, 50)]))
    for g in graphs:
        got, st = og.kcore(og.Graph.from_csr(g), mode)
        np.testing.assert_array_equal(got, orc.kcore(g))
        assert st.fused_iters >= 1 and st.rounds >= st.fused_iters


@pytest.mark.parametrize("mode", [0, 1])
def test_kcore_overflowing_buckets_and_window_refills(og, orc, gg, mode):
    """Buckets of 1024 ids overflow on R-MAT's low levels, whose frontiers are then
    rebuilt by scans; cliques of 10, 300 and 600 vertices put coreness levels more than
    256 apart, so the 256-bucket window is refilled twice.  Both stay exact; a device
    output buffer gives the same values."""
    r = gg.rmat(14, 16, 0.57, 0.19, 0.19, 1, 2, seed=7)
    got, st = og.kcore(og.Graph.from_csr(r), mode, cfg=og.config(arena_entries=1))
    np.testing.assert_array_equal(got, orc.kcore(r))
    assert st.flushes > 0
    n, p = _cliques([10, 300, 600])
    g = _sym_pairs(gg, n, p)
    G = og.Graph.from_csr(g)
    got, st = og.kcore(G, mode)
    ref = orc.kcore(g)
    np.testing.assert_array_equal(got, ref)
    assert sorted(set(ref.tolist())) == [0, 9, 299, 599] and st.redistributions >= 2
    dev = _dev(g.n)
    og.kcore(G, mode, out=dev)
    np.testing.assert_array_equal(_np(dev), ref)


def test_kcore_lazy_makes_fewer_updates_than_eager(og, orc, gg):
    """The histogram reduction applies one update per vertex and round where the eager
    update applies one per edge (Section 5.1); the results agree."""
    r = gg.rmat(14, 16, 0.57, 0.19, 0.19, 1, 2, seed=8)
    G = og.Graph.from_csr(r)
    a, sa = og.kcore(G, og.KCORE_LAZY)
    b, sb = og.kcore(G, og.KCORE_EAGER)
    np.testing.assert_array_equal(a, b)
    assert sa.improved < sb.improved and sa.global_inserts < sb.global_inserts
    with pytest.raises(og.OgError) as e:
        og.kcore(G, 7)
    assert e.value.code == og.E_INVALID


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("hub", [8, 100, 0xFFFFFFFF])
def test_kcore_hub_pass(og, orc, gg, mode, hub):
    """Frontier vertices of out-degree >= hub_degree have their edges split over all warps
    after the peel; thresholds down to 8 (most R-MAT edges) and none give the oracle's
    coreness, with the cliques' levels far apart too."""
    r = gg.rmat(13, 16, 0.57, 0.19, 0.19, 1, 2, seed=9)
    cfg = og.config(hub_degree=hub)
    got, _ = og.kcore(og.Graph.from_csr(r), mode, cfg=cfg)
    np.testing.assert_array_equal(got, orc.kcore(r))
    n, p = _cliques([12, 280])
    g = _sym_pairs(gg, n, p)
    got, _ = og.kcore(og.Graph.from_csr(g), mode, cfg=cfg)
    np.testing.assert_array_equal(got, orc.kcore(g))


@pytest.mark.parametrize("delta", [1, 37, 1000, 1 << 20])
def test_lazy_bucket_update_matches_oracle(og, orc, gg, grid256, delta):
    """The lazy bucket update (Section 3.1: relax, mark each improved vertex once, then
    one insertion per marked vertex into the bucket of its final distance) reaches the
    oracle's distances for SSSP on the grid and R-MAT, makes at most one insertion per
    improvement and fuses nothing; the asynchronous engine request falls back to rounds."""
    g, G = grid256
    cfg = og.config(delta=delta, bucket_update=og.UPDATE_LAZY, engine=og.ENGINE_ASYNC)
    for s in (0, 40000):
        got, _, st = og.query_run(G, og.Q_SSSP, s, cfg=cfg)
        np.testing.assert_array_equal(got, orc.dijkstra(g, s))
        assert st.fused_iters == 0 and st.local_inserts == 0
        assert st.global_inserts + st.overflow_inserts <= st.improved
    r = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1 << 16, seed=5)
    R = og.Graph.from_csr(r)
    for s in gg.sample_sources(r, 2, seed=3):
        got, _, _ = og.query_run(R, og.Q_SSSP, int(s), cfg=og.config(delta=delta * 64,
                                 bucket_update=og.UPDATE_LAZY, hub_degree=64))
        np.testing.assert_array_equal(got, orc.dijkstra(r, int(s)))


def test_lazy_bucket_update_batches_ppsp_astar(og, orc, gg, road300):
    """Lazy batches mixing SSSP, PPSP, A*, wBFS-like Delta 1 and Bellman-Ford stay exact;
    the server refuses a lazy schedule."""
    g, G = road300
    s = [int(x) for x in gg.sample_sources(g, 6, seed=13)]
    qs = [(og.Q_SSSP, s[0], 0, 512), (og.Q_PPSP, s[1], s[2], 1024),
          (og.Q_ASTAR, s[3], s[4], 2048), (og.Q_SSSP, s[5], 0, 1), (og.Q_BF, s[2], 0, 0)]
    out, d, _ = og.batch_run(G, qs, cfg=og.config(bucket_update=og.UPDATE_LAZY))
    out = out.reshape(len(qs), g.n)
    for i in (0, 3, 4):
        np.testing.assert_array_equal(out[i], orc.dijkstra(g, qs[i][1]))
    assert d[1] == orc.ppsp(g, s[1], s[2]) and d[2] == orc.ppsp(g, s[3], s[4])
    with pytest.raises(og.OgError) as e:
        og.Server(G, max_slots=4, cfg=og.config(bucket_update=og.UPDATE_LAZY))
    assert e.value.code == og.E_INVALID


def test_server_on_recycled_device_memory(og, orc, gg, road300):
    """A server whose buffers come back from freed device memory holding junk must offer
    nothing to claim in its idle slots: device memory is filled with a non-zero pattern
    and released first, then a 64-slot server answers 3 queries exactly, with a short
    wait limit so that a claim on a query-less slot would fail fast."""
    import torch
    g, G = road300
    junk = torch.full((1 << 28,), 0x00000F00, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    del junk
    torch.cuda.empty_cache()
    pairs = gg.sample_pairs_grid_steps(g, 3, 10, 200, seed=5)
    srv = og.Server(G, max_slots=64, cfg=og.config(delta=512, fusion_threshold=64,
                                                      spin_limit_ns=200_000_000))
    for i, (s, t) in enumerate(pairs.tolist()):
        assert srv.submit(og.Q_PPSP, int(s), int(t), tag=i)
    got = {}
    for _ in range(10000):
        srv.step(budget_us=200)
        tags, d = srv.poll()
        got.update({int(a): int(b) for a, b in zip(tags, d)})
        if len(got) == len(pairs):
            break
    srv.free()
    assert got == {i: orc.ppsp(g, int(s), int(t)) for i, (s, t) in enumerate(pairs.tolist())}


def test_server_slot_reuse_resets_the_reached_blocks(og, orc, gg, road300):
    """A reused slot is reset only in the 256-vertex blocks its previous query reached
    (its touched bitmap), not over the whole row: 80 queries through 2 slots, long-reach
    queries alternating with short ones and SSSP queries that reach every block, every
    result against the oracle.  A block left unreset would hand a later query a distance
    below the true one."""
    g, G = road300
    pairs = gg.sample_pairs_grid_steps(g, 80, 3, 500, seed=44, log_uniform=True)
    srv = og.Server(G, max_slots=2, cfg=og.config(delta=256, fusion_threshold=64))
    got = {}
    i = 0
    kinds = {}
    while len(got) < len(pairs):
        while i < len(pairs):
            s, t = pairs[i].tolist()
            kind = (og.Q_SSSP, og.Q_PPSP, og.Q_ASTAR)[i % 3]
            if not srv.submit(kind, s, t, tag=i):
                break
            kinds[i] = kind
            i += 1
        srv.step(budget_us=100)
        tags, d = srv.poll()
        got.update({int(a): int(b) for a, b in zip(tags, d)})
    srv.free()
    for j, (s, t) in enumerate(pairs.tolist()):
        if kinds[j] != og.Q_SSSP:
            assert got[j] == orc.ppsp(g, s, t), (j, kinds[j])


ALWAYS_PULL = 0xFFFFFFFF  # pull whenever a query's frontier is non-empty


@pytest.mark.parametrize("delta", [1, 16, 1000])
def test_pull_rounds_match_oracle_on_skewed_and_road_graphs(og, orc, gg, delta):
    """Direction optimisation: rounds in which every unsettled vertex pulls from its
    in-neighbours of the current bucket give the oracle's distances -- forced on every
    round, and only on large frontiers -- for SSSP on R-MAT (weights up to 1000) and a
    road-like grid, and for wBFS."""
    for g in (gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1000, seed=7), gg.road(120, seed=7)):
        G = og.Graph.from_csr(g)
        src = int(gg.sample_sources(g, 1, seed=5)[0])
        ref = orc.dijkstra(g, src)
        for div in (ALWAYS_PULL, 8):
            for fusion in (0xFFFFFFFE, 256):
                cfg = og.config(delta=delta, pull_divisor=div, fusion_threshold=fusion,
                                layout=og.LAYOUT_CSR)
                got, _, st = og.query_run(G, og.Q_SSSP, src, cfg=cfg)
                np.testing.assert_array_equal(got, ref, err_msg=f"{g.name} {div} {fusion}")
        w1 = gg.with_weights(g, 1, 24, seed=3)
        G1 = og.Graph.from_csr(w1)
        got, _, _ = og.query_run(G1, og.Q_WBFS, src, cfg=og.config(pull_divisor=ALWAYS_PULL))
        np.testing.assert_array_equal(got, orc.dijkstra(w1, src))


@pytest.mark.parametrize("seed", range(8))
def test_pull_rounds_on_directed_multigraphs(og, orc, gg, seed):
    """Pull reads the in-edges (the transpose the library builds): directed graphs with
    parallel edges, self loops and zero weights, pulled on every round."""
    g = gg.random_graph(int(1500 + 300 * seed), 9000 + 1000 * seed, wlo=0, whi=60,
                        seed=40 + seed, symmetric=False)
    G = og.Graph.from_csr(g)
    src = int(gg.sample_sources(g, 1, seed=seed)[0])
    got, _, _ = og.query_run(G, og.Q_SSSP, src, cfg=og.config(delta=8, pull_divisor=ALWAYS_PULL))
    np.testing.assert_array_equal(got, orc.dijkstra(g, src))


def test_pull_rounds_in_a_mixed_batch(og, orc, gg, road300):
    """SSSP queries pull while PPSP, A* and Bellman-Ford queries of the same launch push."""
    g, G = road300
    srcs = gg.sample_sources(g, 4, seed=77)
    pairs = gg.sample_pairs_grid_steps(g, 4, 5, 150, seed=78)
    qs = [(og.Q_SSSP, int(s), 0, 0) for s in srcs[:3]] + [(og.Q_BF, int(srcs[3]), 0, 0)] + \
         [(og.Q_PPSP if i % 2 else og.Q_ASTAR, int(a), int(b), 0) for i, (a, b) in enumerate(pairs)]
    out, d, _ = og.batch_run(G, qs, cfg=og.config(delta=512, pull_divisor=16,
                                                  fusion_threshold=128))
    rows = out.reshape(len(qs), g.n)
    for i, (kind, s, t, _) in enumerate(qs):
        if kind in (og.Q_SSSP, og.Q_BF):
            np.testing.assert_array_equal(rows[i], orc.dijkstra(g, s))
        else:
            assert int(d[i]) == orc.ppsp(g, s, t)
