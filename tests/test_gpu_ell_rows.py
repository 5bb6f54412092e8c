"""GPU parity of the round engine's ELL row path (graphs of degree <= 8), bit-exact.

The row path reads a vertex's whole row with its stale check, sends improved vertices of
the current bucket to the CTA bin through one warp scan, stages those of later buckets in
a per-CTA outbox that reaches the global buckets at the end of the round.  Every
schedule must still give the oracle's distances (Section 3.3: fusion never reorders
priorities; any legal order of a label-correcting method reaches the same distances):
Delta x fusion threshold, ragged random graphs with zero weights, self loops and
parallel edges, batches of every query kind, a level larger than the bin (entries spill
to the global bucket, and the outbox overflows into direct inserts), and A*.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OFF, UNBOUNDED = 0xFFFFFFFE, 0xFFFFFFFF


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
def road(gg, og):
    g = gg.road(220, seed=21)
    return g, og.Graph.from_csr(g)


def _ell(og, **kw):
    return og.config(layout=og.LAYOUT_ELL, engine=1, **kw)


@pytest.mark.parametrize("delta", [1, 7, 1000, 1 << 20])
@pytest.mark.parametrize("fusion", [OFF, 1, 64, UNBOUNDED])
def test_row_path_schedule_sweep(og, orc, gg, road, delta, fusion):
    g, G = road
    src = int(gg.sample_sources(g, 1, seed=7)[0])
    got, _, st = og.query_run(G, og.Q_SSSP, src, cfg=_ell(og, delta=delta,
                                                           fusion_threshold=fusion))
    np.testing.assert_array_equal(got, orc.dijkstra(g, src))


@pytest.mark.parametrize("seed", range(12))
def test_row_path_random_degree_le8_graphs(og, orc, gg, seed):
    # ragged random multigraphs with zero weights, self loops and parallel edges, every
    # out-degree <= 8 so the ELL rows exist
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 2500))
    deg = rng.integers(0, 9, n)
    src = np.repeat(np.arange(n), deg)
    dst = rng.integers(0, n, src.shape[0])
    w = rng.integers(0, 50 if seed % 2 else 5000, src.shape[0])
    g = gg.from_edges(n, src, dst, w)
    G = og.Graph.from_csr(g)
    s = int(rng.integers(0, n))
    ref = orc.dijkstra(g, s)
    for delta, fusion in ((1, 64), (16, UNBOUNDED), (3, 1), (1 << 12, 256)):
        got, _, _ = og.query_run(G, og.Q_SSSP, s, cfg=_ell(og, delta=delta,
                                                            fusion_threshold=fusion))
        np.testing.assert_array_equal(got, ref, err_msg=f"{delta} {fusion}")


def test_row_path_level_larger_than_the_bin(og, orc, gg):
    """Eight sources start in one frontier tile, so one CTA runs all eight searches in
    its fused loop (unbounded fusion, one bucket): its levels outgrow the 2,048-entry bin
    and the extra entries go to the global current bucket, many of them through the
    outbox's direct-insert path."""
    import torch
    g = gg.road(300, seed=3)
    G = og.Graph.from_csr(g)
    srcs = gg.sample_sources(g, 8, seed=9)
    qs = [(og.Q_SSSP, int(s), 0, 0) for s in srcs]
    out = torch.empty(len(qs) * g.n, dtype=torch.int32, device="cuda")
    _, _, st = og.batch_run(G, qs, cfg=_ell(og, delta=1 << 31, fusion_threshold=UNBOUNDED,
                                           expand_tile=32), out=out)
    d = out.cpu().numpy().view(np.uint32).reshape(len(qs), g.n)
    for i, s in enumerate(srcs):
        np.testing.assert_array_equal(d[i], orc.dijkstra(g, int(s)))
    assert st.global_inserts > 0


def test_row_path_outbox_overflow_with_unit_buckets(og, orc, gg):
    """Delta = 1 with weights up to 1000: nearly every improvement lands in a later
    bucket, so the outbox (512 entries a round) overflows into direct inserts."""
    import torch
    g = gg.road(200, seed=4)
    G = og.Graph.from_csr(g)
    srcs = gg.sample_sources(g, 16, seed=10)
    qs = [(og.Q_SSSP, int(s), 0, 0) for s in srcs]
    out = torch.empty(len(qs) * g.n, dtype=torch.int32, device="cuda")
    og.batch_run(G, qs, cfg=_ell(og, delta=1, fusion_threshold=64), out=out)
    d = out.cpu().numpy().view(np.uint32).reshape(len(qs), g.n)
    for i, s in enumerate(srcs):
        np.testing.assert_array_equal(d[i], orc.dijkstra(g, int(s)))


def test_row_path_mixed_batch_all_kinds(og, orc, gg, road):
    g, G = road
    srcs = gg.sample_sources(g, 6, seed=12)
    pairs = gg.sample_pairs_grid_steps(g, 8, 5, 200, seed=13)
    qs = [(og.Q_SSSP, int(s), 0, 0) for s in srcs[:3]] + \
         [(og.Q_WBFS, int(srcs[3]), 0, 0), (og.Q_BF, int(srcs[4]), 0, 0)] + \
         [(og.Q_PPSP if i % 2 else og.Q_ASTAR, int(a), int(b), 0) for i, (a, b) in enumerate(pairs)]
    out, d, _ = og.batch_run(G, qs, cfg=_ell(og, delta=512, fusion_threshold=128))
    rows = out.reshape(len(qs), g.n)
    for i, (kind, s, t, _) in enumerate(qs):
        if kind in (og.Q_SSSP, og.Q_WBFS, og.Q_BF):
            np.testing.assert_array_equal(rows[i], orc.dijkstra(g, s), err_msg=str(kind))
        else:
            assert int(d[i]) == orc.ppsp(g, s, t), (kind, s, t)
