"""GPU parity at the benchmarked full sizes, in the launch configurations bench.py times.

* The default workload: the road-like 4900 x 4900 grid (23,997,150 vertices, 82,565,692
  directed edges, every weight >= 100) and the bench's 8 seeded sources in one
  persistent batch launch (`og_batch_run`), under the library's default schedule and
  under the schedule the autotuner picks for this graph (Delta 4096, fusion threshold
  1024, tile 32). Every source's distance array passes the oracle's certificate check
  -- dist[src] = 0, no edge can improve a distance, every reached vertex has a tight
  in-edge -- which with positive weights holds for the exact shortest-path distances
  only; two of the sources are also compared element by element with the oracle's
  Dijkstra.
* R-MAT scale 24 (16,777,216 vertices, 520,762,674 directed edges, weights in
  [1, 2^16)) with the bench's 8 sources and its tuned schedule (Delta 256, fusion off,
  tile 256): the certificate on two sources (a Dijkstra there takes ~40 s a source).
* R-MAT scale 24 wBFS (the same structure with weights in [1, 24)), the bench's 8
  sources in one launch under the library's default schedule (Delta 1): every source's
  distances pass the certificate, and one is compared element by element with Dijkstra.
* k-core on the same R-MAT graph (the bench's `rmat-kcore` graph: the generator's
  structure does not depend on the weight range, and k-core ignores weights), lazy and
  eager in the bench's launch: the lazy result passes the oracle's linear-time k-core
  certificate, which only the exact coreness passes (the oracle's own peeling takes ~5
  minutes at this size), and the eager result equals it.
* Set cover on the same R-MAT graph (its structure does not depend on the weight range,
  and set cover ignores weights, so it is the `rmat-setcover` workload), in the bench's
  launch shape and another one: every set's join step equals the oracle's.
"""
import numpy as np
import pytest

# generous limits (pytest-timeout): graph generation and the one-core oracle dominate
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]


@pytest.fixture(scope="module")
def og():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1911_07260_gb300 as og
    from paper_1911_07260_gb300 import build
    build.build()
    torch.cuda.init()
    return og


def test_full_size_road_batch_vs_oracle(og, orc):
    import torch
    import bench
    g, _, srcs = bench.build_workload(bench.parse_args([]), 0, 1)
    assert (g.n, g.m, len(srcs)) == (23997150, 82565692, 8)
    assert int(g.w.min()) >= 1
    G = og.Graph.from_csr(g)
    queries = [(og.Q_SSSP, int(s), 0, 0) for s in srcs]
    out = torch.empty(len(queries) * g.n, dtype=torch.int32, device="cuda")
    ref = {i: orc.dijkstra(g, int(srcs[i])) for i in (0, len(srcs) - 1)}
    for cfg in (None, og.config(delta=4096, fusion_threshold=1024, expand_tile=32)):
        og.batch_run(G, queries, cfg=cfg, out=out)
        d = out.cpu().numpy().view(np.uint32).reshape(len(queries), g.n)
        for i, s in enumerate(srcs):
            assert orc.check_sssp(g, int(s), d[i]) == (0, 0), (i, cfg)
        for i, r in ref.items():
            np.testing.assert_array_equal(d[i], r)
    del out
    G.free()


@pytest.fixture(scope="module")
def rmat24():
    import bench
    g, _, srcs = bench.build_workload(bench.parse_args(["--workload", "rmat-sssp"]), 0, 1)
    assert (g.n, g.m, len(srcs)) == (16777216, 520762674, 8)
    return g, srcs


def test_full_size_rmat_sssp_batch_certified(og, orc, rmat24):
    import torch
    g, srcs = rmat24
    assert int(g.w.min()) >= 1
    G = og.Graph.from_csr(g)
    queries = [(og.Q_SSSP, int(s), 0, 0) for s in srcs]
    out = torch.empty(len(queries) * g.n, dtype=torch.int32, device="cuda")
    cfg = og.config(delta=256, fusion_threshold=og.FUSION_OFF, expand_tile=256)
    og.batch_run(G, queries, cfg=cfg, out=out)
    d = out.cpu().numpy().view(np.uint32).reshape(len(queries), g.n)
    for i in (0, len(srcs) - 1):
        assert orc.check_sssp(g, int(srcs[i]), d[i]) == (0, 0), i
    del out
    G.free()


def test_full_size_rmat_wbfs_batch_vs_oracle(og, orc):
    import torch
    import bench
    g, _, srcs = bench.build_workload(bench.parse_args(["--workload", "rmat-wbfs"]), 0, 1)
    assert (g.n, g.m, len(srcs)) == (16777216, 520762674, 8)
    assert int(g.w.min()) >= 1 and int(g.w.max()) < 24
    G = og.Graph.from_csr(g)
    queries = [(og.Q_WBFS, int(s), 0, 0) for s in srcs]
    out = torch.empty(len(queries) * g.n, dtype=torch.int32, device="cuda")
    og.batch_run(G, queries, out=out)
    d = out.cpu().numpy().view(np.uint32).reshape(len(queries), g.n)
    del out
    G.free()
    for i, s in enumerate(srcs):
        assert orc.check_sssp(g, int(s), d[i]) == (0, 0), i
    np.testing.assert_array_equal(d[0], orc.dijkstra(g, int(srcs[0])))


def test_full_size_rmat_kcore_certified(og, orc, rmat24):
    import torch
    g, _ = rmat24
    G = og.Graph.from_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    og.kcore(G, og.KCORE_LAZY, out=out)
    lazy = out.cpu().numpy().view(np.uint32).copy()
    og.kcore(G, og.KCORE_EAGER, out=out)
    eager = out.cpu().numpy().view(np.uint32).copy()
    del out
    G.free()
    assert int(lazy.max()) == 1621
    assert orc.check_kcore(g, lazy) == (0, 0)
    np.testing.assert_array_equal(eager, lazy)


def test_full_size_rmat_setcover(og, orc, gg, rmat24):
    g, _ = rmat24
    G = og.Graph.from_csr(g)
    pri = gg.priorities(g.n, seed=1)
    a, st = og.setcover(G, 10000, pri)
    b, _ = og.setcover(G, 10000, pri, cfg=og.config(hub_degree=16, blocks_per_sm=1))
    G.free()
    ref, steps = orc.setcover(g, pri, 10000)  # ~40 s on one core
    np.testing.assert_array_equal(a, ref)
    np.testing.assert_array_equal(b, ref)
    assert st.rounds == steps and st.improved == int((ref > 0).sum())
