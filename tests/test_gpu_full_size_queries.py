"""GPU parity of the batched and the served query workloads at their benchmarked sizes.

* Batching: 256 concurrent queries on the road-like 1024 x 1024 grid (1,048,019
  vertices), 128 SSSP from seeded sources and 128 PPSP with targets 10 .. 1000 grid
  steps away, in ONE `og_batch_run` launch under the schedule `og_autotune_batch` picks
  for the whole batch -- the bench's `batch` workload.  256 queries share the CTA bins
  (16-bit query ids) and the arenas are sized from free device memory.  Every SSSP row
  passes the oracle's certificate (which with positive weights only the exact distances
  pass) and two rows equal the oracle's Dijkstra element by element; every PPSP result
  equals the oracle's point-to-point Dijkstra (PPSP is defined in Section 6.1).
* Serving: 256 A* / PPSP queries (kind by a seeded coin, targets log-uniform 10 .. 1000
  grid steps away) on the road-like 4900 x 4900 grid with its integral coordinates,
  through `og_server_*` with the bench's 128 slots, 400 us launches and fusion threshold
  64; queries are admitted whenever a slot frees up, so later ones join launches that
  earlier ones are still running in.  Every served result equals the same query run
  alone (`og_astar` / `og_ppsp`) and the oracle's point-to-point Dijkstra.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

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


def _oracle_ppsp(orc, g, pairs):
    with ThreadPoolExecutor(16) as ex:  # the C oracle releases the GIL
        return list(ex.map(lambda p: orc.ppsp(g, int(p[0]), int(p[1])), pairs))


def test_batch_of_256_mixed_queries_at_full_size(og, orc, gg):
    import torch
    g = gg.road(1024, 0.15, 0.02, seed=1)
    assert g.n == 1048019
    G = og.Graph.from_csr(g)
    srcs = gg.sample_sources(g, 128, seed=2)
    pairs = gg.sample_pairs_grid_steps(g, 128, 10, 1000, seed=2)
    queries = [(og.Q_SSSP, int(s), 0, 0) for s in srcs] + \
              [(og.Q_PPSP, int(a), int(b), 0) for a, b in pairs]
    cfg = og.autotune_batch(G, queries, 1 << 8, 1 << 16)
    nq = len(queries)
    out = torch.empty(nq * g.n, dtype=torch.int32, device="cuda")
    _, d, _ = og.batch_run(G, queries, cfg=cfg, out=out)
    dist = out.cpu().numpy().view(np.uint32).reshape(nq, g.n)
    for i in range(128):
        assert orc.check_sssp(g, int(srcs[i]), dist[i]) == (0, 0), i
    for i in (0, 127):
        np.testing.assert_array_equal(dist[i], orc.dijkstra(g, int(srcs[i])))
    want = _oracle_ppsp(orc, g, pairs)
    got = [int(x) for x in d[128:]]
    assert got == [int(x) for x in want]
    # a PPSP row holds true distances for every vertex it settled: its target's entry
    for j in range(128):
        assert int(dist[128 + j][int(pairs[j][1])]) == int(want[j])
    G.free()


def test_served_astar_and_ppsp_on_the_full_road_graph(og, orc, gg):
    g = gg.road(4900, 0.15, 0.02, seed=1)
    assert g.n == 23997150 and g.xy is not None
    G = og.Graph.from_csr(g)
    total = 256
    pairs = gg.sample_pairs_grid_steps(g, total, 10, 1000, seed=2, log_uniform=True)
    rng = np.random.default_rng(7)
    kinds = np.where(rng.random(total) < 0.5, og.Q_ASTAR, og.Q_PPSP)
    tune = og.autotune(G, og.Q_PPSP, pairs[:32, 0], pairs[:32, 1], 1 << 6, 1 << 14)
    cfg = og.config(delta=int(tune.delta), fusion_threshold=64)
    srv = og.Server(G, max_slots=128, cfg=cfg)
    got = np.full(total, 0xFFFFFFFE, np.uint32)
    nxt = done = 0
    overlapped = 0  # admissions into a launch sequence with queries already running
    running = 0
    for _ in range(1_000_000):
        while nxt < total and srv.submit(int(kinds[nxt]), int(pairs[nxt, 0]),
                                         int(pairs[nxt, 1]), nxt):
            overlapped += running > 0
            nxt += 1
        running = srv.step(budget_us=400)
        tags, dd = srv.poll()
        got[tags.astype(np.int64)] = dd
        done += len(tags)
        if done == total:
            break
    srv.free()
    assert done == total
    assert overlapped > 0
    alone = np.array([og.astar(G, int(s), int(t), int(cfg.delta)) if k == og.Q_ASTAR else
                      og.ppsp(G, int(s), int(t), int(cfg.delta))
                      for (s, t), k in zip(pairs, kinds)], np.uint32)
    np.testing.assert_array_equal(got, alone)
    want = np.array(_oracle_ppsp(orc, g, pairs), np.uint32)
    np.testing.assert_array_equal(got, want)
    G.free()
