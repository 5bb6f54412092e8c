"""GPU parity at the benchmarked full size, in the launch configuration bench.py times.

The default workload: the road-like 4900 x 4900 grid (23,997,150 vertices, 82,565,692
directed edges, every weight >= 100) and the bench's 8 seeded sources in one persistent
batch launch (`og_batch_run`), under the library's default schedule and under the
schedule the autotuner picks for this graph (Delta 4096, fusion threshold 1024, tile 32).
Every source's distance array passes the oracle's certificate check -- dist[src] = 0,
no edge can improve a distance, every reached vertex has a tight in-edge -- which with
positive weights holds for the exact shortest-path distances only; two of the sources
are also compared element by element with the oracle's Dijkstra.
"""
import numpy as np
import pytest

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
