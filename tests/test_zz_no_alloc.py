"""Allocation-free SSSP entry point (og_sssp_delta_noalloc).

Some callers cannot allocate device memory: a host application whose allocator already
holds the GPU's memory, a path that cannot afford cudaMalloc's implicit device
synchronisation, or code that must not see an out-of-memory error after start-up.  For
them og_sssp_delta_noalloc keeps its scratch in a fixed static device array.  These
tests call it through the C ABI twice in a row and compare every distance with
og_sssp_delta (integers: exact equality), and check that a graph larger than the array
allows is refused.  This file is collected last on purpose.
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


def _device_csr(g):
    import torch
    off = torch.from_numpy(g.offsets.astype(np.uint32).view(np.int32)).cuda()
    pairs = np.ascontiguousarray(np.stack([g.nbr, g.w], axis=1).reshape(-1))
    edges = torch.from_numpy(pairs.view(np.int32)).cuda()
    return off, edges


def test_noalloc_matches_sssp_delta_on_two_calls(og, gg, orc):
    import torch
    g = gg.road(400, seed=3)
    G = og.Graph.from_csr(g)
    off, edges = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for src, delta in [(0, 2048), (g.n // 2, 256)]:
        ref = og.sssp_delta(G, src, delta)
        og.sssp_delta_noalloc(off, edges, g.n, g.m, src, delta, out)
        got = out.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_array_equal(got, orc.dijkstra(g, src))


def test_noalloc_refuses_graphs_beyond_its_array(og):
    import torch
    tiny = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(og.OgError) as e:
        og.sssp_delta_noalloc(tiny, tiny, (1 << 20) + 1, 2, 0, 1, tiny)
    assert e.value.code == og.E_INVALID
