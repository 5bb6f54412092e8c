"""Allocation-free SSSP entry point (og_sssp_delta_noalloc).

Some callers cannot allocate device memory: a host application whose allocator already
holds the GPU's memory, a path that cannot afford cudaMalloc's implicit device
synchronisation, or code that must not see an out-of-memory error after start-up.  For
them og_sssp_delta_noalloc keeps its scratch in a fixed static device array.  These
tests call it through the C ABI twice in a row and compare every distance with
og_sssp_delta and the oracle (integers: exact equality) -- on a road-like grid, on a
skewed R-MAT graph (no hub list: hubs are expanded where they are met) and on a graph
whose buckets spill into the overflow pile -- check that device memory does not move
across a call, that a run which outgrows the array reports OG_E_ARENA and leaves the
entry point usable, that a malformed graph is refused before any search, and that a graph
larger than the array allows is refused.  This file is collected last on purpose.
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


def _run_twice_and_compare(og, orc, g, cases):
    import torch
    G = og.Graph.from_csr(g)
    off, edges = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    try:
        for src, delta in cases:
            ref = og.sssp_delta(G, src, delta)
            want = orc.dijkstra(g, src)
            np.testing.assert_array_equal(ref, want)
            for _ in range(2):  # two calls in a row share the array
                out.fill_(7)
                og.sssp_delta_noalloc(off, edges, g.n, g.m, src, delta, out)
                got = out.cpu().numpy().view(np.uint32)
                np.testing.assert_array_equal(got, want)
    finally:
        G.free()


def test_noalloc_matches_sssp_delta_on_two_calls(og, gg, orc):
    g = gg.road(400, seed=3)
    _run_twice_and_compare(og, orc, g, [(0, 2048), (g.n // 2, 256)])


def test_noalloc_on_a_skewed_graph(og, gg, orc):
    # R-MAT 14: hubs of degree in the thousands, expanded in place (no hub list here)
    g = gg.rmat(14, wlo=1, whi=1 << 10, seed=5)
    src = int(gg.sample_sources(g, 1, seed=4)[0])
    _run_twice_and_compare(og, orc, g, [(src, 64), (src, 1)])


def test_noalloc_overflow_pile_path(og, gg, orc):
    # weights up to 2^16 and Delta = 8: relaxations jump far past the 256 materialised
    # buckets, so most entries go through the overflow pile and its redistribution
    g = gg.rmat(12, wlo=1, whi=1 << 16, seed=6)
    src = int(gg.sample_sources(g, 1, seed=2)[0])
    _run_twice_and_compare(og, orc, g, [(src, 8)])


def test_noalloc_allocates_nothing(og, gg):
    import torch
    g = gg.road(300, seed=4)
    off, edges = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    og.sssp_delta_noalloc(off, edges, g.n, g.m, 0, 1024, out)  # set-up, kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    og.sssp_delta_noalloc(off, edges, g.n, g.m, 5, 1024, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def _pile_flood_graph(gg, chain=1000, fan=2500, big=1 << 24):
    """u_0 -> u_1 -> ... -> u_chain (weight 1) and every u_i -> v_j (weight big - 2i):
    with Delta = 1 the u_i are settled one bucket at a time and each of them lowers every
    v_j again, far beyond the ring, so chain * fan entries pile up unredistributed."""
    u = np.arange(chain + 1)
    v = chain + 1 + np.arange(fan)
    src = [u[:-1]]
    dst = [u[1:]]
    w = [np.ones(chain, np.int64)]
    for i in range(chain + 1):
        src.append(np.full(fan, i))
        dst.append(v)
        w.append(np.full(fan, big - 2 * i))
    return gg.from_edges(chain + 1 + fan, np.concatenate(src), np.concatenate(dst),
                         np.concatenate(w), name="pileflood")


def test_noalloc_reports_an_exhausted_array_and_stays_usable(og, gg, orc):
    import torch
    g = _pile_flood_graph(gg)
    off, edges = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(og.OgError) as e:
        og.sssp_delta_noalloc(off, edges, g.n, g.m, 0, 1, out)
    assert e.value.code == og.E_ARENA
    # the next call starts from cleared state words
    r = gg.road(200, seed=5)
    roff, redges = _device_csr(r)
    rout = torch.empty(r.n, dtype=torch.int32, device="cuda")
    og.sssp_delta_noalloc(roff, redges, r.n, r.m, 3, 1024, rout)
    np.testing.assert_array_equal(rout.cpu().numpy().view(np.uint32), orc.dijkstra(r, 3))


def test_noalloc_refuses_a_malformed_graph(og, gg, orc):
    import torch
    g = gg.grid(40, 40, 1, 100, seed=2)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    off, edges = _device_csr(g)
    bad_nbr = edges.clone()
    bad_nbr[2 * 17] = g.n + 5  # a neighbor id beyond n
    with pytest.raises(og.OgError) as e:
        og.sssp_delta_noalloc(off, bad_nbr, g.n, g.m, 0, 64, out)
    assert e.value.code == og.E_INVALID and "neighbor" in og.last_cuda_error()
    bad_off = off.clone()
    bad_off[10] = bad_off[12] + 1  # offsets no longer non-decreasing
    with pytest.raises(og.OgError) as e:
        og.sssp_delta_noalloc(bad_off, edges, g.n, g.m, 0, 64, out)
    assert e.value.code == og.E_INVALID and "offsets" in og.last_cuda_error()
    with pytest.raises(og.OgError) as e:  # offsets[n] != m
        og.sssp_delta_noalloc(off, edges, g.n, g.m - 1, 0, 64, out)
    assert e.value.code == og.E_INVALID
    og.sssp_delta_noalloc(off, edges, g.n, g.m, 0, 64, out)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), orc.dijkstra(g, 0))


def test_noalloc_refuses_graphs_beyond_its_array(og):
    import torch
    tiny = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(og.OgError) as e:
        og.sssp_delta_noalloc(tiny, tiny, (1 << 20) + 1, 2, 0, 1, tiny)
    assert e.value.code == og.E_INVALID
