"""Pins for the CPU oracle against things other than itself (CPU only).

* hand-worked fixtures (tests/golden/hand_worked.txt),
* brute-force enumeration of simple paths on tiny graphs,
* scipy.sparse.csgraph's Dijkstra (an independent library routine),
* closed forms: path prefix sums, constant-weight grids (c * Manhattan distance),
  unit weights (BFS hop counts), stars, disconnected parts,
* the certificate (edge) invariant and its sensitivity to planted mistakes.
"""
import itertools

import numpy as np
import pytest

from tests.golden import fixtures

INF = 0xFFFFFFFF


def _brute(n, edges, src):
    """Minimum over all simple paths from src (exhaustive DFS; tiny n only)."""
    adj = [[] for _ in range(n)]
    for u, v, w in edges:
        adj[u].append((v, w))
    best = [None] * n

    def dfs(u, acc, seen):
        if best[u] is None or acc < best[u]:
            best[u] = acc
        for v, w in adj[u]:
            if v not in seen:
                seen.add(v)
                dfs(v, acc + w, seen)
                seen.remove(v)

    dfs(src, 0, {src})
    return [INF if b is None else b for b in best]


def _edges_of(g):
    src = np.repeat(np.arange(g.n), np.diff(g.offsets).astype(np.int64))
    return list(zip(src.tolist(), g.nbr.tolist(), g.w.tolist()))


def test_golden_fixtures(gg, orc):
    cases = fixtures.load()
    assert len(cases) >= 5
    for c in cases:
        s, d, w = zip(*c["edges"])
        g = gg.from_edges(c["n"], s, d, w)
        if c["target"] is None:
            assert orc.dijkstra(g, c["src"]).tolist() == c["expect"], c["name"]
            assert orc.bellman_ford(g, c["src"]).tolist() == c["expect"], c["name"]
        else:
            assert orc.ppsp(g, c["src"], c["target"]) == c["expect"][0], c["name"]


@pytest.mark.parametrize("seed", range(300))
def test_dijkstra_vs_brute_force(gg, orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 7))
    m = int(rng.integers(0, 14))
    g = gg.random_graph(n, m, wlo=0, whi=int(rng.choice([2, 5, 50])), seed=seed)
    src = int(rng.integers(0, n))
    ref = _brute(n, _edges_of(g), src)
    assert orc.dijkstra(g, src).tolist() == ref
    assert orc.bellman_ford(g, src).tolist() == ref
    for t in range(n):
        assert orc.ppsp(g, src, t) == ref[t]


@pytest.mark.parametrize("seed", range(20))
def test_dijkstra_vs_scipy(gg, orc, seed):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 300))
    m = int(rng.integers(n, 6 * n))
    g = gg.random_graph(n, m, wlo=1, whi=int(rng.choice([3, 100, 100000])), seed=seed,
                       symmetric=bool(seed % 2), self_loops=True)
    # scipy sums duplicate entries, so collapse parallel edges to their minimum first;
    # self loops never shorten a path and are dropped.
    best = {}
    for u, v, w in _edges_of(g):
        if u != v:
            best[(u, v)] = min(w, best.get((u, v), w))
    if best:
        rows, cols = zip(*best.keys())
        vals = list(best.values())
    else:
        rows, cols, vals = [], [], []
    mat = sp.csr_matrix((np.array(vals, float), (rows, cols)), shape=(n, n))
    for src in rng.integers(0, n, 3):
        ref = csg.dijkstra(mat, directed=True, indices=int(src))
        ref = np.where(np.isinf(ref), INF, ref).astype(np.uint64)
        got = orc.dijkstra(g, int(src))
        np.testing.assert_array_equal(got.astype(np.uint64), ref)


def test_path_prefix_sums(gg, orc):
    w = np.array([5, 0, 17, 1, 999, 3, 0, 42], np.uint32)
    g = gg.path_graph(w)
    expect = np.concatenate([[0], np.cumsum(w)])
    np.testing.assert_array_equal(orc.dijkstra(g, 0), expect)
    # Everything before the source is unreachable on a directed path.
    d = orc.dijkstra(g, 3)
    assert (d[:3] == INF).all()
    np.testing.assert_array_equal(d[3:], np.concatenate([[0], np.cumsum(w[3:])]))


@pytest.mark.parametrize("c", [1, 7, 1000])
def test_constant_grid_is_manhattan(gg, orc, c):
    k = 23
    g = gg.grid(k, k, c, c + 1, seed=3)
    assert (g.w == c).all()
    for src in [0, k * k - 1, 5 * k + 11]:
        r0, c0 = divmod(src, k)
        rr, cc = np.divmod(np.arange(k * k), k)
        manhattan = (np.abs(rr - r0) + np.abs(cc - c0)) * c
        np.testing.assert_array_equal(orc.dijkstra(g, src), manhattan)
        np.testing.assert_array_equal(orc.bfs(g, src) * c, manhattan)


@pytest.mark.parametrize("seed", range(10))
def test_unit_weights_equal_bfs(gg, orc, seed):
    g = gg.random_graph(200, 700, wlo=1, whi=2, seed=seed, symmetric=bool(seed % 2))
    for src in (0, 17, 199):
        np.testing.assert_array_equal(orc.dijkstra(g, src), orc.bfs(g, src))


def test_star_and_disconnected(gg, orc):
    # star 0 -> 1..9 with weight i, plus an isolated component {10, 11}.
    s = [0] * 9 + [10]
    d = list(range(1, 10)) + [11]
    w = list(range(1, 10)) + [4]
    g = gg.from_edges(12, s, d, w)
    got = orc.dijkstra(g, 0)
    assert got.tolist() == [0] + list(range(1, 10)) + [INF, INF]
    assert orc.dijkstra(g, 10).tolist() == [INF] * 10 + [0, 4]


def test_overflow_is_reported(gg, orc):
    g = gg.path_graph([0xFFFFFFF0, 0x10, 0x10])
    with pytest.raises(orc.OracleError):
        orc.dijkstra(g, 0)
    d = orc.dijkstra(g, 0, allow_overflow=True)
    assert d[1] == 0xFFFFFFF0 and d[2] == orc.SATURATED and d[3] == orc.SATURATED


@pytest.mark.parametrize("seed", range(10))
def test_certificate_accepts_oracle_and_rejects_planted_mistakes(gg, orc, seed):
    g = gg.random_graph(300, 1500, wlo=1, whi=50, seed=seed, symmetric=True)
    src = seed
    d = orc.dijkstra(g, src)
    assert orc.check_sssp(g, src, d) == (0, 0)
    reached = np.nonzero((d != INF) & (np.arange(g.n) != src))[0]
    assert reached.size > 10
    v = int(reached[seed % reached.size])
    up = d.copy(); up[v] += 1          # too large: some in-edge is violated
    assert orc.check_sssp(g, src, up)[0] == 2
    down = d.copy(); down[v] -= 1      # too small: no tight in-edge
    assert orc.check_sssp(g, src, down)[0] in (2, 3)
    lost = d.copy(); lost[v] = INF     # dropped vertex
    assert orc.check_sssp(g, src, lost)[0] == 2
    bad_src = d.copy(); bad_src[src] = 1
    assert orc.check_sssp(g, src, bad_src)[0] == 1


def test_pins_catch_plausible_oracle_mistakes(gg, orc):
    """Run the oracle on mutated inputs that model a transposed operand (edges read
    backwards) and a misindexed weight array; the brute-force pin must reject both."""
    rejected_t = rejected_w = 0
    for seed in range(40):
        g = gg.random_graph(6, 10, wlo=1, whi=20, seed=seed, self_loops=False)
        e = _edges_of(g)
        ref = _brute(g.n, e, 0)
        rev = gg.from_edges(g.n, [x[1] for x in e], [x[0] for x in e], [x[2] for x in e])
        rejected_t += orc.dijkstra(rev, 0).tolist() != ref
        shifted = gg.Graph("shift", g.offsets, g.nbr, np.roll(g.w, 1))
        rejected_w += orc.dijkstra(shifted, 0).tolist() != ref
    assert rejected_t > 20 and rejected_w > 20


def test_ppsp_stops_at_target_with_final_value(gg, orc):
    g = gg.grid(40, 40, 1, 1000, seed=5)
    full = orc.dijkstra(g, 0)
    for t in [1, 39, 800, 1599]:
        assert orc.ppsp(g, 0, t) == int(full[t])


def test_oracle_rejects_bad_arguments(gg, orc):
    g = gg.path_graph([1, 2])
    with pytest.raises(orc.OracleError):
        orc.dijkstra(g, 3)
    with pytest.raises(orc.OracleError):
        orc.dijkstra(g, 0, target=9)


# ---- k-core (coreness by peeling) -------------------------------------------------------

def _sym(gg, n, pairs):
    """Symmetric simple graph from undirected pairs (unit weights)."""
    s = [u for u, v in pairs] + [v for u, v in pairs]
    d = [v for u, v in pairs] + [u for u, v in pairs]
    return gg.from_edges(n, s, d, [1] * len(s))


def _core_brute(n, pairs):
    """Coreness by its definition: the largest k such that v lies in a vertex set whose
    induced subgraph has minimum degree >= k (every subset enumerated; tiny n only)."""
    adj = [set() for _ in range(n)]
    for u, v in pairs:
        adj[u].add(v)
        adj[v].add(u)
    core = [0] * n
    for r in range(1, n + 1):
        for S in itertools.combinations(range(n), r):
            Sset = set(S)
            k = min(len(adj[v] & Sset) for v in S)
            for v in S:
                core[v] = max(core[v], k)
    return core


def test_kcore_closed_forms(gg, orc):
    """Clique K_n: n - 1; cycle: 2; path and star: 1; isolated: 0; complete bipartite
    K_{a,b}: min(a, b); 4-neighbour grid: 2 everywhere."""
    n = 9
    g = _sym(gg, n, list(itertools.combinations(range(n), 2)))
    assert orc.kcore(g).tolist() == [n - 1] * n
    g = _sym(gg, 12, [(i, (i + 1) % 12) for i in range(12)])
    assert orc.kcore(g).tolist() == [2] * 12
    g = _sym(gg, 8, [(i, i + 1) for i in range(6)])  # path on 0..6, vertex 7 isolated
    assert orc.kcore(g).tolist() == [1] * 7 + [0]
    g = _sym(gg, 10, [(0, i) for i in range(1, 10)])
    assert orc.kcore(g).tolist() == [1] * 10
    a, b = 4, 7
    g = _sym(gg, a + b, [(i, a + j) for i in range(a) for j in range(b)])
    assert orc.kcore(g).tolist() == [min(a, b)] * (a + b)
    assert set(orc.kcore(gg.grid(17, 23, 1, 9, seed=3)).tolist()) == {2}


@pytest.mark.parametrize("seed", range(12))
def test_kcore_vs_definition_brute_force(gg, orc, seed):
    """Random simple graphs on 9 vertices, densities from sparse to near-complete."""
    rng = np.random.default_rng(seed)
    n = 9
    p = 0.15 + 0.07 * seed
    pairs = [(u, v) for u, v in itertools.combinations(range(n), 2) if rng.random() < p]
    g = _sym(gg, n, pairs)
    assert orc.kcore(g).tolist() == _core_brute(n, pairs)


def test_kcore_multigraph_counts_csr_entries():
    """Hand-worked: with parallel edges every CSR entry counts toward the degree and
    every removal lowers the neighbour once per entry.  Vertices 0 and 1 joined by three
    parallel edges (both directions) and vertex 2 hanging off 1 by one edge:
    deg = (3, 4, 1); 2 goes at level 1, then 1 drops to 3, and 0 and 1 stay 3-cores."""
    import graphgen as gg
    import oracle as orc
    s = [0, 0, 0, 1, 1, 1, 1, 2]
    d = [1, 1, 1, 0, 0, 0, 2, 1]
    g = gg.from_edges(3, s, d, [1] * len(s))
    assert orc.kcore(g).tolist() == [3, 3, 1]


def test_kcore_level_sets_are_cores(gg, orc):
    """On an R-MAT graph: for every k the vertices of coreness >= k induce a subgraph of
    minimum degree >= k, and no vertex of coreness k has k + 1 neighbours of coreness
    >= k + 1 (else adding it to them would give a larger (k+1)-core)."""
    g = gg.rmat(11, 16, 0.57, 0.19, 0.19, 1, 2, seed=2)
    core = orc.kcore(g).astype(np.int64)
    off = g.offsets.astype(np.int64)
    src = np.repeat(np.arange(g.n), np.diff(off))
    dst = g.nbr.astype(np.int64)
    for k in range(1, int(core.max()) + 1):
        keep = core >= k
        inside = keep[src] & keep[dst]
        deg_in = np.bincount(src[inside], minlength=g.n)
        assert (deg_in[keep] >= k).all()
        up = core[dst] >= k + 1
        at_k = core[src] == k
        cnt = np.bincount(src[at_k & up], minlength=g.n)
        assert (cnt[core == k] <= k).all()


def _kcore_graphs(gg):
    """Symmetric, multigraph, directed and self-loop cases for the k-core certificate."""
    out = [("clique9", _sym(gg, 9, list(itertools.combinations(range(9), 2)))),
           ("path+isolated", _sym(gg, 8, [(i, i + 1) for i in range(6)])),
           ("K4,7", _sym(gg, 11, [(i, 4 + j) for i in range(4) for j in range(7)])),
           ("grid", gg.grid(9, 11, 1, 9, seed=3)),
           ("rmat9", gg.rmat(9, 8, 0.57, 0.19, 0.19, 1, 2, seed=2)),
           ("multigraph", gg.from_edges(3, [0, 0, 0, 1, 1, 1, 1, 2], [1, 1, 1, 0, 0, 0, 2, 1],
                                        [1] * 8))]
    rng = np.random.default_rng(7)
    for i in range(4):
        n = 40 + 10 * i
        s = rng.integers(0, n, 4 * n)
        d = rng.integers(0, n, 4 * n)  # directed, with self-loops and parallel entries
        out.append((f"directed{i}", gg.from_edges(n, s, d, np.ones(len(s), np.uint32))))
    return out


@pytest.mark.parametrize("case", range(6))
def test_kcore_vs_networkx_core_number(gg, orc, case):
    """On simple undirected graphs the peeling's coreness equals networkx's core_number
    (an independent implementation of the textbook definition): random graphs from
    sparse to dense, and cleaned symmetric R-MAT graphs with their skewed degrees."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(100 + case)
    if case < 4:
        n = 300 + 150 * case
        m = int(n * (2 + 6 * case))
        a, b = rng.integers(0, n, m), rng.integers(0, n, m)
        keep = a != b
        pairs = {(int(min(x, y)), int(max(x, y))) for x, y in zip(a[keep], b[keep])}
        g = _sym(gg, n, sorted(pairs))
    else:
        g = gg.rmat(9 + case, 16, 0.57, 0.19, 0.19, 1, 2, seed=case)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    assert not (src == g.nbr).any()  # simple: no self-loops
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(src.tolist(), g.nbr.tolist()))
    assert 2 * G.number_of_edges() == g.m  # symmetric, no parallel entries
    want = nx.core_number(G)
    got = orc.kcore(g)
    assert got.tolist() == [want[v] for v in range(g.n)]
    assert orc.check_kcore(g, got) == (0, 0)


def test_kcore_certificate_accepts_the_oracle_and_nothing_else(gg, orc):
    """The certificate holds for or_kcore's output on every graph kind, and fails for
    every vector that differs from it in one vertex by +1 or -1 (the coreness vector is
    the only one that passes)."""
    for name, g in _kcore_graphs(gg):
        core = orc.kcore(g)
        assert orc.check_kcore(g, core) == (0, 0), name
        for v in range(g.n):
            for dv in (1, -1):
                if core[v] == 0 and dv < 0:
                    continue
                c = core.astype(np.int64)
                c[v] += dv
                assert orc.check_kcore(g, c.astype(np.uint32))[0] in (1, 2), (name, v, dv)


@pytest.mark.parametrize("seed", range(20))
def test_kcore_certificate_on_random_directed_multigraphs(gg, orc, seed):
    """Directed graphs with self-loops and parallel entries, from very sparse to dense:
    the oracle's peeling passes, and 50 random changes of one to three values fail."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(5, 120))
    m = int(rng.integers(0, 12 * n))
    g = gg.from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m), np.ones(m, np.uint32))
    core = orc.kcore(g)
    assert orc.check_kcore(g, core) == (0, 0)
    for _ in range(50):
        c = core.astype(np.int64)
        idx = rng.integers(0, n, rng.integers(1, 4))
        c[idx] = np.maximum(0, c[idx] + rng.choice([-1, 1], len(idx)))
        if (c == core).all():
            continue
        assert orc.check_kcore(g, c.astype(np.uint32))[0] in (1, 2)


def test_kcore_certificate_codes(gg, orc):
    """A value above the vertex's degree fails (a) at that vertex; all zeros on a graph
    with an edge fails (b) at level 0; degrees fail unless every vertex is extracted at
    its own degree (a cycle: degree 2 = coreness 2)."""
    g = _sym(gg, 8, [(i, i + 1) for i in range(6)])  # path on 0..6, vertex 7 isolated
    c = orc.kcore(g).copy()
    c[3] = 3
    assert orc.check_kcore(g, c) == (1, 3)
    code, v = orc.check_kcore(g, np.zeros(g.n, np.uint32))
    assert code == 2 and 0 <= v < 7
    deg = np.diff(g.offsets).astype(np.uint32)
    assert orc.check_kcore(g, deg)[0] == 1
    cyc = _sym(gg, 12, [(i, (i + 1) % 12) for i in range(12)])
    assert orc.check_kcore(cyc, np.diff(cyc.offsets).astype(np.uint32)) == (0, 0)
    with pytest.raises(orc.OracleError):
        orc.check_kcore(g, np.zeros(g.n - 1, np.uint32))


def test_kcore_certificate_on_random_perturbations(gg, orc):
    """R-MAT scale 12: 300 vectors with a few random changes each are all rejected."""
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 1, 2, seed=4)
    core = orc.kcore(g)
    assert orc.check_kcore(g, core) == (0, 0)
    rng = np.random.default_rng(11)
    for _ in range(300):
        c = core.astype(np.int64)
        idx = rng.integers(0, g.n, rng.integers(1, 4))
        c[idx] = np.maximum(0, c[idx] + rng.choice([-2, -1, 1, 2], len(idx)))
        if (c == core).all():
            continue
        assert orc.check_kcore(g, c.astype(np.uint32))[0] in (1, 2)


# ---- k-core mutants: plausible mistakes planted in a copy of the oracle's source ---------

# The floor at the level k and the level that only rises each keep the result exact on
# their own (a priority never falls below k, so the level never has to fall), so removing
# one of them alone changes nothing; the mistake is losing both.
_KCORE_MUTANTS = {
    # neighbours lowered below the current level and the level following them down
    "no_floor_level_drops": [("if (done[w] || prio[w] <= k) continue;",
                              "if (done[w] || prio[w] == 0) continue;"),
                             ("if (prio[v] > k) k = prio[v];", "k = prio[v];")],
    # a neighbour loses two per extracted vertex instead of one
    "double_decrement": [("prio[w] -= 1;", "prio[w] -= (prio[w] > k + 1) ? 2 : 1;")],
    # the level set from the neighbour count instead of the extracted priority
    "level_from_degree": [("if (prio[v] > k) k = prio[v];",
                           "if (off[v + 1] - off[v] > k) k = (uint32_t)(off[v + 1] - off[v]);")],
}

_KCORE_RUNNER = r"""
import ctypes, itertools, sys, numpy as np
sys.path.insert(0, sys.argv[2])
import graphgen as gg
from tests.test_oracle_pins import _core_brute
L = ctypes.CDLL(sys.argv[1])
vp, u32 = ctypes.c_void_p, ctypes.c_uint32
L.or_kcore.argtypes = [u32, vp, vp, vp]
bad = 0
for seed in range(12):
    rng = np.random.default_rng(seed)
    n = 9
    p = 0.15 + 0.07 * seed
    pairs = [(u, v) for u, v in itertools.combinations(range(n), 2) if rng.random() < p]
    s = [u for u, v in pairs] + [v for u, v in pairs]
    d = [v for u, v in pairs] + [u for u, v in pairs]
    g = gg.from_edges(n, s, d, [1] * len(s))
    off = np.ascontiguousarray(g.offsets, np.uint64)
    nbr = np.ascontiguousarray(g.nbr, np.uint32)
    out = np.empty(n, np.uint32)
    L.or_kcore(n, off.ctypes.data, nbr.ctypes.data, out.ctypes.data)
    bad += out.tolist() != _core_brute(n, pairs)
print(bad)
"""


@pytest.mark.parametrize("name", sorted(_KCORE_MUTANTS))
def test_kcore_pins_reject_planted_mistakes(gg, orc, tmp_path, name):
    """Each mutant of or_kcore (compiled from a patched copy of oracle.c) must disagree
    with the coreness definition (subset brute force) on some of the random graphs."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "oracle.c")).read()
    for old, new in _KCORE_MUTANTS[name]:
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c)],
                   check=True)
    r = subprocess.run([sys.executable, "-c", _KCORE_RUNNER, str(so), root],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 or int(r.stdout.strip().splitlines()[-1]) > 0, name


# ---- Dijkstra mutants ---------------------------------------------------------------------

_DIJKSTRA_MUTANTS = {
    # the heap orders by the largest key (the comparison of a push reversed)
    "max_heap_push": [("if (h[p].key <= x.key) break;", "if (h[p].key >= x.key) break;")],
    # each edge takes the weight of the next edge in the array
    "shifted_weight": [("      uint64_t nd = d[u] + w[e];\n      if (nd < d[v]) {",
                        "      uint64_t nd = d[u] + w[e + 1 < m ? e + 1 : e];\n"
                        "      if (nd < d[v]) {")],
    # a vertex keeps the label of its first discovery (no decrease of a known distance)
    "first_label_only": [("      uint64_t nd = d[u] + w[e];\n      if (nd < d[v]) {",
                          "      uint64_t nd = d[u] + w[e];\n      if (d[v] == UINT64_MAX) {")],
}

_DIJKSTRA_RUNNER = r"""
import ctypes, sys, numpy as np
sys.path.insert(0, sys.argv[2])
import graphgen as gg
from tests.test_oracle_pins import _brute, _edges_of
L = ctypes.CDLL(sys.argv[1])
vp, u32 = ctypes.c_void_p, ctypes.c_uint32
L.or_dijkstra.argtypes = [u32, vp, vp, vp, u32, u32, vp]
bad = 0
for seed in range(40):
    g = gg.random_graph(7, 14, wlo=1, whi=20, seed=seed, self_loops=False)
    off = np.ascontiguousarray(g.offsets, np.uint64)
    nbr = np.ascontiguousarray(g.nbr, np.uint32)
    w = np.ascontiguousarray(g.w, np.uint32)
    out = np.empty(g.n, np.uint32)
    L.or_dijkstra(g.n, off.ctypes.data, nbr.ctypes.data, w.ctypes.data, 0, 0xFFFFFFFF,
                  out.ctypes.data)
    bad += out.tolist() != _brute(g.n, _edges_of(g), 0)
print(bad)
"""


@pytest.mark.parametrize("name", sorted(_DIJKSTRA_MUTANTS))
def test_dijkstra_pins_reject_planted_mistakes(gg, orc, tmp_path, name):
    """Each mutant of or_dijkstra (a patched copy of oracle.c) must disagree with the
    brute-force minimum over simple paths on some of 40 random graphs."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "oracle.c")).read()
    for old, new in _DIJKSTRA_MUTANTS[name]:
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c)],
                   check=True)
    r = subprocess.run([sys.executable, "-c", _DIJKSTRA_RUNNER, str(so), root],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 or int(r.stdout.strip().splitlines()[-1]) > 0, name


@pytest.mark.parametrize("runner", ["kcore", "dijkstra", "setcover"])
def test_mutant_runners_accept_the_unmodified_oracle(gg, orc, tmp_path, runner):
    """Control for the planted-mistake tests: the unmodified oracle, compiled the same way
    and run by the same runner, exits 0 and disagrees with nothing (so a mutant counts as
    caught only for what it changed, not for a broken runner)."""
    import os
    import subprocess
    import sys
    from tests import test_oracle_setcover as tsc
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = tmp_path / "libplain.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so),
                    os.path.join(root, "oracle", "oracle.c")], check=True)
    code = {"kcore": _KCORE_RUNNER, "dijkstra": _DIJKSTRA_RUNNER,
            "setcover": tsc._RUNNER}[runner]
    r = subprocess.run([sys.executable, "-c", code, str(so), root], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-500:]
    assert int(r.stdout.strip().splitlines()[-1]) == 0
