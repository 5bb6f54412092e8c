"""Pins for the oracle's approximate set cover (CPU only), against things other than
itself:

* hand-worked fixtures (tests/golden/setcover_hand.txt),
* closed forms on stars and cliques,
* invariance under relabelling the vertices and under disjoint union,
* per-step certificates of what the method guarantees (Section 6.1, "Approximate Set
  Cover": sets are taken from the highest bucket of cost per element, as a nearly
  independent subset): every set that joins covers at least max residual / (1 + eps)^2
  new elements, the sets of one step together cover at least that much each, and the
  cover is valid,
* the approximation bound (1 + eps)^2 * H(max |S|) * OPT against brute-force optima,
* mutants of the oracle's own source (a threshold off by one, buckets in the wrong
  order, a partial cover, a stale claim counted), which these pins must reject.
"""
import ctypes
import itertools
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.golden import fixtures

M = 10**6


def _graph(gg, n, pairs):
    return gg.from_edges(n, [u for u, v in pairs], [v for u, v in pairs], [1] * len(pairs))


def _sym_simple(gg, n, pairs):
    pairs = sorted({(min(u, v), max(u, v)) for u, v in pairs if u != v})
    return _graph(gg, n, pairs + [(v, u) for u, v in pairs])


def _sets(g):
    off = g.offsets.astype(np.int64)
    return [g.nbr[off[v]:off[v + 1]].tolist() for v in range(g.n)]


def _random_sym(gg, n, p, seed):
    rng = np.random.default_rng(seed)
    pairs = [(u, v) for u, v in itertools.combinations(range(n), 2) if rng.random() < p]
    return _sym_simple(gg, n, pairs)


def certify(g, step_out, steps, eps_ppm):
    """Replays the cover step by step from the join steps alone and checks what the
    method guarantees.  Returns a list of violations (empty = certified)."""
    S = _sets(g)
    n = g.n
    bad = []
    R = (M + eps_ppm) ** 2
    step_out = [int(x) for x in step_out]
    if any(s < 0 or s > steps for s in step_out):
        bad.append("step out of range")
    covered = [False] * n
    chosen = [False] * n
    by_step = {}
    for v, s in enumerate(step_out):
        if s:
            by_step.setdefault(s, []).append(v)
    for s in sorted(by_step):
        C = by_step[s]
        res = [sum(1 for u in S[v] if not covered[u]) if not chosen[v] else 0
               for v in range(n)]
        maxres = max(res)
        new = set()
        for v in C:
            if res[v] == 0:
                bad.append(f"set {v} joined at step {s} with nothing left to cover")
            if res[v] * R < maxres * M * M:
                bad.append(f"set {v} at step {s}: {res[v]} new vs max residual {maxres}")
            new.update(u for u in S[v] if not covered[u])
        if len(new) * R < len(C) * maxres * M * M:
            bad.append(f"step {s}: {len(C)} sets cover only {len(new)} new elements "
                       f"(max residual {maxres})")
        for v in C:
            chosen[v] = True
            for u in S[v]:
                covered[u] = True
    universe = {u for row in S for u in row}
    if any(not covered[u] for u in universe):
        bad.append("not a cover")
    return bad


def _opt(g):
    S = [set(r) for r in _sets(g)]
    universe = set().union(*S)
    cand = [v for v in range(g.n) if S[v]]
    for r in range(0, len(cand) + 1):
        for C in itertools.combinations(cand, r):
            if set().union(*(S[v] for v in C)) >= universe:
                return r
    return len(cand)


def test_golden_setcover_fixtures(gg, orc):
    fx = fixtures.load_setcover()
    assert len(fx) >= 6
    for f in fx:
        e = f["edges"]
        g = _graph(gg, f["n"], e)
        s, k = orc.setcover(g, np.array(f["pri"]), f["eps_ppm"])
        assert s.tolist() == f["expect"], f["name"]
        assert k == f["steps"], f["name"]


@pytest.mark.parametrize("k", range(1, 9))
def test_star_closed_form(gg, orc, k):
    """Star with centre 0 and leaves 1..k: the centre's set (all leaves) joins at step 1;
    the centre element is then covered by the leaf of smallest priority at step 2; the
    other leaves leave at step 3.  A single edge (k = 1): both sets join at step 1."""
    rng = np.random.default_rng(k)
    g = _sym_simple(gg, k + 1, [(0, i) for i in range(1, k + 1)])
    pri = rng.permutation(k + 1)
    s, steps = orc.setcover(g, pri)
    want = [0] * (k + 1)
    if k == 1:
        want = [1, 1]
        assert steps == 1
    else:
        want[0] = 1
        want[1 + int(np.argmin(pri[1:]))] = 2
        assert steps == 3
    assert s.tolist() == want


@pytest.mark.parametrize("k", range(3, 10))
def test_clique_closed_form(gg, orc, k):
    """Clique K_k (S_v = every vertex but v): the set of smallest priority v0 receives
    all k - 1 of its elements and joins at step 1; element v0 is then the only one left;
    the others move down (step 2) and the one of second smallest priority takes it at
    step 3; the rest leave at step 4."""
    rng = np.random.default_rng(100 + k)
    g = _sym_simple(gg, k, list(itertools.combinations(range(k), 2)))
    pri = rng.permutation(k)
    s, steps = orc.setcover(g, pri)
    order = np.argsort(pri)
    want = [0] * k
    want[int(order[0])] = 1
    want[int(order[1])] = 3
    assert s.tolist() == want and steps == 4


def test_no_edges_and_isolated_vertices(gg, orc):
    g = gg.from_edges(5, [], [], [])
    s, steps = orc.setcover(g, np.arange(5))
    assert s.tolist() == [0] * 5 and steps == 0
    g = _sym_simple(gg, 6, [(1, 2)])
    s, steps = orc.setcover(g, np.arange(6))
    assert s.tolist() == [0, 1, 1, 0, 0, 0] and steps == 1


@pytest.mark.parametrize("seed", range(8))
def test_relabelling_is_equivariant(gg, orc, seed):
    """Renaming the vertices (and carrying each set's priority with it) renames the
    result; the step numbers are unchanged."""
    g = _random_sym(gg, 40, 0.12, seed)
    rng = np.random.default_rng(seed)
    pri = rng.permutation(g.n)
    sig = rng.permutation(g.n)
    s, k = orc.setcover(g, pri)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    h = gg.from_edges(g.n, sig[src].tolist(), sig[g.nbr].tolist(), [1] * g.m)
    pri2 = np.empty_like(pri)
    pri2[sig] = pri
    s2, k2 = orc.setcover(h, pri2)
    assert k2 == k
    assert s2[sig].tolist() == s.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_disjoint_union_is_union_of_covers(gg, orc, seed):
    """Two components never compete for an element, so the sets chosen on their disjoint
    union are the sets chosen on each (step numbers differ: steps are global)."""
    a = _random_sym(gg, 30, 0.15, 2 * seed)
    b = _random_sym(gg, 25, 0.2, 2 * seed + 1)
    rng = np.random.default_rng(seed)
    pa, pb = rng.permutation(a.n), rng.permutation(b.n)
    sa, _ = orc.setcover(a, pa)
    sb, _ = orc.setcover(b, pb)
    ea = list(zip(np.repeat(np.arange(a.n), np.diff(a.offsets.astype(np.int64))).tolist(),
                  a.nbr.tolist()))
    eb = list(zip(np.repeat(np.arange(b.n), np.diff(b.offsets.astype(np.int64))).tolist(),
                  b.nbr.tolist()))
    u = _graph(gg, a.n + b.n, ea + [(x + a.n, y + a.n) for x, y in eb])
    # interleave the priorities; only their order inside each component matters
    pu = np.argsort(np.argsort(np.concatenate([2 * pa, 2 * pb + 1])))
    su, _ = orc.setcover(u, pu)
    assert ((su[:a.n] > 0) == (sa > 0)).all()
    assert ((su[a.n:] > 0) == (sb > 0)).all()


@pytest.mark.parametrize("eps_ppm", [0, 10000, 250000, 1000000])
@pytest.mark.parametrize("seed", range(10))
def test_certificates_on_random_graphs(gg, orc, eps_ppm, seed):
    n = 30 + 7 * seed
    g = _random_sym(gg, n, 0.04 + 0.02 * (seed % 5), seed)
    pri = np.random.default_rng(seed).permutation(n)
    s, k = orc.setcover(g, pri, eps_ppm)
    assert certify(g, s, k, eps_ppm) == []


@pytest.mark.parametrize("seed", range(6))
def test_certificates_on_rmat_and_grid(gg, orc, seed):
    g = gg.rmat(10, 8, 0.57, 0.19, 0.19, 1, 2, seed=seed) if seed % 2 == 0 else \
        gg.grid(20 + seed, 17, 1, 2, seed=seed)
    pri = np.random.default_rng(seed).permutation(g.n)
    for eps in (0, 10000):
        s, k = orc.setcover(g, pri, eps)
        assert certify(g, s, k, eps) == []


def test_eps_zero_takes_largest_residual_exactly(gg, orc):
    """eps = 0: every bucket is one residual size and a set joins only if it receives all
    of its elements, so each joining set covers exactly the largest residual, and the
    sets of one step cover disjoint new elements."""
    g = _random_sym(gg, 60, 0.08, 7)
    S = _sets(g)
    s, k = orc.setcover(g, np.random.default_rng(7).permutation(g.n), 0)
    covered, chosen = set(), set()
    for step in range(1, k + 1):
        C = [v for v in range(g.n) if s[v] == step]
        if not C:
            continue
        res = {v: len(set(S[v]) - covered) for v in range(g.n) if v not in chosen}
        mx = max(res.values())
        new = [set(S[v]) - covered for v in C]
        assert all(len(x) == mx for x in new)
        assert len(set().union(*new)) == sum(len(x) for x in new)
        for v in C:
            chosen.add(v)
            covered |= set(S[v])


@pytest.mark.parametrize("seed", range(16))
def test_approximation_bound_vs_brute_force(gg, orc, seed):
    n = 10
    g = _random_sym(gg, n, 0.2 + 0.03 * seed, 50 + seed)
    if g.m == 0:
        return
    S = _sets(g)
    H = sum(1.0 / i for i in range(1, max(len(r) for r in S) + 1))
    opt = _opt(g)
    for eps in (0, 10000, 1000000):
        s, _ = orc.setcover(g, np.random.default_rng(seed).permutation(n), eps)
        assert int((s > 0).sum()) <= (1 + eps / M) ** 2 * H * opt + 1e-9


def test_rejects_bad_priorities_and_eps(gg, orc):
    g = _sym_simple(gg, 4, [(0, 1), (1, 2)])
    with pytest.raises(orc.OracleError):
        orc.setcover(g, np.array([0, 1, 1, 3]))
    with pytest.raises(orc.OracleError):
        orc.setcover(g, np.array([0, 1, 2, 4]))
    with pytest.raises(orc.OracleError):
        orc.setcover(g, np.arange(4), 1000001)


# ---- mutants: plausible mistakes planted in a copy of the oracle's source ----------------

_MUTANTS = {
    # the join threshold one element too low
    "tau_minus_one": ("if (won >= tau) join[nj++] = v;", "if (won + 1 >= tau) join[nj++] = v;"),
    # buckets worked off from the lowest instead of the highest
    "ascending": ("for (uint32_t j = (uint32_t)nb; j-- > 0;) {\n    uint32_t cnt = 0;",
                  "for (uint32_t jj = 0; jj < (uint32_t)nb; ++jj) {\n"
                  "    uint32_t j = jj;\n    uint32_t cnt = 0;"),
    # a joining set covers only the elements it received
    "cover_won_only": ("for (uint64_t e = off[v]; e < off[v + 1]; ++e) cov[nbr[e]] = 1;",
                       "for (uint64_t e = off[v]; e < off[v + 1]; ++e)\n"
                       "          if (claim[nbr[e]] == pri[v]) cov[nbr[e]] = 1;"),
    # the received count also takes covered elements (stale claims of earlier steps)
    "won_counts_covered": ("won += (!cov[nbr[e]] && claim[nbr[e]] == pri[v]) ? 1 : 0;",
                           "won += (claim[nbr[e]] == pri[v]) ? 1 : 0;"),
}

_RUNNER = r"""
import ctypes, sys, numpy as np
sys.path.insert(0, sys.argv[2])
import graphgen as gg
from tests.test_oracle_setcover import certify, _random_sym, _graph
from tests.golden import fixtures
L = ctypes.CDLL(sys.argv[1])
vp, u32 = ctypes.c_void_p, ctypes.c_uint32
L.or_setcover.argtypes = [u32, vp, vp, u32, vp, vp, vp]
def run(g, pri, eps):
    off = np.ascontiguousarray(g.offsets, np.uint64)
    nbr = np.ascontiguousarray(g.nbr, np.uint32)
    pri = np.ascontiguousarray(pri, np.uint32)
    out = np.empty(g.n, np.uint32)
    k = ctypes.c_uint64(0)
    L.or_setcover(g.n, off.ctypes.data, nbr.ctypes.data, eps, pri.ctypes.data,
                  out.ctypes.data, ctypes.byref(k))
    return out, k.value
bad = 0
for f in fixtures.load_setcover():
    out, k = run(_graph(gg, f["n"], f["edges"]), f["pri"], f["eps_ppm"])
    bad += out.tolist() != f["expect"] or k != f["steps"]
for seed in range(12):
    g = _random_sym(gg, 40, 0.06 + 0.02 * (seed % 4), seed)
    for eps in (0, 10000, 250000, 1000000):
        out, k = run(g, np.random.default_rng(seed).permutation(g.n), eps)
        bad += bool(certify(g, out, k, eps))
print(bad)
"""


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_planted_mistakes(gg, orc, tmp_path, name):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) == 1, name
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c)],
                   check=True)
    try:
        r = subprocess.run([sys.executable, "-c", _RUNNER, str(so), root], capture_output=True,
                           text=True, timeout=60)
        caught = r.returncode != 0 or int(r.stdout.strip().splitlines()[-1]) > 0
    except subprocess.TimeoutExpired:
        caught = True  # the mutant never finishes: not a correct cover either
    assert caught, name


# ---- the fast certificate (or_check_setcover) against the replay above --------------------

def _perturb(s, rng):
    """A plausible wrong answer: a chosen set dropped, moved to another step, an unchosen
    set added to a step, or two sets' steps swapped."""
    s = s.copy()
    chosen = np.nonzero(s)[0]
    other = np.nonzero(s == 0)[0]
    k = int(s.max()) if s.size else 0
    kind = rng.integers(4)
    if kind == 0 and chosen.size:
        s[rng.choice(chosen)] = 0
    elif kind == 1 and chosen.size and k > 1:
        s[rng.choice(chosen)] = rng.integers(1, k + 1)
    elif kind == 2 and other.size and k:
        s[rng.choice(other)] = rng.integers(1, k + 1)
    elif chosen.size > 1:
        a, b = rng.choice(chosen, 2, replace=False)
        s[a], s[b] = s[b], s[a]
    return s


@pytest.mark.parametrize("eps", [0, 10000, 250000, 1000000])
def test_fast_certificate_agrees_with_the_replay(gg, orc, eps):
    """The O(n + m) certificate and the step-by-step replay check the same properties:
    both accept the oracle's covers, and they agree on every perturbed answer."""
    rng = np.random.default_rng(eps)
    rejected = 0
    for seed in range(12):
        g = _random_sym(gg, 30 + 5 * seed, 0.05 + 0.02 * (seed % 5), 100 + seed)
        pri = np.random.default_rng(seed).permutation(g.n)
        s, k = orc.setcover(g, pri, eps)
        assert orc.check_setcover(g, s, k, eps) == (0, 0)
        assert certify(g, s, k, eps) == []
        for _ in range(15):
            t = _perturb(s, rng)
            fast = orc.check_setcover(g, t, k, eps)[0] == 0
            slow = certify(g, t, k, eps) == []
            assert fast == slow, (seed, t.tolist())
            rejected += not fast
    assert rejected > 30


def test_fast_certificate_codes(gg, orc):
    g = _sym_simple(gg, 6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)])
    s, k = orc.setcover(g, np.arange(6), 10000)
    assert orc.check_setcover(g, s, k) == (0, 0)
    t = s.copy()
    t[:] = 0
    assert orc.check_setcover(g, t, k)[0] == 1        # nothing chosen: not a cover
    t = s.copy()
    t[0] = k + 1
    assert orc.check_setcover(g, t, k) == (4, 0)      # a step beyond the run
    star = _sym_simple(gg, 8, [(0, i) for i in range(1, 8)])
    s, k = orc.setcover(star, np.arange(8), 10000)
    t = s.copy()
    t[1:] = 1                                         # every leaf joins with the centre
    assert orc.check_setcover(star, t, k)[0] in (2, 3)
