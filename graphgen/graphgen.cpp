// Seeded synthetic graph generators (host C++17).
//
// These build the inputs that both the CPU oracle and the CUDA path consume.  They hold
// none of the shortest-path arithmetic: they only lay out vertices, edges, weights and
// coordinates.  Every random draw comes from a counter-based hash (SplitMix64's
// finalizer, Steele/Lea/Flood 2014) keyed by (seed, stream, counter), so the output is
// the same on every machine, for any thread count.  Built with -ffp-contract=off so the
// few floating-point steps (road weights) round identically on x86 and Arm.
//
// Graph families (weights are per undirected edge and equal in both directions):
//   grid  : rows x cols 4-neighbour grid, integer weights uniform in [wlo, whi).
//   road  : side x side grid, each grid edge dropped with probability drop_p, one
//           diagonal per unit cell with probability diag_p (orientation by coin), the
//           largest connected component kept and relabelled in row-major order;
//           weight = max(round(100 * len * U), ceil(100 * len)) with U ~ U[1, 1.5).
//   rmat  : R-MAT (a, b, c, d) with 2^scale vertices and edgefactor * 2^scale samples,
//           ids permuted by a seeded shuffle, self-loops and duplicates dropped,
//           symmetrised; integer weights uniform in [wlo, whi).
// Output is CSR with every adjacency list sorted by neighbour id.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

namespace {

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return mix64(mix64(seed * 0x9E3779B97F4A7C15ULL + stream) + ctr * 0xD1B54A32D192ED03ULL);
}
inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
inline uint32_t uint_in(uint64_t x, uint32_t lo, uint32_t hi) {  // [lo, hi)
  return lo + (uint32_t)(((x >> 32) * (uint64_t)(hi - lo)) >> 32);
}

enum : uint64_t {
  S_DROP = 1, S_DIAG = 2, S_ORIENT = 3, S_WGRID = 4, S_WDIAG = 5,
  S_RMAT = 6, S_PERM = 7, S_WRMAT = 8,
};

struct Graph {
  uint32_t n = 0;
  uint64_t m = 0;
  std::vector<uint64_t> off;
  std::vector<uint32_t> nbr, w;
  std::vector<float> xy;          // 2n or empty
  std::vector<int32_t> grid2id;   // side*side or empty (road / grid only)
  uint32_t side_r = 0, side_c = 0;
};

int nthreads_default() {
  unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 1 : (int)std::min(h, 64u);
}

template <class F>
void parallel_for(uint64_t n, int nt, F f) {
  if (nt <= 1 || n < 4096) { f(0, n); return; }
  std::vector<std::thread> th;
  uint64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    uint64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([=] { f(b, e); });
  }
  for (auto& x : th) x.join();
}

// Builds symmetric CSR from an undirected edge list (u, v, w); u != v assumed.
// Adjacency lists sorted by neighbour id; duplicate (u, v) pairs must already be absent.
void csr_from_undirected(Graph& g, uint32_t n, const std::vector<uint32_t>& eu,
                         const std::vector<uint32_t>& ev, const std::vector<uint32_t>& ew,
                         int nt) {
  g.n = n;
  g.off.assign((size_t)n + 1, 0);
  const size_t E = eu.size();
  for (size_t i = 0; i < E; ++i) { g.off[eu[i] + 1]++; g.off[ev[i] + 1]++; }
  for (uint32_t i = 0; i < n; ++i) g.off[i + 1] += g.off[i];
  g.m = g.off[n];
  g.nbr.resize(g.m);
  g.w.resize(g.m);
  std::vector<uint64_t> pos(g.off.begin(), g.off.end() - 1);
  for (size_t i = 0; i < E; ++i) {
    uint64_t p = pos[eu[i]]++;
    g.nbr[p] = ev[i]; g.w[p] = ew[i];
    p = pos[ev[i]]++;
    g.nbr[p] = eu[i]; g.w[p] = ew[i];
  }
  parallel_for(n, nt, [&](uint64_t b, uint64_t e) {
    std::vector<std::pair<uint32_t, uint32_t>> tmp;
    for (uint64_t v = b; v < e; ++v) {
      uint64_t lo = g.off[v], hi = g.off[v + 1];
      tmp.clear();
      for (uint64_t k = lo; k < hi; ++k) tmp.emplace_back(g.nbr[k], g.w[k]);
      std::sort(tmp.begin(), tmp.end());
      for (uint64_t k = lo; k < hi; ++k) { g.nbr[k] = tmp[k - lo].first; g.w[k] = tmp[k - lo].second; }
    }
  });
}

struct DSU {
  std::vector<uint32_t> p, sz;
  explicit DSU(uint32_t n) : p(n), sz(n, 1) { std::iota(p.begin(), p.end(), 0u); }
  uint32_t find(uint32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void unite(uint32_t a, uint32_t b) {
    a = find(a); b = find(b);
    if (a == b) return;
    if (sz[a] < sz[b] || (sz[a] == sz[b] && a > b)) std::swap(a, b);
    p[b] = a; sz[a] += sz[b];
  }
};

inline uint32_t road_weight(double len, double U) {
  double x = 100.0 * len * U;
  uint32_t r = (uint32_t)std::floor(x + 0.5);
  uint32_t c = (uint32_t)std::ceil(100.0 * len);
  return r > c ? r : c;
}

}  // namespace

extern "C" {

typedef struct Graph gg_graph;

uint32_t gg_n(const gg_graph* g) { return g->n; }
uint64_t gg_m(const gg_graph* g) { return g->m; }
int gg_has_xy(const gg_graph* g) { return g->xy.empty() ? 0 : 1; }
uint32_t gg_side_rows(const gg_graph* g) { return g->side_r; }
uint32_t gg_side_cols(const gg_graph* g) { return g->side_c; }

// Copies the CSR (and coordinates / grid map when present) into caller buffers.
void gg_copy(const gg_graph* g, uint64_t* off, uint32_t* nbr, uint32_t* w, float* xy,
             int32_t* grid2id) {
  if (off) std::memcpy(off, g->off.data(), g->off.size() * sizeof(uint64_t));
  if (nbr && g->m) std::memcpy(nbr, g->nbr.data(), g->m * sizeof(uint32_t));
  if (w && g->m) std::memcpy(w, g->w.data(), g->m * sizeof(uint32_t));
  if (xy && !g->xy.empty()) std::memcpy(xy, g->xy.data(), g->xy.size() * sizeof(float));
  if (grid2id && !g->grid2id.empty())
    std::memcpy(grid2id, g->grid2id.data(), g->grid2id.size() * sizeof(int32_t));
}

void gg_free(gg_graph* g) { delete g; }

// rows x cols 4-neighbour grid; weight uniform integer in [wlo, whi) per undirected edge.
gg_graph* gg_grid(uint32_t rows, uint32_t cols, uint32_t wlo, uint32_t whi, uint64_t seed) {
  if (rows == 0 || cols == 0 || whi <= wlo) return nullptr;
  Graph* g = new Graph();
  const uint32_t n = rows * cols;
  std::vector<uint32_t> eu, ev, ew;
  const uint64_t nh = (uint64_t)rows * (cols - 1);
  for (uint32_t r = 0; r < rows; ++r)
    for (uint32_t c = 0; c + 1 < cols; ++c) {
      uint64_t e = (uint64_t)r * (cols - 1) + c;
      eu.push_back(r * cols + c); ev.push_back(r * cols + c + 1);
      ew.push_back(uint_in(rnd(seed, S_WGRID, e), wlo, whi));
    }
  for (uint32_t r = 0; r + 1 < rows; ++r)
    for (uint32_t c = 0; c < cols; ++c) {
      uint64_t e = nh + (uint64_t)r * cols + c;
      eu.push_back(r * cols + c); ev.push_back((r + 1) * cols + c);
      ew.push_back(uint_in(rnd(seed, S_WGRID, e), wlo, whi));
    }
  csr_from_undirected(*g, n, eu, ev, ew, nthreads_default());
  g->xy.resize(2 * (size_t)n);
  g->grid2id.resize(n);
  for (uint32_t v = 0; v < n; ++v) {
    g->xy[2 * (size_t)v] = (float)(v % cols);
    g->xy[2 * (size_t)v + 1] = (float)(v / cols);
    g->grid2id[v] = (int32_t)v;
  }
  g->side_r = rows; g->side_c = cols;
  return g;
}

// Road-like grid (see file comment).
gg_graph* gg_road(uint32_t side, double drop_p, double diag_p, uint64_t seed) {
  if (side < 2) return nullptr;
  const int nt = nthreads_default();
  const uint64_t N0 = (uint64_t)side * side;
  if (N0 >= (1ull << 32)) return nullptr;
  const uint64_t nh = (uint64_t)side * (side - 1);  // horizontal edges; vertical the same
  const uint64_t ncell = (uint64_t)(side - 1) * (side - 1);
  const double sqrt2 = std::sqrt(2.0);

  // Keep flags for 2*nh grid edges and presence for ncell diagonals (parallel, hashed).
  std::vector<uint8_t> keep(2 * nh), dpres(ncell);
  parallel_for(2 * nh, nt, [&](uint64_t b, uint64_t e) {
    for (uint64_t i = b; i < e; ++i) keep[i] = u01(rnd(seed, S_DROP, i)) >= drop_p;
  });
  parallel_for(ncell, nt, [&](uint64_t b, uint64_t e) {
    for (uint64_t i = b; i < e; ++i) dpres[i] = u01(rnd(seed, S_DIAG, i)) < diag_p;
  });

  auto edge_ends = [&](uint64_t i, uint32_t& a, uint32_t& b) {
    if (i < nh) {  // horizontal: index r*(side-1)+c
      uint64_t r = i / (side - 1), c = i % (side - 1);
      a = (uint32_t)(r * side + c); b = a + 1;
    } else {       // vertical: index nh + r*side + c
      uint64_t j = i - nh, r = j / side, c = j % side;
      a = (uint32_t)(r * side + c); b = a + side;
    }
  };
  auto diag_ends = [&](uint64_t k, uint32_t& a, uint32_t& b) {
    uint64_t r = k / (side - 1), c = k % (side - 1);
    if ((rnd(seed, S_ORIENT, k) & 1) == 0) { a = (uint32_t)(r * side + c); b = a + side + 1; }
    else { a = (uint32_t)(r * side + c + 1); b = a + side - 1; }
  };

  DSU dsu((uint32_t)N0);
  for (uint64_t i = 0; i < 2 * nh; ++i)
    if (keep[i]) { uint32_t a, b; edge_ends(i, a, b); dsu.unite(a, b); }
  for (uint64_t k = 0; k < ncell; ++k)
    if (dpres[k]) { uint32_t a, b; diag_ends(k, a, b); dsu.unite(a, b); }

  // Largest component; ties broken by smallest root id.
  uint32_t best = 0, bestsz = 0;
  for (uint64_t v = 0; v < N0; ++v) {
    uint32_t r = dsu.find((uint32_t)v);
    if (r == v && (dsu.sz[r] > bestsz)) { best = r; bestsz = dsu.sz[r]; }
  }
  Graph* g = new Graph();
  g->grid2id.assign(N0, -1);
  uint32_t n = 0;
  for (uint64_t v = 0; v < N0; ++v)
    if (dsu.find((uint32_t)v) == best) g->grid2id[v] = (int32_t)n++;

  std::vector<uint32_t> eu, ev, ew;
  eu.reserve(2 * nh); ev.reserve(2 * nh); ew.reserve(2 * nh);
  for (uint64_t i = 0; i < 2 * nh; ++i) {
    if (!keep[i]) continue;
    uint32_t a, b; edge_ends(i, a, b);
    if (g->grid2id[a] < 0) continue;  // both ends share a component
    double U = 1.0 + 0.5 * u01(rnd(seed, S_WGRID, i));
    eu.push_back((uint32_t)g->grid2id[a]); ev.push_back((uint32_t)g->grid2id[b]);
    ew.push_back(road_weight(1.0, U));
  }
  for (uint64_t k = 0; k < ncell; ++k) {
    if (!dpres[k]) continue;
    uint32_t a, b; diag_ends(k, a, b);
    if (g->grid2id[a] < 0) continue;
    double U = 1.0 + 0.5 * u01(rnd(seed, S_WDIAG, k));
    eu.push_back((uint32_t)g->grid2id[a]); ev.push_back((uint32_t)g->grid2id[b]);
    ew.push_back(road_weight(sqrt2, U));
  }
  keep.clear(); keep.shrink_to_fit(); dpres.clear(); dpres.shrink_to_fit();
  csr_from_undirected(*g, n, eu, ev, ew, nt);
  g->xy.resize(2 * (size_t)n);
  for (uint64_t v = 0; v < N0; ++v) {
    int32_t id = g->grid2id[v];
    if (id < 0) continue;
    g->xy[2 * (size_t)id] = (float)(v % side);
    g->xy[2 * (size_t)id + 1] = (float)(v / side);
  }
  g->side_r = side; g->side_c = side;
  return g;
}

// R-MAT (see file comment).  d = 1 - a - b - c.
gg_graph* gg_rmat(uint32_t scale, uint32_t edgefactor, double a, double b, double c,
                  uint32_t wlo, uint32_t whi, uint64_t seed) {
  if (scale == 0 || scale > 30 || whi <= wlo) return nullptr;
  const int nt = nthreads_default();
  const uint32_t N = 1u << scale;
  const uint64_t M = (uint64_t)edgefactor * N;
  std::vector<uint32_t> su(M), sv(M);
  const double ab = a + b, abc = a + b + c;
  parallel_for(M, nt, [&](uint64_t lo, uint64_t hi) {
    for (uint64_t i = lo; i < hi; ++i) {
      uint32_t u = 0, v = 0;
      uint64_t x = 0;
      for (uint32_t lvl = 0; lvl < scale; ++lvl) {
        if ((lvl & 1) == 0) x = rnd(seed, S_RMAT, i * 16 + lvl / 2);
        uint32_t half = (lvl & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
        double p = (double)half * (1.0 / 4294967296.0);
        uint32_t ub, vb;
        if (p < a) { ub = 0; vb = 0; }
        else if (p < ab) { ub = 0; vb = 1; }
        else if (p < abc) { ub = 1; vb = 0; }
        else { ub = 1; vb = 1; }
        u = (u << 1) | ub; v = (v << 1) | vb;
      }
      su[i] = u; sv[i] = v;
    }
  });
  // Seeded Fisher-Yates shuffle of vertex ids.
  std::vector<uint32_t> perm(N);
  std::iota(perm.begin(), perm.end(), 0u);
  for (uint32_t i = N - 1; i > 0; --i) {
    uint32_t j = (uint32_t)(rnd(seed, S_PERM, i) % ((uint64_t)i + 1));
    std::swap(perm[i], perm[j]);
  }
  parallel_for(M, nt, [&](uint64_t lo, uint64_t hi) {
    for (uint64_t i = lo; i < hi; ++i) { su[i] = perm[su[i]]; sv[i] = perm[sv[i]]; }
  });
  perm.clear(); perm.shrink_to_fit();

  // Symmetric adjacency with duplicates, then per-vertex sort + unique.
  Graph* g = new Graph();
  g->n = N;
  std::vector<uint64_t> cnt((size_t)N + 1, 0);
  for (uint64_t i = 0; i < M; ++i)
    if (su[i] != sv[i]) { cnt[su[i] + 1]++; cnt[sv[i] + 1]++; }
  for (uint32_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  std::vector<uint32_t> adj(cnt[N]);
  {
    std::vector<uint64_t> pos(cnt.begin(), cnt.end() - 1);
    for (uint64_t i = 0; i < M; ++i) {
      uint32_t u = su[i], v = sv[i];
      if (u == v) continue;
      adj[pos[u]++] = v; adj[pos[v]++] = u;
    }
  }
  su.clear(); su.shrink_to_fit(); sv.clear(); sv.shrink_to_fit();
  std::vector<uint64_t> deg(N, 0);
  parallel_for(N, nt, [&](uint64_t lo, uint64_t hi) {
    for (uint64_t v = lo; v < hi; ++v) {
      uint32_t* p = adj.data() + cnt[v];
      uint64_t len = cnt[v + 1] - cnt[v];
      std::sort(p, p + len);
      deg[v] = (uint64_t)(std::unique(p, p + len) - p);
    }
  });
  g->off.assign((size_t)N + 1, 0);
  for (uint32_t v = 0; v < N; ++v) g->off[v + 1] = g->off[v] + deg[v];
  g->m = g->off[N];
  g->nbr.resize(g->m);
  g->w.resize(g->m);
  parallel_for(N, nt, [&](uint64_t lo, uint64_t hi) {
    for (uint64_t v = lo; v < hi; ++v) {
      const uint32_t* p = adj.data() + cnt[v];
      uint64_t o = g->off[v];
      for (uint64_t k = 0; k < deg[v]; ++k) {
        uint32_t x = p[k];
        uint64_t lo32 = v < x ? v : x, hi32 = v < x ? x : v;
        g->nbr[o + k] = x;
        g->w[o + k] = uint_in(rnd(seed, S_WRMAT, (lo32 << 32) | hi32), wlo, whi);
      }
    }
  });
  return g;
}

}  // extern "C"

extern "C" {
// New weights for an existing CSR: uniform in [wlo, whi), drawn from the unordered
// endpoint pair so that both directions of a symmetric edge get the same weight.
void gg_reweight(uint32_t n, const uint64_t* off, const uint32_t* nbr, uint32_t* w_out,
                 uint32_t wlo, uint32_t whi, uint64_t seed) {
  parallel_for(n, nthreads_default(), [&](uint64_t lo, uint64_t hi) {
    for (uint64_t v = lo; v < hi; ++v)
      for (uint64_t k = off[v]; k < off[v + 1]; ++k) {
        uint64_t x = nbr[k];
        uint64_t a = v < x ? v : x, b = v < x ? x : v;
        w_out[k] = uint_in(rnd(seed, S_WRMAT, (a << 32) | b), wlo, whi);
      }
  });
}
}  // extern "C"
