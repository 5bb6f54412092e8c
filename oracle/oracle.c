/*
 * CPU oracle for shortest-path distances, k-core and set cover -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  The product path (paper_1911_07260_gb300) never calls it and shares no
 * code, header, table or helper with it.
 *
 * What it computes.  Delta-stepping with or without bucket fusion (Section 3, the
 * lazy / eager / eager-with-fusion figures) is a label-correcting method that stops only
 * when no bucket holds a vertex whose distance can still improve, so it reaches exactly
 * the shortest-path distances of the plain definition (Section 6.1, "SSSP and wBFS"):
 *     dist(v) = min over paths s -> v of the sum of edge weights, or "unreachable".
 * The oracle computes that definition directly:
 *   - or_dijkstra:      binary-heap Dijkstra with lazy deletion, 64-bit sums.  With a
 *                       target it stops once the target is popped (its value is final),
 *                       which is the PPSP / A* result (Section 6.1, "PPSP", "A* Search").
 *   - or_bfs:           hop counts (unit weights), the wBFS special case.
 *   - or_bellman_ford:  repeated relaxation of every edge until nothing changes; the
 *                       unordered method of Section 1, used as an independent check.
 *   - or_check_sssp:    certificate check: dist[src] = 0; for every edge u->v with u
 *                       reached, dist[v] <= dist[u] + w; every reached v != src has an
 *                       in-edge with equality; unreached vertices hold the sentinel.
 *                       With every weight >= 1 these conditions imply exactness.
 *   - or_kcore:         coreness of every vertex by the peeling procedure the paper
 *                       uses for k-core (Section 6.1, "k-core"): repeatedly take an
 *                       unextracted vertex of minimum priority (priority = degree at
 *                       the start), raise the level k to that priority if it is larger,
 *                       record coreness = k, and lower by one the priority of every
 *                       unextracted neighbour whose priority is above k (the constant
 *                       -1 sum update, floored at k).  Degrees and decrements count CSR
 *                       entries, so on a symmetric simple graph this is the usual
 *                       coreness; the minimum is taken with the binary heap above
 *                       (stale heap entries are skipped).
 *   - or_check_kcore:   certificate of a coreness vector c for or_kcore's peeling, in
 *                       O(n + m) (the heap makes or_kcore O(m log n)): (a) every v keeps
 *                       at least c(v) entries once every entry w -> v with c(w) < c(v)
 *                       is taken away, so no level below c(v) can extract v; (b) taking
 *                       the levels k in ascending order, after every vertex with
 *                       c < k is gone, repeatedly extracting a vertex with c = k that
 *                       has at most k entries left removes every vertex with c = k.
 *                       (a) and (b) hold together for or_kcore's output only: (b) makes
 *                       each level's closure take all of {c = k}, (a) keeps it from
 *                       taking anything else.  On a symmetric graph (a) reads "v has at
 *                       least c(v) neighbours u with c(u) >= c(v)", the definition of the
 *                       c(v)-core, and (b) shows v outside the (c(v) + 1)-core.
 *   - or_setcover:      approximate unweighted set cover (Section 6.1, "Approximate Set
 *                       Cover"), the graph read as a set system: the set of vertex v is
 *                       its adjacency list S_v (entries counted with multiplicity), the
 *                       universe is the union of the S_v, every set costs 1.  Sets are
 *                       bucketed by the number of their still uncovered elements on the
 *                       integer ladder t_0 = 1, t_(j+1) = t_j + max(1, floor(t_j * eps)),
 *                       eps = eps_ppm / 10^6 (bucket j: t_j <= D < t_(j+1)).  The highest
 *                       non-empty bucket j is worked off in steps; one step (1) recounts
 *                       D for each set of the bucket: D = 0 leaves, 0 < D < t_j moves to
 *                       the bucket of D, the rest are active; (2) gives each uncovered
 *                       element of an active set to the active set of smallest priority
 *                       that contains it; (3) lets every active set that received at
 *                       least tau_j = ceil(t_j / (1 + eps)) of its elements join the cover
 *                       (a nearly independent subset of the bucket) and cover all of its
 *                       elements; the other active sets stay in bucket j.  step_out[v] is
 *                       the 1-based step in which v joined, 0 if it never did.
 *                       Parity pinned by closed forms (star, clique), hand-worked paths,
 *                       invariance under relabelling and disjoint union, and per-step
 *                       certificates of the approximate greedy choice, the near
 *                       independence and the (1 + eps)^2 H(max |S|) approximation bound
 *                       against brute-force optima.
 *   - or_check_setcover: certificate of a set cover given as join steps: replays the
 *                       steps in order and checks that every set that joins covers at
 *                       least one and at least (largest residual) / (1 + eps)^2 new
 *                       elements, that the sets of one step together cover at least that
 *                       much each (they are nearly independent), and that the result
 *                       covers the universe -- what the method guarantees, whatever its
 *                       priorities.  Residuals are kept current through the reverse
 *                       adjacency and a count per residual size, so the check is
 *                       O(n + m + steps) rather than a rescan per step.
 *
 * Conventions.  Distances are uint32 with 0xFFFFFFFF = unreachable (the paper's INT_MAX
 * initialisation, Section 4.1).  A finite distance >= 0xFFFFFFFE cannot be represented;
 * the oracle then returns OR_OVERFLOW and stores 0xFFFFFFFE.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_OVERFLOW 1
#define OR_INVALID (-1)
#define OR_NOMEM (-2)

#define UNREACHED 0xFFFFFFFFu
#define SATURATED 0xFFFFFFFEu
#define NO_TARGET 0xFFFFFFFFu

typedef struct {
  uint64_t key;
  uint32_t v;
} heap_item;

/* Plain binary min-heap on key. */
static void heap_push(heap_item *h, uint64_t *size, heap_item x) {
  uint64_t i = (*size)++;
  while (i > 0) {
    uint64_t p = (i - 1) / 2;
    if (h[p].key <= x.key) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static heap_item heap_pop(heap_item *h, uint64_t *size) {
  heap_item top = h[0];
  heap_item last = h[--(*size)];
  uint64_t i = 0, n = *size;
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, s = i;
    uint64_t best_key = last.key;
    if (l < n && h[l].key < best_key) { s = l; best_key = h[l].key; }
    if (r < n && h[r].key < best_key) { s = r; }
    if (s == i) break;
    h[i] = h[s];
    i = s;
  }
  if (n > 0) h[i] = last;
  return top;
}

static int store_dist(uint32_t n, const uint64_t *d64, uint32_t *dist_out) {
  int st = OR_OK;
  for (uint32_t v = 0; v < n; ++v) {
    if (d64[v] == UINT64_MAX) dist_out[v] = UNREACHED;
    else if (d64[v] >= SATURATED) { dist_out[v] = SATURATED; st = OR_OVERFLOW; }
    else dist_out[v] = (uint32_t)d64[v];
  }
  return st;
}

/* Dijkstra from src.  target == 0xFFFFFFFF: all distances.  Otherwise stops when the
 * target is popped; dist_out[target] is then final (other entries are upper bounds). */
int or_dijkstra(uint32_t n, const uint64_t *off, const uint32_t *nbr, const uint32_t *w,
                uint32_t src, uint32_t target, uint32_t *dist_out) {
  if (n == 0 || src >= n || (target != NO_TARGET && target >= n)) return OR_INVALID;
  uint64_t m = off[n];
  uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * n);
  heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (m + 1));
  unsigned char *done = (unsigned char *)calloc(n, 1);
  if (!d || !h || !done) { free(d); free(h); free(done); return OR_NOMEM; }
  for (uint32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  uint64_t hs = 0;
  d[src] = 0;
  heap_item s0 = {0, src};
  heap_push(h, &hs, s0);
  while (hs > 0) {
    heap_item it = heap_pop(h, &hs);
    uint32_t u = it.v;
    if (done[u] || it.key != d[u]) continue; /* lazy deletion of stale heap entries */
    done[u] = 1;
    if (u == target) break;
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = nbr[e];
      uint64_t nd = d[u] + w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_item x = {nd, v};
        heap_push(h, &hs, x);
      }
    }
  }
  int st = store_dist(n, d, dist_out);
  free(d); free(h); free(done);
  return st;
}

/* Breadth-first hop counts from src (every edge counts 1). */
int or_bfs(uint32_t n, const uint64_t *off, const uint32_t *nbr, uint32_t src,
           uint32_t *dist_out) {
  if (n == 0 || src >= n) return OR_INVALID;
  uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * n);
  if (!q) return OR_NOMEM;
  for (uint32_t v = 0; v < n; ++v) dist_out[v] = UNREACHED;
  uint64_t head = 0, tail = 0;
  dist_out[src] = 0;
  q[tail++] = src;
  while (head < tail) {
    uint32_t u = q[head++];
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = nbr[e];
      if (dist_out[v] == UNREACHED) {
        dist_out[v] = dist_out[u] + 1;
        q[tail++] = v;
      }
    }
  }
  free(q);
  return OR_OK;
}

/* Bellman-Ford: relax every edge, repeat until a full pass changes nothing (at most
 * n passes with non-negative weights). */
int or_bellman_ford(uint32_t n, const uint64_t *off, const uint32_t *nbr,
                    const uint32_t *w, uint32_t src, uint32_t *dist_out) {
  if (n == 0 || src >= n) return OR_INVALID;
  uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * n);
  if (!d) return OR_NOMEM;
  for (uint32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  d[src] = 0;
  for (uint32_t pass = 0; pass < n; ++pass) {
    int changed = 0;
    for (uint32_t u = 0; u < n; ++u) {
      if (d[u] == UINT64_MAX) continue;
      for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
        uint64_t nd = d[u] + w[e];
        if (nd < d[nbr[e]]) { d[nbr[e]] = nd; changed = 1; }
      }
    }
    if (!changed) break;
  }
  int st = store_dist(n, d, dist_out);
  free(d);
  return st;
}

/* Certificate check of an SSSP result.  Returns 0 if valid, else a code and the first
 * offending vertex in *bad:
 *   1: dist[src] != 0            2: an edge u->v with dist[v] > dist[u] + w
 *   3: reached v != src without a tight in-edge
 *   4: a value equal to the saturation marker 0xFFFFFFFE                              */
int or_check_sssp(uint32_t n, const uint64_t *off, const uint32_t *nbr, const uint32_t *w,
                  uint32_t src, const uint32_t *dist, uint32_t *bad) {
  if (n == 0 || src >= n) return OR_INVALID;
  *bad = 0;
  if (dist[src] != 0) { *bad = src; return 1; }
  unsigned char *tight = (unsigned char *)calloc(n, 1);
  if (!tight) return OR_NOMEM;
  int code = 0;
  for (uint32_t u = 0; u < n && !code; ++u) {
    if (dist[u] == SATURATED) { *bad = u; code = 4; break; }
    if (dist[u] == UNREACHED) continue;
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = nbr[e];
      uint64_t cand = (uint64_t)dist[u] + w[e];
      uint64_t dv = dist[v] == UNREACHED ? UINT64_MAX : dist[v];
      if (dv > cand) { *bad = v; code = 2; break; }
      if (dv == cand) tight[v] = 1;
    }
  }
  for (uint32_t v = 0; v < n && !code; ++v)
    if (v != src && dist[v] != UNREACHED && !tight[v]) { *bad = v; code = 3; }
  free(tight);
  return code;
}

/* Coreness by peeling (see the header).  core_out: uint32[n]. */
int or_kcore(uint32_t n, const uint64_t *off, const uint32_t *nbr, uint32_t *core_out) {
  if (n == 0) return OR_INVALID;
  const uint64_t m = off[n];
  uint32_t *prio = (uint32_t *)malloc(sizeof(uint32_t) * n);
  unsigned char *done = (unsigned char *)calloc(n, 1);
  heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (n + m + 1));
  if (!prio || !done || !h) {
    free(prio);
    free(done);
    free(h);
    return OR_NOMEM;
  }
  uint64_t hs = 0;
  for (uint32_t v = 0; v < n; ++v) {
    prio[v] = (uint32_t)(off[v + 1] - off[v]);
    heap_item x = {prio[v], v};
    heap_push(h, &hs, x);
  }
  uint32_t k = 0;
  while (hs > 0) {
    heap_item t = heap_pop(h, &hs);
    uint32_t v = t.v;
    if (done[v] || t.key != prio[v]) continue; /* extracted, or an older priority */
    if (prio[v] > k) k = prio[v];
    done[v] = 1;
    core_out[v] = k;
    for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
      uint32_t w = nbr[e];
      if (done[w] || prio[w] <= k) continue;
      prio[w] -= 1;
      heap_item x = {prio[w], w};
      heap_push(h, &hs, x);
    }
  }
  free(prio);
  free(done);
  free(h);
  return OR_OK;
}

/* Certificate of a coreness vector (see the header): returns 0 when core[] is what
 * or_kcore computes, 1 when (a) fails at vertex *bad, 2 when (b) fails (*bad = a vertex
 * of the level that could not be extracted), OR_INVALID / OR_NOMEM otherwise. */
int or_check_kcore(uint32_t n, const uint64_t *off, const uint32_t *nbr, const uint32_t *core,
                   uint32_t *bad) {
  if (n == 0 || !core || !bad) return OR_INVALID;
  *bad = 0;
  const uint64_t m = off[n];
  for (uint64_t e = 0; e < m; ++e)
    if (nbr[e] >= n) return OR_INVALID;
  /* (a): entries w -> v with core[w] < core[v] (on a directed graph they may outnumber
   * v's own entries, so they are counted, not subtracted) */
  uint64_t *left = (uint64_t *)calloc(n, sizeof(uint64_t));
  if (!left) return OR_NOMEM;
  for (uint32_t w = 0; w < n; ++w)
    for (uint64_t e = off[w]; e < off[w + 1]; ++e)
      if (core[w] < core[nbr[e]]) left[nbr[e]] += 1;
  for (uint32_t v = 0; v < n; ++v) {
    if ((uint64_t)core[v] + left[v] > off[v + 1] - off[v]) {
      *bad = v;
      free(left);
      return 1;
    }
  }
  /* (b): levels in ascending order (vertices sorted by core[] with a counting sort; (a)
   * bounds every core[v] by v's degree, so the levels fit in m + 1 counters) */
  uint32_t maxc = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (core[v] > maxc) maxc = core[v];
  uint64_t *start = (uint64_t *)calloc((size_t)maxc + 2, sizeof(uint64_t));
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * n);
  unsigned char *state = (unsigned char *)calloc(n, 1); /* 1 queued, 2 extracted */
  if (!start || !order || !queue || !state) {
    free(left);
    free(start);
    free(order);
    free(queue);
    free(state);
    return OR_NOMEM;
  }
  for (uint32_t v = 0; v < n; ++v) start[core[v] + 1] += 1;
  for (uint32_t k = 0; k <= maxc; ++k) start[k + 1] += start[k];
  {
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)maxc + 1));
    if (!fill) {
      free(left);
      free(start);
      free(order);
      free(queue);
      free(state);
      return OR_NOMEM;
    }
    memcpy(fill, start, sizeof(uint64_t) * ((size_t)maxc + 1));
    for (uint32_t v = 0; v < n; ++v) order[fill[core[v]]++] = v;
    free(fill);
  }
  /* entries left to each vertex while the levels are extracted, floored at 0 (the
   * peeling floors a priority at the level, and "left <= k" is the same test) */
  for (uint32_t v = 0; v < n; ++v) left[v] = off[v + 1] - off[v];
  int code = 0;
  for (uint32_t k = 0; k <= maxc && code == 0; ++k) {
    uint64_t qh = 0, qt = 0;
    for (uint64_t i = start[k]; i < start[k + 1]; ++i) {
      const uint32_t v = order[i];
      if (left[v] <= k) {
        state[v] = 1;
        queue[qt++] = v;
      }
    }
    while (qh < qt) {
      const uint32_t v = queue[qh++];
      state[v] = 2;
      for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
        const uint32_t u = nbr[e];
        if (state[u] == 2) continue;
        if (left[u] > 0) left[u] -= 1;
        if (core[u] == k && state[u] == 0 && left[u] <= k) {
          state[u] = 1;
          queue[qt++] = u;
        }
      }
    }
    if (qt != start[k + 1] - start[k]) {
      for (uint64_t i = start[k]; i < start[k + 1]; ++i) {
        if (state[order[i]] != 2) {
          *bad = order[i];
          break;
        }
      }
      code = 2;
    }
  }
  free(left);
  free(start);
  free(order);
  free(queue);
  free(state);
  return code;
}

/* Bucket of a residual size d >= 1 on the ladder t[0 .. nb] (t[nb] > every size):
 * the largest j with t[j] <= d. */
static uint32_t sc_bucket(const uint64_t *t, uint32_t nb, uint64_t d) {
  uint32_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo + 1) / 2;
    if (t[mid] <= d) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

int or_setcover(uint32_t n, const uint64_t *off, const uint32_t *nbr, uint32_t eps_ppm,
                const uint32_t *pri, uint32_t *step_out, uint64_t *steps_out) {
  if (n == 0 || eps_ppm > 1000000u) return OR_INVALID;
  const uint64_t M = 1000000ull;
  /* priorities: a permutation of 0 .. n-1 */
  unsigned char *seen = (unsigned char *)calloc(n, 1);
  if (!seen) return OR_NOMEM;
  for (uint32_t v = 0; v < n; ++v) {
    if (pri[v] >= n || seen[pri[v]]) {
      free(seen);
      return OR_INVALID;
    }
    seen[pri[v]] = 1;
  }
  free(seen);
  uint64_t maxdeg = 0;
  for (uint32_t v = 0; v < n; ++v) {
    step_out[v] = 0;
    if (off[v + 1] - off[v] > maxdeg) maxdeg = off[v + 1] - off[v];
  }
  *steps_out = 0;
  if (maxdeg == 0) return OR_OK;
  /* the ladder, until it passes the largest set */
  uint64_t tcap = 64, nb = 0;
  uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * tcap);
  if (!t) return OR_NOMEM;
  t[0] = 1;
  while (t[nb] <= maxdeg) {
    uint64_t step = t[nb] * eps_ppm / M;
    if (step < 1) step = 1;
    if (nb + 2 > tcap) {
      tcap *= 2;
      uint64_t *t2 = (uint64_t *)realloc(t, sizeof(uint64_t) * tcap);
      if (!t2) {
        free(t);
        return OR_NOMEM;
      }
      t = t2;
    }
    t[nb + 1] = t[nb] + step;
    ++nb;
  }
  /* bucket lists as singly linked lists (a set is in one list at a time) */
  uint32_t *head = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  uint32_t *nxt = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *mem = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *act = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *join = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *claim = (uint32_t *)malloc(sizeof(uint32_t) * n);
  unsigned char *cov = (unsigned char *)calloc(n, 1);
  if (!head || !nxt || !mem || !act || !join || !claim || !cov) {
    free(t); free(head); free(nxt); free(mem); free(act); free(join); free(claim); free(cov);
    return OR_NOMEM;
  }
  for (uint64_t j = 0; j < nb; ++j) head[j] = UNREACHED;
  for (uint32_t v = n; v-- > 0;) {
    uint64_t d = off[v + 1] - off[v];
    if (d == 0) continue;
    uint32_t j = sc_bucket(t, (uint32_t)nb, d);
    nxt[v] = head[j];
    head[j] = v;
  }
  uint64_t step = 0;
  for (uint32_t j = (uint32_t)nb; j-- > 0;) {
    uint32_t cnt = 0;
    for (uint32_t v = head[j]; v != UNREACHED; v = nxt[v]) mem[cnt++] = v;
    head[j] = UNREACHED;
    const uint64_t tau = (t[j] * M + (M + eps_ppm) - 1) / (M + eps_ppm);
    while (cnt > 0) {
      ++step;
      /* (1) recount the uncovered elements of each set of the bucket */
      uint32_t na = 0;
      for (uint32_t i = 0; i < cnt; ++i) {
        uint32_t v = mem[i];
        uint64_t d = 0;
        for (uint64_t e = off[v]; e < off[v + 1]; ++e) d += cov[nbr[e]] ? 0 : 1;
        if (d == 0) continue;
        if (d < t[j]) {
          uint32_t jb = sc_bucket(t, (uint32_t)nb, d);
          nxt[v] = head[jb];
          head[jb] = v;
          continue;
        }
        act[na++] = v;
      }
      /* (2) each uncovered element goes to the smallest-priority active set holding it */
      for (uint32_t i = 0; i < na; ++i)
        for (uint64_t e = off[act[i]]; e < off[act[i] + 1]; ++e)
          if (!cov[nbr[e]]) claim[nbr[e]] = UNREACHED;
      for (uint32_t i = 0; i < na; ++i)
        for (uint64_t e = off[act[i]]; e < off[act[i] + 1]; ++e) {
          uint32_t u = nbr[e];
          if (!cov[u] && pri[act[i]] < claim[u]) claim[u] = pri[act[i]];
        }
      /* (3) sets that received at least tau of their elements join; the rest stay */
      uint32_t nj = 0, nl = 0;
      for (uint32_t i = 0; i < na; ++i) {
        uint32_t v = act[i];
        uint64_t won = 0;
        for (uint64_t e = off[v]; e < off[v + 1]; ++e)
          won += (!cov[nbr[e]] && claim[nbr[e]] == pri[v]) ? 1 : 0;
        if (won >= tau) join[nj++] = v;
        else mem[nl++] = v;
      }
      for (uint32_t i = 0; i < nj; ++i) {
        uint32_t v = join[i];
        step_out[v] = (uint32_t)step;
        for (uint64_t e = off[v]; e < off[v + 1]; ++e) cov[nbr[e]] = 1;
      }
      cnt = nl;
    }
  }
  *steps_out = step;
  free(t); free(head); free(nxt); free(mem); free(act); free(join); free(claim); free(cov);
  return OR_OK;
}

int or_check_setcover(uint32_t n, const uint64_t *off, const uint32_t *nbr, uint32_t eps_ppm,
                      const uint32_t *step_out, uint64_t steps, uint32_t *bad) {
  if (n == 0 || eps_ppm > 1000000u) return OR_INVALID;
  *bad = 0;
  const uint64_t m = off[n];
  for (uint32_t v = 0; v < n; ++v)
    if (step_out[v] > steps) { *bad = v; return 4; }
  uint64_t maxdeg = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (off[v + 1] - off[v] > maxdeg) maxdeg = off[v + 1] - off[v];
  /* reverse adjacency: the sets holding element u, one entry per occurrence */
  uint64_t *roff = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t *rset = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
  uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * n);
  uint64_t *res = (uint64_t *)malloc(sizeof(uint64_t) * n);
  uint64_t *cnt = (uint64_t *)calloc(maxdeg + 1, sizeof(uint64_t));
  uint64_t *soff = (uint64_t *)calloc(steps + 2, sizeof(uint64_t));
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n);
  unsigned char *cov = (unsigned char *)calloc(n, 1);
  unsigned char *chosen = (unsigned char *)calloc(n, 1);
  uint64_t *mark = (uint64_t *)calloc(n, sizeof(uint64_t));
  int rc = 0;
  if (!roff || !rset || !fill || !res || !cnt || !soff || !order || !cov || !chosen || !mark) {
    rc = OR_NOMEM;
    goto done;
  }
  for (uint64_t e = 0; e < m; ++e) roff[nbr[e] + 1]++;
  for (uint32_t u = 0; u < n; ++u) roff[u + 1] += roff[u];
  for (uint32_t u = 0; u < n; ++u) fill[u] = roff[u];
  for (uint32_t v = 0; v < n; ++v)
    for (uint64_t e = off[v]; e < off[v + 1]; ++e) rset[fill[nbr[e]]++] = v;
  /* residual = uncovered entries of each set not chosen yet; cnt[r] = such sets */
  for (uint32_t v = 0; v < n; ++v) {
    res[v] = off[v + 1] - off[v];
    cnt[res[v]]++;
  }
  uint64_t top = maxdeg;
  /* the sets of each step, in step order */
  for (uint32_t v = 0; v < n; ++v) soff[step_out[v] + 1]++;
  for (uint64_t s = 0; s <= steps; ++s) soff[s + 1] += soff[s];
  for (uint32_t v = 0; v < n; ++v) fill[v] = 0;
  {
    uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * (steps + 1));
    if (!pos) { rc = OR_NOMEM; goto done; }
    for (uint64_t s = 0; s <= steps; ++s) pos[s] = soff[s];
    for (uint32_t v = 0; v < n; ++v) order[pos[step_out[v]]++] = v;
    free(pos);
  }
  const unsigned __int128 R = (unsigned __int128)(1000000ull + eps_ppm) * (1000000ull + eps_ppm);
  const unsigned __int128 MM = (unsigned __int128)1000000ull * 1000000ull;
  for (uint64_t s = 1; s <= steps; ++s) {
    const uint64_t b = soff[s], e_ = soff[s + 1];
    if (b == e_) continue;
    while (top > 0 && cnt[top] == 0) --top;
    const uint64_t maxres = top;
    uint64_t fresh = 0;
    for (uint64_t i = b; i < e_; ++i) {
      const uint32_t v = order[i];
      if (res[v] == 0 || (unsigned __int128)res[v] * R < (unsigned __int128)maxres * MM) {
        *bad = v;
        rc = 2;
        goto done;
      }
      for (uint64_t k = off[v]; k < off[v + 1]; ++k) {
        const uint32_t u = nbr[k];
        if (!cov[u] && mark[u] != s) {
          mark[u] = s;
          ++fresh;
        }
      }
    }
    if ((unsigned __int128)fresh * R <
        (unsigned __int128)(e_ - b) * (unsigned __int128)maxres * MM) {
      *bad = (uint32_t)s;
      rc = 3;
      goto done;
    }
    /* apply the step: the chosen sets leave, their new elements are covered */
    for (uint64_t i = b; i < e_; ++i) {
      const uint32_t v = order[i];
      cnt[res[v]]--;
      chosen[v] = 1;
    }
    for (uint64_t i = b; i < e_; ++i) {
      const uint32_t v = order[i];
      for (uint64_t k = off[v]; k < off[v + 1]; ++k) {
        const uint32_t u = nbr[k];
        if (cov[u]) continue;
        cov[u] = 1;
        for (uint64_t r = roff[u]; r < roff[u + 1]; ++r) {
          const uint32_t w = rset[r];
          if (chosen[w]) continue;
          cnt[res[w]]--;
          res[w]--;
          cnt[res[w]]++;
        }
      }
    }
  }
  for (uint32_t u = 0; u < n; ++u)
    if (roff[u + 1] > roff[u] && !cov[u]) { *bad = u; rc = 1; goto done; }
done:
  free(roff); free(rset); free(fill); free(res); free(cnt); free(soff); free(order);
  free(cov); free(chosen); free(mark);
  return rc;
}
