// Device side of k-core decomposition by peeling (Section 6.1, "k-core"), with the two
// bucket-update strategies the paper compares (Section 6.4, the table comparing
// eager and lazy bucket updates):
//   * lazy with the constant-sum (histogram) reduction of Section 5.1: a round extracts
//     the frontier (every vertex whose priority equals the level k) and only counts, per
//     neighbour w with priority above k, how many extracted vertices it lost; a second
//     phase then applies each count once -- priority = max(priority - count, k) -- and
//     makes one bucket insertion per counted vertex;
//   * eager (Section 3.2): every edge lowers the neighbour's priority by one with a
//     compare-and-swap floored at k and inserts the vertex into its new bucket at once.
// Buckets follow the lazy priority queue of Section 5.1: a window of kKRing materialised
// buckets [base, base + kKRing); vertices above the window are not stored and are found
// by a scan over all priorities when the window runs dry; vertices that drop to the
// current level go to a per-level frontier list.  A bucket that ran out of space is
// marked and its level is rebuilt by a scan (priority == k) instead.
// One cooperative persistent launch; phases are separated by a bounded grid barrier whose
// last arriver decides the next phase (kdecide).  The final priorities are the coreness.
#include <stddef.h>

#include "og_device.cuh"

#include "og_kcore.cuh"

namespace og {

namespace {

constexpr int kKBatch = 4;  // edges per thread per batch

struct KSmem {
  uint32_t phase, err, last, grab;
  uint32_t k, base, cur, fr_list, fsel, fr_n, asel, tsel;
  uint32_t lb_pos[kBlock + 1];  // edge prefix sums of a sub-tile's entries
  uint32_t lb_beg[kBlock];
  uint32_t wtmp[kWarps + 1];
  unsigned long long t_bar, t_peel, t_apply, t_hub;  // per-CTA phase time (thread 0)
};

struct KCnt {
  uint32_t items, stale, relax, improved, inserts;
};

// Warp-aggregated append of v (lanes with ok) to list[0 .. cap) through counter *n.
// Returns false on the lanes whose slot fell beyond cap.  All 32 lanes must call it.
__device__ __forceinline__ bool warp_append(uint32_t* list, uint32_t* n, uint32_t cap, bool ok,
                                            uint32_t v) {
  const unsigned m = __ballot_sync(FULL, ok);
  if (m == 0u) return true;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(n, (uint32_t)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (!ok) return true;
  const uint32_t pos = base + __popc(m & lanemask_lt());
  if (pos >= cap) return false;
  list[pos] = v;
  return true;
}

// Append of v to window bucket b (lanes with ok); lanes with the same bucket share one
// atomicAdd.  A bucket out of space is marked lossy.  All 32 lanes must call it.
__device__ __forceinline__ void ring_insert(const KParams& P, bool ok, uint32_t b, uint32_t v) {
  const unsigned m = __ballot_sync(FULL, ok);
  if (m == 0u || !ok) return;
  const unsigned peers = __match_any_sync(m, b);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(P.counts + b, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const uint32_t pos = base + __popc(peers & lanemask_lt());
  if (pos < P.cap) P.ring[(size_t)b * P.cap + pos] = v;
  else P.lossy[b] = 1u;
}

// A vertex whose priority just became np: the current level's next frontier if np == k,
// its window bucket if np is inside the window, else nothing (a later window refill finds
// it).  All 32 lanes must call it.
__device__ __forceinline__ void insert_prio(const KParams& P, const KSmem& S, KCnt& C, bool ok,
                                            uint32_t v, uint32_t np) {
  const bool to_list = ok && np == S.k;
  const bool to_ring = ok && np != S.k && np - S.base < kKRing;
  C.inserts += (to_list || to_ring) ? 1u : 0u;
  if (!warp_append(P.list[S.asel], &P.ks->next_n[S.asel], P.n, to_list, v))
    report_bad(P.sync, 32u, v, np);
  ring_insert(P, to_ring, np - S.base, v);
}

// Exclusive scan of a[0 .. kBlock) in place, a[kBlock] = total.  All threads call it.
__device__ __forceinline__ void kscan(uint32_t* a, uint32_t* wtmp) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t x = a[tid];
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  if (lane == 31) wtmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < (uint32_t)kWarps ? wtmp[lane] : 0u;
    uint32_t ws = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, ws, o);
      if ((int)lane >= o) ws += t;
    }
    if (lane < (uint32_t)kWarps) wtmp[lane] = ws - s;
    if (lane == kWarps - 1) wtmp[kWarps] = ws;
  }
  __syncthreads();
  a[tid] = wtmp[warp] + incl - x;
  if (tid == 0) a[kBlock] = wtmp[kWarps];
  __syncthreads();
}

// Applies the removal of level-k vertices to a batch of their out-neighbours w (lanes
// with ok).  Lazy: each neighbour with a priority above k gets one count (the first
// count lists it as touched).  Eager: the neighbour's priority is lowered by one
// (compare-and-swap, floored at k) and the vertex goes to its new bucket.  All 32 lanes
// must call it.
__device__ __forceinline__ void update_batch(const KParams& P, const KSmem& S, KCnt& C,
                                             const bool (&ok)[kKBatch],
                                             const uint32_t (&w)[kKBatch]) {
  const uint32_t k = S.k;
  uint32_t p[kKBatch];
#pragma unroll
  for (int b = 0; b < kKBatch; ++b) p[b] = ok[b] ? __ldcg(P.prio + w[b]) : 0u;
  if (!P.eager) {
    bool first[kKBatch];
#pragma unroll
    for (int b = 0; b < kKBatch; ++b) {
      const bool hit = ok[b] && p[b] > k;
      first[b] = hit && atomicAdd(P.cnt + w[b], 1u) == 0u;
      C.relax += ok[b] ? 1u : 0u;
    }
#pragma unroll
    for (int b = 0; b < kKBatch; ++b)
      if (!warp_append(P.touched[S.tsel], &P.ks->touched_n[S.tsel], P.n, first[b], w[b]))
        report_bad(P.sync, 33u, w[b], 0u);
  } else {
#pragma unroll
    for (int b = 0; b < kKBatch; ++b) {
      // Each failed compare-and-swap means another thread lowered the priority, so the
      // loop runs at most p - k times.
      uint32_t c = p[b], np = 0;
      bool dec = false;
      while (ok[b] && c > k) {
        const uint32_t prev = atomicCAS(P.prio + w[b], c, c - 1u);
        if (prev == c) {
          dec = true;
          np = c - 1u;
          break;
        }
        c = prev;
      }
      C.relax += ok[b] ? 1u : 0u;
      C.improved += dec ? 1u : 0u;
      insert_prio(P, S, C, dec, w[b], np);
    }
  }
}

// Lists a frontier vertex of out-degree >= hub_min for the hub phase: one 64-bit
// atomicAdd reserves its slot (high word) and its range of kBigChunk-edge chunks (low
// word); the chunk map names the slot of each chunk.  False when the list or the map is
// full (the caller then expands the vertex itself).
__device__ __noinline__ bool push_khub(const KParams& P, uint32_t u, uint32_t beg, uint32_t end) {
  const uint32_t nch = (end - beg + kBigChunk - 1) / kBigChunk;
  const unsigned long long x = atomicAdd(&P.ks->hub_word, (1ull << 32) | nch);
  const uint32_t slot = (uint32_t)(x >> 32), cbase = (uint32_t)x;
  const bool fits = slot < P.hub_cap && cbase <= P.map_cap && nch <= P.map_cap - cbase;
  if (fits) {
    BigItem it;
    it.u = u;
    it.g = 0;
    it.q = 0;
    it.beg = beg;
    it.end = end;
    it.cbase = cbase;
    P.hub[slot] = it;
  }
  const uint32_t lim = cbase < P.map_cap ? min(P.map_cap - cbase, nch) : 0u;
  for (uint32_t c = 0; c < lim; ++c) P.hub_map[cbase + c] = fits ? slot : kNone;
  return fits;
}

// The hub phase: the warps of all CTAs claim 128-edge pieces of the round's hubs (one
// counter; piece c lies in chunk c / 8, whose hub the chunk map names).
__device__ void hub_phase(const KParams& P, KSmem& S, KCnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  constexpr uint32_t kPiece = 32 * kKBatch, kPieces = kBigChunk / kPiece;
  const uint32_t* nb = reinterpret_cast<const uint32_t*>(P.adj);
  const uint32_t nsub = min((uint32_t)__ldcg(&P.ks->hub_word), P.map_cap) * kPieces;
  for (;;) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(&P.ks->hub_claim, 1u);
    c = __shfl_sync(FULL, c, 0);
    if (c >= nsub) break;
    const uint32_t slot = __ldcg(P.hub_map + c / kPieces);
    if (slot >= P.hub_cap) continue;  // chunk of a hub that did not fit (expanded in place)
    const BigItem* it = P.hub + slot;
    const uint32_t hb = __ldcg(&it->beg), he = __ldcg(&it->end), cb = __ldcg(&it->cbase);
    const uint32_t e0 = hb + (c / kPieces - cb) * kBigChunk + (c % kPieces) * kPiece;
    bool ok[kKBatch];
    uint32_t w[kKBatch];
#pragma unroll
    for (int b = 0; b < kKBatch; ++b) {
      const uint32_t e = e0 + 32u * b + lane;
      ok[b] = e < he;
      w[b] = ok[b] ? __ldg(nb + 2 * (size_t)e) : 0u;
    }
    update_batch(P, S, C, ok, w);
  }
}

// Extracts the frontier of level k.  CTAs claim tiles of frontier entries; a tile's live
// entries (priority still k) have their out-degrees scanned and all threads walk the
// joined edge list, thread t of a batch taking edge e0 + t.  Lazy: each neighbour with a
// priority above k gets one count per edge (the first count lists it as touched).
// Eager: the neighbour's priority is lowered by one (compare-and-swap, floored at k) and
// the vertex is inserted into its new bucket.
__device__ void peel_phase(const KParams& P, KSmem& S, KCnt& C) {
  const uint32_t tid = threadIdx.x;
  const uint32_t k = S.k, total = S.fr_n;
  const uint32_t* fr = S.fr_list ? P.list[S.fsel] : P.ring + (size_t)S.cur * P.cap;
  const uint32_t* nb = reinterpret_cast<const uint32_t*>(P.adj);  // .x of {nbr, w}
  // A small frontier is spread over all CTAs: the tile shrinks to about total / grid.
  const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t tile = min(P.tile, max(32u, (per + 31u) & ~31u));
  for (;;) {
    if (tid == 0) S.grab = atomicAdd(&P.sync->work, tile);
    __syncthreads();
    const uint32_t base = S.grab;
    __syncthreads();
    if (base >= total) break;
    for (uint32_t k0 = 0; k0 < tile; k0 += kBlock) {
      const uint32_t i = base + k0 + tid;
      uint32_t beg = 0, deg = 0;
      if (k0 + tid < tile && i < total) {
        const uint32_t u = __ldcg(fr + i);
        if (u < P.n) {
          C.items++;
          beg = __ldg(P.off + u);
          const uint32_t end = __ldg(P.off + u + 1);
          if (__ldcg(P.prio + u) == k) {
            deg = end - beg;
            if (deg >= P.hub_min && P.hub && push_khub(P, u, beg, end)) deg = 0;
          } else {
            C.stale++;  // priority fell below the bucket's level earlier: extracted
          }
        } else {
          report_bad(P.sync, 31u, u, i);
        }
      }
      S.lb_pos[tid] = deg;
      S.lb_beg[tid] = beg;
      __syncthreads();
      kscan(S.lb_pos, S.wtmp);
      const uint32_t etot = S.lb_pos[kBlock];
      for (uint32_t e0 = 0; e0 < etot; e0 += kBlock * kKBatch) {
        bool ok[kKBatch];
        uint32_t w[kKBatch];
#pragma unroll
        for (int b = 0; b < kKBatch; ++b) {
          const uint32_t idx = e0 + (uint32_t)b * kBlock + tid;
          ok[b] = idx < etot;
          uint32_t j = 0;
          if (ok[b]) {
#pragma unroll
            for (uint32_t s = kBlock / 2; s > 0; s >>= 1)
              if (S.lb_pos[j + s] <= idx) j += s;
          }
          const uint32_t e = S.lb_beg[j] + (idx - S.lb_pos[j]);
          w[b] = ok[b] ? __ldg(nb + 2 * (size_t)e) : 0u;
        }
        update_batch(P, S, C, ok, w);
      }
      __syncthreads();
    }
  }
}

// Lazy, apply phase: every vertex counted in the previous phase takes its count once
// (priority = max(priority - count, k), read and reset with one atomicExch so that a count
// arriving concurrently lands either here or in the next list) and moves to its window
// bucket; a vertex that drops to k is extracted at once -- its out-degrees are scanned
// across the CTA and its neighbours counted into the other list, as in the peel phase --
// so one phase per peeling round suffices.  Counts of one level add up: applying them
// together equals applying them round by round (each decrement is floored at k).
__device__ void apply_phase(const KParams& P, KSmem& S, KCnt& C) {
  const uint32_t tid = threadIdx.x;
  const uint32_t r = S.tsel ^ 1u;
  const uint32_t tn = min(__ldcg(&P.ks->touched_n[r]), P.n);
  const uint32_t k = S.k;
  const uint32_t* nb = reinterpret_cast<const uint32_t*>(P.adj);
  for (uint32_t i0 = blockIdx.x * kBlock; i0 < tn; i0 += gridDim.x * kBlock) {
    const uint32_t i = i0 + tid;
    bool has = i < tn;
    uint32_t w = 0, np = 0, beg = 0, deg = 0;
    if (has) {
      w = __ldcg(P.touched[r] + i);
      if (w < P.n) {
        const uint32_t c = atomicExch(P.cnt + w, 0u);
        const uint32_t p = __ldcg(P.prio + w);  // > k: it was counted at this level
        if (p > k) {
          np = p - k > c ? p - c : k;
          P.prio[w] = np;
          C.improved++;
          if (np == k) {  // dropped to the level: extracted now
            C.items++;
            beg = __ldg(P.off + w);
            deg = __ldg(P.off + w + 1) - beg;
            if (deg >= P.hub_min && P.hub && push_khub(P, w, beg, beg + deg)) deg = 0;
          }
        } else {
          has = false;
        }
      } else {
        report_bad(P.sync, 34u, w, i);
        has = false;
      }
    }
    const bool to_ring = has && np != k && np - S.base < kKRing;
    C.inserts += to_ring ? 1u : 0u;
    ring_insert(P, to_ring, np - S.base, w);
    S.lb_pos[tid] = deg;
    S.lb_beg[tid] = beg;
    __syncthreads();
    kscan(S.lb_pos, S.wtmp);
    const uint32_t etot = S.lb_pos[kBlock];
    for (uint32_t e0 = 0; e0 < etot; e0 += kBlock * kKBatch) {
      bool ok[kKBatch];
      uint32_t wv[kKBatch];
#pragma unroll
      for (int b = 0; b < kKBatch; ++b) {
        const uint32_t idx = e0 + (uint32_t)b * kBlock + tid;
        ok[b] = idx < etot;
        uint32_t j = 0;
        if (ok[b]) {
#pragma unroll
          for (uint32_t s = kBlock / 2; s > 0; s >>= 1)
            if (S.lb_pos[j + s] <= idx) j += s;
        }
        const uint32_t e = S.lb_beg[j] + (idx - S.lb_pos[j]);
        wv[b] = ok[b] ? __ldg(nb + 2 * (size_t)e) : 0u;
      }
      update_batch(P, S, C, ok, wv);
    }
    __syncthreads();
  }
}

// Window refill, step 1: the smallest priority >= lo over all vertices.
__device__ void min_phase(const KParams& P) {
  const uint32_t lo = __ldcg(&P.ks->lo);
  uint32_t best = kInf;
  for (uint32_t v = blockIdx.x * kBlock + threadIdx.x; v < P.n; v += gridDim.x * kBlock) {
    const uint32_t p = __ldcg(P.prio + v);
    if (p >= lo) best = min(best, p);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL, best, o));
  if ((threadIdx.x & 31) == 0 && best != kInf) atomicMin(&P.ks->kmin, best);
}

// Window refill, step 2: every vertex with a priority inside the window to its bucket.
__device__ void fill_phase(const KParams& P, KSmem& S, KCnt& C) {
  for (uint32_t v0 = blockIdx.x * kBlock; v0 < P.n; v0 += gridDim.x * kBlock) {
    const uint32_t v = v0 + threadIdx.x;
    const uint32_t p = v < P.n ? __ldcg(P.prio + v) : 0u;
    const bool in = v < P.n && p >= S.base && p - S.base < kKRing;
    C.inserts += in ? 1u : 0u;
    ring_insert(P, in, p - S.base, v);
  }
}

// A bucket that ran out of space: its level's frontier rebuilt from the priorities.
__device__ void scan_phase(const KParams& P, KSmem& S) {
  for (uint32_t v0 = blockIdx.x * kBlock; v0 < P.n; v0 += gridDim.x * kBlock) {
    const uint32_t v = v0 + threadIdx.x;
    const bool at = v < P.n && __ldcg(P.prio + v) == S.k;
    if (!warp_append(P.list[S.asel], &P.ks->next_n[S.asel], P.n, at, v))
      report_bad(P.sync, 35u, v, S.k);
  }
}

// Warp-uniform reads for the decider: lane 0 reads, every lane takes its value.  Lane 0
// of the deciding warp also rewrites some of these words, and the lanes of a warp are not
// guaranteed to run in lockstep, so a lane reading a word itself could see the new value
// while the others saw the old one, decide differently and leave the others waiting in
// a collective.
__device__ __forceinline__ uint32_t kread(const uint32_t* p) {
  uint32_t v = 0;
  if ((threadIdx.x & 31) == 0) v = __ldcg(p);
  return __shfl_sync(FULL, v, 0);
}

// The decider's view of KState: lane i loads word i in one round trip (every other CTA
// has arrived, so no word changes any more), and each field is taken from its lane by a
// shuffle, so every lane sees the same value.
constexpr uint32_t kKStateWords = sizeof(KState) / 4;
static_assert(kKStateWords <= 31 && sizeof(KState) % 8 == 0, "KState and the error word fit one warp load");
#define KS_WORD(f) ((uint32_t)(offsetof(KState, f) / 4))

// Run by warp 0 of the CTA that arrives last at a grid barrier: the next phase and level.
// Every value a decision depends on is warp-uniform: the state block is read once
// (snapshot) and the bucket arrays through ballots or kread.
__device__ void kdecide(const KParams& P, uint32_t done) {
  const uint32_t lane = threadIdx.x & 31;
  KState* ks = P.ks;
  Sync* sy = P.sync;
  const uint32_t snap = lane < kKStateWords ? __ldcg(reinterpret_cast<const uint32_t*>(ks) + lane)
                                            : (lane == 31 ? ld_relaxed(&sy->err) : 0u);
  auto F = [&](uint32_t w) -> uint32_t { return __shfl_sync(FULL, snap, (int)w); };
  const bool fatal = (F(31) & kErrFatal) != 0u;
  uint32_t next = kKStop;
  // Level c of the window: a bucket that overflowed is rebuilt by a scan.
  auto start_level = [&](uint32_t c) -> uint32_t {
    const uint32_t base = F(KS_WORD(base)), levels = F(KS_WORD(levels));
    const uint32_t scans = F(KS_WORD(scans)), asel = F(KS_WORD(asel));
    if (lane == 0) {
      ks->cur = c;
      ks->k = base + c;
      ks->levels = levels + 1u;
    }
    if (kread(P.lossy + c)) {
      if (lane == 0) {
        ks->next_n[asel] = 0u;
        ks->scans = scans + 1u;
      }
      return kKScan;
    }
    if (lane == 0) {
      ks->fr_list = 0u;
      ks->fr_n = min(__ldcg(P.counts + c), P.cap);
    }
    return kKPeel;
  };
  // The level is done: the next non-empty (or overflowed) bucket of the window, else a
  // refill of the window from the smallest priority above it.
  auto level_done = [&]() -> uint32_t {
    const uint32_t cur = F(KS_WORD(cur));
    for (uint32_t c0 = cur + 1; c0 < kKRing; c0 += 32) {
      const uint32_t c = c0 + lane;
      const bool ne = c < kKRing && (__ldcg(P.counts + c) > 0u || __ldcg(P.lossy + c) != 0u);
      const unsigned b = __ballot_sync(FULL, ne);
      if (b) return start_level(c0 + (uint32_t)(__ffs(b) - 1));
    }
    const uint32_t base = F(KS_WORD(base)), refills = F(KS_WORD(refills));
    if (lane == 0) {  // window exhausted: refill from the smallest priority above it
      ks->lo = base + kKRing;
      ks->kmin = kInf;
      ks->refills = refills + 1u;
    }
    return kKMin;
  };
  // Eager: vertices that dropped to k wait in list[asel]; they are the next round.
  auto after_round = [&]() -> uint32_t {
    if (lane == 0) P.stats->v[kStRounds] += 1ull;
    const uint32_t a = F(KS_WORD(asel)) & 1u;
    const uint32_t na = F(KS_WORD(next_n) + a);
    if (na > 0u) {  // vertices dropped to k: another round at this level
      if (lane == 0) {
        ks->fr_list = 1u;
        ks->fsel = a;
        ks->fr_n = min(na, P.n);
        ks->asel = a ^ 1u;
        ks->next_n[a ^ 1u] = 0u;
      }
      return kKPeel;
    }
    return level_done();
  };
  // Lazy: the vertices counted into touched[tsel] are applied (and those that drop to k
  // extracted) by the next apply phase, which counts into the other list, reset here.
  auto lazy_next = [&]() -> uint32_t {
    if (lane == 0) P.stats->v[kStRounds] += 1ull;
    const uint32_t t = F(KS_WORD(tsel)) & 1u;
    if (F(KS_WORD(touched_n) + t) > 0u) {
      if (lane == 0) {
        ks->tsel = t ^ 1u;
        ks->touched_n[t ^ 1u] = 0u;
      }
      return kKApply;
    }
    return level_done();
  };
  if (!fatal) {
    switch (done) {
      case kKPrologue:
        if (lane == 0) {
          ks->lo = 1u;  // priority 0: isolated vertices, coreness 0 already
          ks->kmin = kInf;
        }
        next = kKMin;
        break;
      case kKMin: {
        const uint32_t km = F(KS_WORD(kmin));
        if (km == kInf) {
          next = kKStop;
        } else {
          for (uint32_t c = lane; c < kKRing; c += 32) {
            P.counts[c] = 0u;
            P.lossy[c] = 0u;
          }
          if (lane == 0) ks->base = km;
          next = kKFill;
        }
        break;
      }
      case kKFill:
        next = start_level(0u);
        break;
      case kKScan: {
        const uint32_t a = F(KS_WORD(asel)) & 1u;
        const uint32_t na = F(KS_WORD(next_n) + a);
        if (lane == 0) {
          ks->fr_list = 1u;
          ks->fsel = a;
          ks->fr_n = min(na, P.n);
          ks->asel = a ^ 1u;
          ks->next_n[a ^ 1u] = 0u;
        }
        next = kKPeel;
        break;
      }
      case kKPeel:
      case kKApply:
        if (F(KS_WORD(hub_word) + 1) > 0u) {  // hubs listed (high word): their edges first
          next = kKHub;
          break;
        }
        next = P.eager ? after_round() : lazy_next();
        break;
      case kKHub:
        if (lane == 0) {
          ks->hub_word = 0ull;
          ks->hub_claim = 0u;
        }
        next = P.eager ? after_round() : lazy_next();
        break;
      default:
        next = kKStop;
    }
  }
  __syncwarp();
  if (lane == 0) {
    sy->phase = next;
    sy->work = 0u;
  }
}
#undef KS_WORD

// Bounded grid barrier (as in the Delta-stepping engine): the last CTA to arrive runs
// kdecide and releases the others, who give up after spin_ns or on a fatal error.
__device__ void kbarrier(const KParams& P, KSmem& S, uint32_t& bar, uint32_t done) {
  __syncthreads();
  const uint64_t t_in = threadIdx.x == 0 ? gtimer() : 0ull;
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t a = atomicAdd(&P.sync->arrive, 1u);
    S.last = (a == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (S.last) {
    __threadfence();
    if (threadIdx.x < 32) kdecide(P, done);
    __syncthreads();
    if (threadIdx.x == 0) {
      P.sync->arrive = 0;
      __threadfence();
      st_release(&P.sync->gen, bar + 1);
    }
  } else if (threadIdx.x == 0) {
    const uint64_t t0 = gtimer();
    uint32_t spins = 0;
    while (ld_acquire(&P.sync->gen) <= bar) {
      if (ld_relaxed(&P.sync->err) & kErrFatal) break;
      if ((++spins & 31u) == 0 && gtimer() - t0 > P.spin_ns) {
        atomicOr(&P.sync->err, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // The acquire that observed the new generation orders these loads after the
    // decider's writes, so they can all be issued together.
    S.phase = ld_relaxed(&P.sync->phase);
    S.err = ld_relaxed(&P.sync->err);
    const KState* ks = P.ks;
    S.k = __ldcg(&ks->k);
    S.base = __ldcg(&ks->base);
    S.cur = __ldcg(&ks->cur);
    S.fr_list = __ldcg(&ks->fr_list);
    S.fsel = __ldcg(&ks->fsel);
    S.fr_n = __ldcg(&ks->fr_n);
    S.asel = __ldcg(&ks->asel);
    S.tsel = __ldcg(&ks->tsel);
    S.t_bar += gtimer() - t_in;
  }
  __syncthreads();
  ++bar;
}

}  // namespace

extern "C" __global__ void __launch_bounds__(kBlock, 4) og_kcore_kernel(KParams P) {
  __shared__ KSmem S;
  KCnt C = {0, 0, 0, 0, 0};
  uint32_t bar = 0;
  if (threadIdx.x == 0) S.t_bar = S.t_peel = S.t_apply = S.t_hub = 0ull;
  kbarrier(P, S, bar, kKPrologue);
  for (;;) {
    const uint32_t phase = S.phase;
    if (phase == kKStop || (S.err & kErrFatal)) break;
    const uint64_t t0 = threadIdx.x == 0 ? gtimer() : 0ull;
    if (phase == kKMin) min_phase(P);
    else if (phase == kKFill) fill_phase(P, S, C);
    else if (phase == kKScan) scan_phase(P, S);
    else if (phase == kKPeel) peel_phase(P, S, C);
    else if (phase == kKApply) apply_phase(P, S, C);
    else if (phase == kKHub) hub_phase(P, S, C);
    if (threadIdx.x == 0) {
      const uint64_t dt = gtimer() - t0;
      if (phase == kKPeel) S.t_peel += dt;
      else if (phase == kKApply) S.t_apply += dt;
      else if (phase == kKHub) S.t_hub += dt;
    }
    kbarrier(P, S, bar, phase);
  }
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t vals[5] = {C.items, C.stale, C.relax, C.improved, C.inserts};
  const int idx[5] = {kStItems, kStStale, kStRelax, kStImproved, kStGlobal};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint32_t s = warp_sum(vals[i]);
    if (lane == 0 && s) atomicAdd(&P.stats->v[idx[i]], (unsigned long long)s);
  }
  if (threadIdx.x == 0) {
    atomicAdd(&P.stats->v[kStTBarrier], S.t_bar);
    atomicAdd(&P.stats->v[kStTFrontier], S.t_peel);
    atomicAdd(&P.stats->v[kStTFused], S.t_apply);
    atomicAdd(&P.stats->v[kStTHub], S.t_hub);
  }
}

// priority <- out-degree
extern "C" __global__ void og_kcore_init_kernel(const uint32_t* off, uint32_t* prio, uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    prio[v] = off[v + 1] - off[v];
}

cudaError_t kcore_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, og_kcore_kernel, kBlock, 0);
}

cudaError_t launch_kcore(const KParams& P, int grid, cudaStream_t st) {
  void* args[] = {const_cast<KParams*>(&P)};
  return cudaLaunchCooperativeKernel((const void*)og_kcore_kernel, dim3(grid), dim3(kBlock), args,
                                     0, st);
}

cudaError_t launch_kcore_init(const uint32_t* off, uint32_t* prio, uint32_t n, int sms,
                              cudaStream_t st) {
  og_kcore_init_kernel<<<sms * 4, 256, 0, st>>>(off, prio, n);
  return cudaGetLastError();
}

}  // namespace og
