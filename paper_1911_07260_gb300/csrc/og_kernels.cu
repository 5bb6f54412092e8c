// Device side of libog: Delta-stepping with eager bucket update and bucket fusion.
//
// Mapping of the paper's method (Section 3.2 / 3.3 and the figure of SSSP with
// eager bucket updates and bucket fusion) onto one persistent,
// cooperatively launched kernel:
//   * the thread-local buckets of the paper become CTA-local bins in shared memory for
//     the current bucket, plus per-query materialised global buckets (a ring of B device
//     arrays) and one overflow pile for buckets beyond the ring;
//   * one "round" = every CTA claims tiles of the current bucket's global frontier and
//     relaxes their out-edges (atomicMin on the uint32 distance; an improved vertex is
//     appended to bucket floor(d / Delta) -- the eager update), then runs the fusion
//     loop: while its local bin of the current bucket is non-empty and smaller than the
//     threshold it processes that bin with block-level synchronisation only; a bin that
//     reaches the threshold is copied to the global bucket so the next round spreads it
//     over all CTAs;
//   * between rounds a bounded grid barrier runs; the CTA that arrives last picks the
//     next bucket of every query (the smallest non-empty one, scanned with a warp ballot)
//     and applies the PPSP / A* stop rule before it releases the others.
// Within a round: frontier tiles are expanded CTA-wide and edge-balanced (expand_cta),
// fused levels per warp (expand_warp); vertices of out-degree >= hub_degree are listed
// and their edges split over every warp after the frontier pass (BIG phase).  Two more
// modes share the kernel: the lazy bucket update (Section 3.1: marks during the round,
// one insertion per marked vertex in the APPLY phase) and unordered Bellman-Ford
// (QDesc.delta = 0: every improvement goes to bucket cur + 1).
#include "og_device.cuh"

namespace og {

struct Smem {
  uint32_t cur[kMaxQ];     // current bucket per query
  uint32_t delta[kMaxQ];
  uint32_t head[kMaxQ];    // frontier start in the current ring slot
  uint32_t pref[kMaxQ + 1];// frontier prefix sums (scratch in the decider)
  uint32_t binN[2];        // CTA-local bin fill counts
  uint32_t grab;
  uint32_t last;
  uint32_t phase;
  uint32_t err;
  uint32_t f_active, f_redist;
  uint32_t wtmp[kWarps + 1];
  uint32_t lb_pos[kBlock + 1];  // CTA-wide expansion: edge prefix sums of the entries
  uint32_t lb_beg[kBlock], lb_g[kBlock], lb_q[kBlock];
  unsigned long long t_front, t_fused, t_bar, t_hub;  // per-CTA phase time (thread 0)
};

struct Bins {
  uint2* e[2];
  uint16_t* q[2];
};

struct Cnt {
  uint32_t items, stale, relax, improved, local, global, ovf;
};

// Appends the improved vertices of a warp (lanes with ins) to their buckets: the CTA-local
// bin when the bucket is the query's current one and fusion is on, else the ring slot of
// the bucket (warp-aggregated: lanes with the same (query, slot) share one atomicAdd),
// else the overflow pile.  Must be called by all 32 lanes.
__device__ __forceinline__ void insert_warp(const Params& P, Smem& S, const Bins& B, int out,
                                            bool ins, bool allow_local, uint32_t v,
                                            uint32_t nd, uint32_t key, uint32_t q, Cnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  if (__ballot_sync(FULL, ins) == 0u) return;  // nothing improved in this group
  int dest = 0;  // 0 none, 1 local bin, 2 ring, 3 overflow
  if (ins) {
    const uint32_t cq = S.cur[q];
    if (key < cq) {  // only with an inconsistent A* heuristic: clamp, disable early exit
      key = cq;
      P.qs[q].no_exit = 1u;
    }
    dest = (allow_local && key == cq) ? 1 : ((key - cq < P.B) ? 2 : 3);
  }
  const unsigned lm = __ballot_sync(FULL, dest == 1);
  if (lm) {
    const int leader = __ffs(lm) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(&S.binN[out], (uint32_t)__popc(lm));
    base = __shfl_sync(FULL, base, leader);
    if (dest == 1) {
      const uint32_t pos = base + __popc(lm & lanemask_lt());
      if (pos < P.bin_cap) {
        B.e[out][pos] = make_uint2(v, nd);
        B.q[out][pos] = (uint16_t)q;
        C.local++;
      } else {
        dest = 2;  // bin full: the entry goes to the global current bucket
      }
    }
  }
  const unsigned rm = __ballot_sync(FULL, dest == 2);
  if (dest == 2) {
    const uint32_t cid = q * P.B + (key & P.Bmask);
    const unsigned peers = __match_any_sync(rm, cid);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(P.counts + cid, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t pos = base + __popc(peers & lanemask_lt());
    if (pos < P.cap) {
      P.ring[(size_t)cid * P.cap + pos] = make_uint2(v, nd);
      C.global++;
    } else {
      dest = 3;  // slot full: spill to the overflow pile
    }
  }
  if (dest == 3) {
    QState* s = P.qs + q;
    const uint32_t sel = __ldcg(&s->ovf_sel);
    const uint32_t pos = atomicAdd(&s->ovf_n, 1u);
    atomicMin(&s->ovf_min, key);
    if (pos < P.ocap) {
      P.ovf[((size_t)q * 2 + sel) * P.ocap + pos] = make_uint2(v, nd);
      C.ovf++;
    } else {
      s->aborted = 1u;
      atomicOr(&P.sync->err, kErrArena);
    }
  }
}

// Lazy bucket update: appends {vertex, query} of the lanes with first (the vertex's first
// improvement this round) to the round's list, warp-aggregated.  All 32 lanes call it.
__device__ __forceinline__ void mark_warp(const Params& P, bool first, uint32_t v, uint32_t q) {
  const unsigned m = __ballot_sync(FULL, first);
  if (m == 0u) return;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&P.sync->lz_n, (uint32_t)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (!first) return;
  const uint32_t pos = base + __popc(m & lanemask_lt());
  if (pos < P.lz_cap) P.lz_list[pos] = make_uint2(v, q);
  else report_bad(P.sync, 41u, v, q);  // more marks in one round than the list holds
}

// Relaxes up to K edges per lane: nd = g + w (saturating), atomicMin on dist[v]; an
// improvement is inserted eagerly into bucket floor((nd + h) / Delta).  All K neighbor
// loads are issued before any atomic and all K atomics before any insert, so a lane keeps
// K independent memory operations in flight instead of paying one round trip per edge.
// Relaxes up to K already-loaded edges per lane: nd = g + w (saturating), atomicMin on
// dist[v]; an improvement is inserted eagerly into bucket floor((nd + h) / Delta).  All K
// atomics are issued before any insert, so a lane keeps K independent memory operations
// in flight instead of paying one round trip per edge.
template <int K>
__device__ __forceinline__ void relax_edges(const Params& P, Smem& S, const Bins& B, int out,
                                            bool allow_local, const bool (&ok)[K],
                                            const uint2 (&ew)[K], const uint32_t (&g)[K],
                                            const uint32_t (&q)[K], Cnt& C) {
  uint32_t h[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    h[k] = 0;
    if (P.has_astar && ok[k]) {
      const QDesc* d = P.qd + q[k];
      if (__ldg(&d->kind) == kASTAR)
        h[k] = heuristic(P.xy, P.xy_integral, ew[k].x, __ldg(&d->tx), __ldg(&d->ty));
    }
  }
  uint32_t nd[K], old[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const unsigned long long s = (unsigned long long)g[k] + ew[k].y;
    nd[k] = s >= kSat ? kSat : (uint32_t)s;
    if (ok[k] && s >= kSat) atomicOr(&P.sync->err, kErrSat);
  }
  bool go[K];
#pragma unroll
  for (int k = 0; k < K; ++k) go[k] = ok[k];
  if (P.precheck) {
    uint32_t seen[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
      seen[k] = ok[k] ? ld_cached(P.dist + (size_t)q[k] * P.n + ew[k].x) : 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) go[k] = ok[k] && nd[k] < seen[k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    old[k] = go[k] ? atomicMin(P.dist + (size_t)q[k] * P.n + ew[k].x, nd[k]) : 0u;
  if (P.lazy) {  // lazy bucket update: mark each improved vertex once this round
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ins = go[k] && nd[k] < old[k];
      C.relax += ok[k] ? 1u : 0u;
      C.improved += ins ? 1u : 0u;
      bool first = false;
      if (ins) {
        const uint32_t bit = 1u << (ew[k].x & 31u);
        first = (atomicOr(P.lz_bits + (size_t)q[k] * P.lz_words + (ew[k].x >> 5), bit) & bit) == 0u;
      }
      mark_warp(P, first, ew[k].x, q[k]);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool ins = go[k] && nd[k] < old[k];
    C.relax += ok[k] ? 1u : 0u;
    C.improved += ins ? 1u : 0u;
    if (ins && P.prefetch) prefetch_row(P.ell, P.off, ew[k].x);
    // Delta 0 marks a Bellman-Ford query: the next round's bucket, whatever the distance.
    const uint32_t dq = S.delta[q[k]];
    const uint32_t key = ins ? (dq ? bucket_of(nd[k], h[k], dq) : S.cur[q[k]] + 1u) : 0u;
    insert_warp(P, S, B, out, ins, allow_local, ew[k].x, nd[k], key, q[k], C);
  }
}

// CSR edges: the K neighbor loads are issued together, then relax_edges.
template <int K>
__device__ __forceinline__ void relax_batch(const Params& P, Smem& S, const Bins& B, int out,
                                            bool allow_local, const bool (&ok)[K],
                                            const uint32_t (&e)[K], const uint32_t (&g)[K],
                                            const uint32_t (&q)[K], Cnt& C) {
  uint2 ew[K];
#pragma unroll
  for (int k = 0; k < K; ++k) ew[k] = ok[k] ? __ldg(P.adj + e[k]) : make_uint2(0u, 0u);
  relax_edges<K>(P, S, B, out, allow_local, ok, ew, g, q, C);
}

constexpr int kLightBatch = 4;  // light-edge groups of 32 relaxed per batch
constexpr int kHeavyBatch = 4;  // groups of 32 edges of one heavy vertex per batch

// Lists a hub for the BIG phase.  One 64-bit atomicAdd reserves the hub's slot (high
// word) and its range of kBigChunk-edge chunks (low word) together, so chunk ranges grow
// with the slot; the chunk map then names the slot of each of its chunks.  Returns false
// when the list or the map is full: the caller expands the vertex itself, and the chunks
// it reserved are marked kNone.
__device__ __noinline__ bool push_hub(const Params& P, uint32_t u, uint32_t g, uint32_t q,
                                      uint32_t beg, uint32_t end) {
  const uint32_t nch = (end - beg + kBigChunk - 1) / kBigChunk;
  const unsigned long long w = atomicAdd(&P.sync->big_word, (1ull << 32) | nch);
  const uint32_t slot = (uint32_t)(w >> 32), cbase = (uint32_t)w;
  const bool fits = slot < P.big_cap && cbase <= P.map_cap && nch <= P.map_cap - cbase;
  if (fits) {
    BigItem it;
    it.u = u;
    it.g = g;
    it.q = q;
    it.beg = beg;
    it.end = end;
    it.cbase = cbase;
    P.big[slot] = it;
  }
  const uint32_t lim = cbase < P.map_cap ? min(P.map_cap - cbase, nch) : 0u;
  for (uint32_t c = 0; c < lim; ++c) P.big_map[cbase + c] = fits ? slot : kNone;
  return fits;
}

// Expands the bucket entries held by a warp (one per lane with has): drops entries whose
// vertex has a smaller distance by now (a newer entry exists), then relaxes all out-edges.
// Vertices with >= 32 edges are expanded by the whole warp one at a time; the others are
// flattened into one edge list that the 32 lanes walk together, so consecutive lanes
// read consecutive edges of a vertex.  Must be called by all 32 lanes.
template <bool ELL>
__device__ __forceinline__ void expand_warp(const Params& P, Smem& S, const Bins& B, int out,
                                            bool allow_local, bool has, uint32_t u,
                                            uint32_t g, uint32_t q, Cnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  if (ELL) {
    // ELL rows: each lane reads its vertex's whole row (64 bytes, no offsets lookup) in
    // parallel with the stale check and relaxes its up to 8 edges together.
    uint2 ew[kEllWidth];
    bool live = has;
    uint32_t d = 0;
    if (has) {
      C.items++;
      d = __ldcg(P.dist + (size_t)q * P.n + u);
      load_row(P.ell, u, ew);
    } else {
#pragma unroll
      for (int k = 0; k < kEllWidth; ++k) ew[k] = make_uint2(kNone, 0u);
    }
    if (has && d != g) {
      live = false;
      C.stale++;
    }
    bool ok[kEllWidth];
    uint32_t gg[kEllWidth], qq[kEllWidth];
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k) {
      ok[k] = live && ew[k].x != kNone;
      gg[k] = g;
      qq[k] = q;
    }
    relax_edges<kEllWidth>(P, S, B, out, allow_local, ok, ew, gg, qq, C);
    return;
  }
  uint32_t beg = 0, end = 0;
  if (has) {
    C.items++;
    const uint32_t d = __ldcg(P.dist + (size_t)q * P.n + u);
    beg = __ldg(P.off + u);
    end = __ldg(P.off + u + 1);
    if (d != g) {
      has = false;
      C.stale++;
      beg = end = 0;
    }
  }
  if (end - beg >= P.hub_min && P.big && push_hub(P, u, g, q, beg, end)) beg = end = 0;
  const bool heavy = end - beg >= 32u;
  unsigned hm = __ballot_sync(FULL, heavy);
  while (hm) {
    const int l = __ffs(hm) - 1;
    hm &= hm - 1;
    const uint32_t hb = __shfl_sync(FULL, beg, l), he = __shfl_sync(FULL, end, l);
    const uint32_t hg = __shfl_sync(FULL, g, l), hq = __shfl_sync(FULL, q, l);
    for (uint32_t e0 = hb; e0 < he; e0 += 32 * kHeavyBatch) {
      bool ok[kHeavyBatch];
      uint32_t ee[kHeavyBatch], gg[kHeavyBatch], qq[kHeavyBatch];
#pragma unroll
      for (int k = 0; k < kHeavyBatch; ++k) {
        ee[k] = e0 + 32u * k + lane;
        ok[k] = ee[k] < he;
        gg[k] = hg;
        qq[k] = hq;
      }
      relax_batch<kHeavyBatch>(P, S, B, out, allow_local, ok, ee, gg, qq, C);
    }
  }
  const uint32_t ld = heavy ? 0u : end - beg;
  uint32_t incl = ld;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  const uint32_t excl = incl - ld;
  for (uint32_t base = 0; base < total; base += 32 * kLightBatch) {
    bool ok[kLightBatch];
    uint32_t ee[kLightBatch], gg[kLightBatch], qq[kLightBatch];
#pragma unroll
    for (int k = 0; k < kLightBatch; ++k) {
      const uint32_t idx = base + 32u * k + lane;
      uint32_t pos = 0;  // owner lane: number of lanes whose inclusive sum is <= idx
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const uint32_t x = __shfl_sync(FULL, incl, pos + s - 1);
        if (x <= idx) pos += s;
      }
      const uint32_t ob = __shfl_sync(FULL, beg, pos), oe = __shfl_sync(FULL, excl, pos);
      gg[k] = __shfl_sync(FULL, g, pos);
      qq[k] = __shfl_sync(FULL, q, pos);
      ok[k] = idx < total;
      ee[k] = ob + (idx - oe);
    }
    relax_batch<kLightBatch>(P, S, B, out, allow_local, ok, ee, gg, qq, C);
  }
}

// Block-wide exclusive scan of a[0..n) in place (each thread scans a run of
// ceil(n / kBlock) consecutive elements); a[n] = total.
__device__ void block_exscan(uint32_t* a, uint32_t n, uint32_t* wtmp) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t per = (n + kBlock - 1) / kBlock;
  const uint32_t lo = min(n, tid * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += a[i];
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) wtmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < (uint32_t)kWarps ? wtmp[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, wi, o);
      if ((int)lane >= o) wi += t;
    }
    __syncwarp();
    if (lane < (uint32_t)kWarps) wtmp[lane] = wi - w;
  }
  __syncthreads();
  uint32_t run = wtmp[warp] + incl - s;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t x = a[i];
    a[i] = run;
    run += x;
  }
  if (tid == kBlock - 1) a[n] = run;
  __syncthreads();
}

// Expands up to kBlock bucket entries (one per thread with has) with the whole CTA: after
// the stale check the entries' out-degrees are scanned, and all threads walk the joined
// edge list together, edge idx going to the entry whose range holds it (binary search in
// shared memory).  Thread t of a batch takes edge e0 + t, so a warp reads 32 consecutive
// edges and one high-degree entry no longer holds up a single warp.  Hubs are listed for
// the BIG phase instead.  Must be called by all threads of the CTA (CSR layout only).
__device__ __forceinline__ void expand_cta(const Params& P, Smem& S, const Bins& B, int out,
                                           bool allow_local, bool has, uint32_t u,
                                           uint32_t g, uint32_t q, Cnt& C) {
  const uint32_t tid = threadIdx.x;
  uint32_t beg = 0, deg = 0;
  if (has) {
    C.items++;
    const uint32_t d = __ldcg(P.dist + (size_t)q * P.n + u);
    beg = __ldg(P.off + u);
    const uint32_t end = __ldg(P.off + u + 1);
    if (d != g) {
      C.stale++;
    } else {
      deg = end - beg;
      if (deg >= P.hub_min && P.big && push_hub(P, u, g, q, beg, end)) deg = 0;
    }
  }
  S.lb_pos[tid] = deg;
  S.lb_beg[tid] = beg;
  S.lb_g[tid] = g;
  S.lb_q[tid] = q;
  __syncthreads();
  block_exscan(S.lb_pos, kBlock, S.wtmp);
  const uint32_t total = S.lb_pos[kBlock];
  for (uint32_t e0 = 0; e0 < total; e0 += kBlock * kLightBatch) {
    bool ok[kLightBatch];
    uint32_t ee[kLightBatch], gg[kLightBatch], qq[kLightBatch];
#pragma unroll
    for (int k = 0; k < kLightBatch; ++k) {
      const uint32_t idx = e0 + (uint32_t)k * kBlock + tid;
      ok[k] = idx < total;
      uint32_t j = 0;  // last entry whose edge range starts at or before idx
      if (ok[k]) {
#pragma unroll
        for (uint32_t s = kBlock / 2; s > 0; s >>= 1)
          if (S.lb_pos[j + s] <= idx) j += s;
      }
      ee[k] = S.lb_beg[j] + (idx - S.lb_pos[j]);
      gg[k] = S.lb_g[j];
      qq[k] = S.lb_q[j];
    }
    relax_batch<kLightBatch>(P, S, B, out, allow_local, ok, ee, gg, qq, C);
  }
  __syncthreads();  // the lb arrays are refilled by the next call
}

// Run by the CTA that arrives last at a grid barrier, before it releases the others:
// advances every query's bucket cursor and publishes the next phase and frontier.
__device__ void decide(const Params& P, Smem& S, uint32_t done_phase) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Sync* sy = P.sync;
  const uint32_t err = ld_relaxed(&sy->err);
  const bool fatal = (err & kErrFatal) != 0;
  if (done_phase == kPhRelax && !fatal && (__ldcg(&sy->big_word) >> 32) > 0u) {
    // Listed hubs first: the same round continues with the BIG phase.
    if (tid == 0) {
      sy->phase = kPhBig;
      sy->work = 0;
    }
    return;
  }
  if (done_phase == kPhBig) {
    if (tid == 0) {
      sy->big_word = 0ull;
      sy->big_claim = 0u;
    }
    done_phase = kPhRelax;
  }
  if (done_phase == kPhRelax && !fatal && P.lazy && __ldcg(&sy->lz_n) > 0u) {
    // Lazy bucket update: the marked vertices make their insertions before the round ends.
    if (tid == 0) {
      sy->phase = kPhApply;
      sy->work = 0;
    }
    return;
  }
  if (done_phase == kPhApply) {
    if (tid == 0) sy->lz_n = 0u;
    done_phase = kPhRelax;
  }
  if (tid == 0) {
    S.f_active = 0;
    S.f_redist = 0;
  }
  __syncthreads();
  for (uint32_t q = warp; q < P.nq; q += kWarps) {
    QState* qs = P.qs + q;
    uint32_t* cnts = P.counts + (size_t)q * P.B;
    uint32_t active = __ldcg(&qs->active);
    uint32_t size = 0;
    if (active && __ldcg(&qs->aborted)) {
      active = 0;
      if (lane == 0) {
        qs->active = 0;
        qs->redist = 0;
        qs->result = kInf;
      }
    }
    if (active && !fatal) {
      uint32_t cur = __ldcg(&qs->cur), head = __ldcg(&qs->head), tail = __ldcg(&qs->tail);
      uint32_t redist = __ldcg(&qs->redist);
      if (done_phase == kPhRelax) {
        const uint32_t c = cur & P.Bmask;
        const uint32_t cnt = min(__ldcg(cnts + c), P.cap);
        if (cnt > tail) {  // the current bucket received entries: process it again
          head = tail;
          tail = cnt;
        } else {           // current bucket finished: find the next non-empty one
          uint32_t next = kInf;
          for (uint32_t base = 1; base < P.B; base += 32) {
            const uint32_t k = base + lane;
            const bool ne = k < P.B && __ldcg(cnts + ((cur + k) & P.Bmask)) > 0u;
            const unsigned b = __ballot_sync(FULL, ne);
            if (b) {
              next = cur + base + (uint32_t)(__ffs(b) - 1);
              break;
            }
          }
          __syncwarp();
          if (lane == 0) cnts[c] = 0u;
          const uint32_t ovf_n = __ldcg(&qs->ovf_n), ovf_min = __ldcg(&qs->ovf_min);
          if (ovf_n > 0 && ovf_min <= next) {
            redist = 1;
            if (lane == 0) {
              qs->redist_min = next;
              qs->ovf_n2 = 0;
              qs->ovf_min2 = kInf;
            }
          } else if (next == kInf) {
            active = 0;
          } else {
            cur = next;
            head = 0;
            tail = min(__ldcg(cnts + (next & P.Bmask)), P.cap);
          }
        }
      } else if (done_phase == kPhRedistMin && redist) {
        const uint32_t nc = __ldcg(&qs->redist_min);
        if (nc == kInf) {  // every pile entry was out of date and the ring is empty
          active = 0;
          redist = 0;
          if (lane == 0) qs->ovf_n = 0;
        } else {
          cur = nc;
        }
      } else if (done_phase == kPhRedistMove && redist) {
        if (lane == 0) {
          qs->ovf_sel = __ldcg(&qs->ovf_sel) ^ 1u;
          qs->ovf_n = __ldcg(&qs->ovf_n2);
          qs->ovf_min = __ldcg(&qs->ovf_min2);
        }
        redist = 0;
        head = 0;
        tail = min(__ldcg(cnts + (cur & P.Bmask)), P.cap);
      }
      const QDesc* qd = P.qd + q;
      const uint32_t kind = __ldg(&qd->kind);
      const uint32_t dst = __ldg(&qd->dst);
      if (active && !redist && (kind == kPPSP || kind == kASTAR) && !__ldcg(&qs->no_exit)) {
        // Stop rule of Section 6.1 (PPSP): entering bucket i with i * Delta >= the best
        // distance to the target found so far.
        const uint32_t dt = __ldcg(P.dist + (size_t)q * P.n + dst);
        if (dt != kInf && (unsigned long long)cur * __ldg(&qd->delta) >= dt) active = 0;
      }
      if (lane == 0) {
        qs->cur = cur;
        qs->head = head;
        qs->tail = tail;
        qs->redist = redist;
        qs->active = active;
        if (!active)
          qs->result = dst < P.n ? __ldcg(P.dist + (size_t)q * P.n + dst) : 0u;
        if (active) S.f_active = 1;
        if (redist) S.f_redist = 1;
      }
      size = (active && !redist) ? tail - head : 0u;
    }
    if (lane == 0) S.pref[q] = size;
  }
  __syncthreads();
  block_exscan(S.pref, P.nq, S.wtmp);
  for (uint32_t q = tid; q <= P.nq; q += kBlock) P.fr_pref[q] = S.pref[q];
  if (tid == 0) {
    uint32_t next = kPhStop;
    if (!fatal) {
      if (done_phase == kPhRedistMin)
        next = S.f_redist ? kPhRedistMove : (S.f_active ? kPhRelax : kPhStop);
      else if (done_phase == kPhRedistMove)
        next = S.f_active ? kPhRelax : kPhStop;
      else
        next = S.f_redist ? kPhRedistMin : (S.f_active ? kPhRelax : kPhStop);
    }
    if (next == kPhRelax) {
      if (sy->rounds >= P.max_rounds) next = kPhStop;
      else sy->rounds = sy->rounds + 1;
    }
    sy->phase = next;
    sy->work = 0;
    sy->total = S.pref[P.nq];
    sy->any_active = S.f_active;
    P.stats->v[kStRounds] += (next == kPhRelax) ? 1ull : 0ull;
    if (done_phase == kPhRedistMove) P.stats->v[kStRedist] += 1ull;
  }
}

// Grid-wide barrier with bounded waiting.  The last CTA to arrive runs decide() and then
// releases the generation word; the others poll it with an acquire load and give up
// (setting kErrTimeout) after spin_ns nanoseconds or as soon as a fatal error is posted.
__device__ void grid_barrier(const Params& P, Smem& S, uint32_t& bar, uint32_t done_phase) {
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
    decide(P, S, done_phase);
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
    S.phase = ld_acquire(&P.sync->phase);
    S.err = ld_relaxed(&P.sync->err);
    S.t_bar += gtimer() - t_in;
  }
  __syncthreads();
  ++bar;
}

// One round for all active queries: frontier pass over the global current buckets, then
// the CTA-local fusion loop (Section 3.3): the CTA's warps drain its local bin together,
// one level per iteration, with block-level synchronisation only.
template <bool ELL>
__device__ void relax_phase(const Params& P, Smem& S, const Bins& B, Cnt& C, uint32_t& fused) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t q = tid; q < P.nq; q += kBlock) {
    S.cur[q] = __ldcg(&P.qs[q].cur);
    S.head[q] = __ldcg(&P.qs[q].head);
    S.pref[q] = __ldcg(P.fr_pref + q);
  }
  if (tid == 0) {
    S.pref[P.nq] = __ldcg(P.fr_pref + P.nq);
    S.binN[0] = 0;
    S.binN[1] = 0;
  }
  __syncthreads();
  const uint32_t total = S.pref[P.nq];
  const bool fuse = P.T != 0;
  const uint64_t t_start = tid == 0 ? gtimer() : 0ull;
  for (;;) {
    if (tid == 0) S.grab = atomicAdd(&P.sync->work, P.tile);
    __syncthreads();
    const uint32_t base = S.grab;
    __syncthreads();
    if (base >= total) break;
    for (uint32_t k = tid; k < (ELL ? P.tile : (P.tile + kBlock - 1) / kBlock * kBlock);
         k += kBlock) {
      const uint32_t i = base + k;
      const bool has = k < P.tile && i < total;
      uint32_t u = 0, g = 0, q = 0;
      if (has) {
        uint32_t lo = 0, hi = P.nq;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (S.pref[mid] <= i) lo = mid; else hi = mid;
        }
        q = lo;
        const uint32_t pos = S.head[q] + (i - S.pref[q]);
        const uint2 en =
            __ldcg(P.ring + ((size_t)q * P.B + (S.cur[q] & P.Bmask)) * P.cap + pos);
        u = en.x;
        g = en.y;
      }
      if constexpr (ELL) expand_warp<true>(P, S, B, 0, fuse, has, u, g, q, C);
      else expand_cta(P, S, B, 0, fuse, has, u, g, q, C);
    }
  }
  const uint64_t t_mid = tid == 0 ? gtimer() : 0ull;
  if (tid == 0) S.t_front += t_mid - t_start;
  if (!fuse) return;
  int in = 0;
  for (;;) {
    __syncthreads();
    const uint32_t nin = S.binN[in];
    if (nin == 0) break;
    const uint32_t cnt = min(nin, P.bin_cap);
    const uint32_t lim = (cnt + 31u) & ~31u;
    if (nin >= P.T) {
      // Large local bucket: hand it to the global bucket for the next round.
      for (uint32_t k = tid; k < lim; k += kBlock) {
        const bool has = k < cnt;
        uint2 en = make_uint2(0, 0);
        uint32_t q = 0;
        if (has) {
          en = B.e[in][k];
          q = B.q[in][k];
        }
        insert_warp(P, S, B, in ^ 1, has, false, en.x, en.y, has ? S.cur[q] : 0u, q, C);
      }
      __syncthreads();
      if (tid == 0) S.binN[in] = 0;
      break;
    }
    for (uint32_t k = tid; k < lim; k += kBlock) {
      const bool has = k < cnt;
      uint2 en = make_uint2(0, 0);
      uint32_t q = 0;
      if (has) {
        en = B.e[in][k];
        q = B.q[in][k];
      }
      expand_warp<ELL>(P, S, B, in ^ 1, true, has, en.x, en.y, q, C);
    }
    __syncthreads();
    if (tid == 0) S.binN[in] = 0;
    in ^= 1;
    ++fused;
  }
  __syncthreads();
  if (tid == 0) S.t_fused += gtimer() - t_mid;
}

// Overflow redistribution, step 1: the smallest bucket among live pile entries.
__device__ void redist_min_phase(const Params& P) {
  const uint32_t gtid = blockIdx.x * kBlock + threadIdx.x, gstride = gridDim.x * kBlock;
  for (uint32_t q = 0; q < P.nq; ++q) {
    QState* qs = P.qs + q;
    if (!__ldcg(&qs->redist)) continue;
    const uint32_t sel = __ldcg(&qs->ovf_sel);
    const uint32_t n = min(__ldcg(&qs->ovf_n), P.ocap);
    const QDesc* qd = P.qd + q;
    const bool astar = __ldg(&qd->kind) == kASTAR;
    const uint32_t delta = __ldg(&qd->delta);
    const uint2* pile = P.ovf + ((size_t)q * 2 + sel) * P.ocap;
    uint32_t best = kInf;
    for (uint32_t i = gtid; i < n; i += gstride) {
      const uint2 en = __ldcg(pile + i);
      if (__ldcg(P.dist + (size_t)q * P.n + en.x) != en.y) continue;
      const uint32_t h = astar ? heuristic(P.xy, P.xy_integral, en.x, __ldg(&qd->tx), __ldg(&qd->ty)) : 0u;
      best = min(best, delta ? bucket_of(en.y, h, delta) : __ldcg(&qs->redist_min));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL, best, o));
    if ((threadIdx.x & 31) == 0 && best != kInf) atomicMin(&qs->redist_min, best);
  }
}

// Overflow redistribution, step 2: live entries of the new ring window move into the
// ring, the rest into the other pile.
__device__ void redist_move_phase(const Params& P) {
  const uint32_t gtid = blockIdx.x * kBlock + threadIdx.x, gstride = gridDim.x * kBlock;
  for (uint32_t q = 0; q < P.nq; ++q) {
    QState* qs = P.qs + q;
    if (!__ldcg(&qs->redist)) continue;
    const uint32_t sel = __ldcg(&qs->ovf_sel);
    const uint32_t n = min(__ldcg(&qs->ovf_n), P.ocap);
    const uint32_t cur = __ldcg(&qs->cur);
    const QDesc* qd = P.qd + q;
    const bool astar = __ldg(&qd->kind) == kASTAR;
    const uint32_t delta = __ldg(&qd->delta);
    const uint2* pile = P.ovf + ((size_t)q * 2 + sel) * P.ocap;
    uint2* other = P.ovf + ((size_t)q * 2 + (sel ^ 1u)) * P.ocap;
    for (uint32_t i = gtid; i < n; i += gstride) {
      const uint2 en = __ldcg(pile + i);
      if (__ldcg(P.dist + (size_t)q * P.n + en.x) != en.y) continue;
      const uint32_t h = astar ? heuristic(P.xy, P.xy_integral, en.x, __ldg(&qd->tx), __ldg(&qd->ty)) : 0u;
      const uint32_t key = delta ? bucket_of(en.y, h, delta) : cur;
      bool to_pile = true;
      if (key - cur < P.B) {
        const uint32_t cid = q * P.B + (key & P.Bmask);
        const uint32_t pos = atomicAdd(P.counts + cid, 1u);
        if (pos < P.cap) {
          P.ring[(size_t)cid * P.cap + pos] = en;
          to_pile = false;
        }
      }
      if (to_pile) {
        const uint32_t pos = atomicAdd(&qs->ovf_n2, 1u);
        atomicMin(&qs->ovf_min2, key);
        if (pos < P.ocap) {
          other[pos] = en;
        } else {
          qs->aborted = 1u;
          atomicOr(&P.sync->err, kErrArena);
        }
      }
    }
  }
}

// The BIG phase: the warps of all CTAs claim kBigSub-edge pieces of the hubs listed in
// this round (one counter; piece c lies in chunk c / kBigSubs, whose hub the chunk map
// names), so a hub is spread over the whole grid.  Improved vertices go to the global
// buckets.
__device__ void big_phase(const Params& P, Smem& S, const Bins& B, Cnt& C) {
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint64_t t_start = tid == 0 ? gtimer() : 0ull;
  for (uint32_t q = tid; q < P.nq; q += kBlock) S.cur[q] = __ldcg(&P.qs[q].cur);
  __syncthreads();
  const uint32_t nsub = min((uint32_t)__ldcg(&P.sync->big_word), P.map_cap) * kBigSubs;
  for (;;) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(&P.sync->big_claim, 1u);
    c = __shfl_sync(FULL, c, 0);
    if (c >= nsub) break;
    const uint32_t slot = __ldcg(P.big_map + c / kBigSubs);
    if (slot >= P.big_cap) continue;  // chunk of a hub that did not fit (expanded in place)
    const BigItem* it = P.big + slot;
    const uint32_t hb = __ldcg(&it->beg), he = __ldcg(&it->end);
    const uint32_t hg = __ldcg(&it->g), hq = __ldcg(&it->q), cb = __ldcg(&it->cbase);
    const uint32_t e0 = hb + (c / kBigSubs - cb) * kBigChunk + (c % kBigSubs) * kBigSub;
    for (uint32_t s0 = e0; s0 < min(he, e0 + kBigSub); s0 += 32 * kHeavyBatch) {
      bool ok[kHeavyBatch];
      uint32_t ee[kHeavyBatch], gg[kHeavyBatch], qq[kHeavyBatch];
#pragma unroll
      for (int k = 0; k < kHeavyBatch; ++k) {
        ee[k] = s0 + 32u * k + lane;
        ok[k] = ee[k] < he;
        gg[k] = hg;
        qq[k] = hq;
      }
      relax_batch<kHeavyBatch>(P, S, B, 0, false, ok, ee, gg, qq, C);
    }
  }
  __syncthreads();
  if (tid == 0) S.t_hub += gtimer() - t_start;
}

// The lazy bucket update's reduction (Section 3.1): every vertex marked this round is
// inserted once, into the bucket of its distance now (the minimum of the round's
// updates); its mark is cleared for the next round.
__device__ void lazy_apply_phase(const Params& P, Smem& S, const Bins& B, Cnt& C) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t q = tid; q < P.nq; q += kBlock) S.cur[q] = __ldcg(&P.qs[q].cur);
  __syncthreads();
  const uint32_t tn = min(__ldcg(&P.sync->lz_n), P.lz_cap);
  for (uint32_t i0 = blockIdx.x * kBlock; i0 < tn; i0 += gridDim.x * kBlock) {
    const uint32_t i = i0 + tid;
    bool has = i < tn;
    uint32_t v = 0, q = 0, d = 0, key = 0;
    if (has) {
      const uint2 en = __ldcg(P.lz_list + i);
      v = en.x;
      q = en.y;
      if (v < P.n && q < P.nq) {
        atomicAnd(P.lz_bits + (size_t)q * P.lz_words + (v >> 5), ~(1u << (v & 31u)));
        d = __ldcg(P.dist + (size_t)q * P.n + v);
        const QDesc* qd = P.qd + q;
        const uint32_t h = (P.has_astar && __ldg(&qd->kind) == kASTAR)
                               ? heuristic(P.xy, P.xy_integral, v, __ldg(&qd->tx), __ldg(&qd->ty))
                               : 0u;
        const uint32_t dq = S.delta[q];
        key = dq ? bucket_of(d, h, dq) : S.cur[q] + 1u;
      } else {
        report_bad(P.sync, 42u, v, q);
        has = false;
      }
    }
    insert_warp(P, S, B, 0, has, false, v, d, key, q, C);
  }
}

template <bool ELL>
__device__ __forceinline__ void delta_body(const Params& P) {
  extern __shared__ __align__(16) unsigned char og_dyn_smem[];
  __shared__ Smem S;
  Bins B;
  B.e[0] = reinterpret_cast<uint2*>(og_dyn_smem);
  B.e[1] = B.e[0] + P.bin_cap;
  B.q[0] = reinterpret_cast<uint16_t*>(B.e[1] + P.bin_cap);
  B.q[1] = B.q[0] + P.bin_cap;
  for (uint32_t q = threadIdx.x; q < P.nq; q += kBlock) S.delta[q] = __ldg(&P.qd[q].delta);
  Cnt C = {0, 0, 0, 0, 0, 0, 0};
  uint32_t fused = 0;
  uint32_t bar = 0;
  if (threadIdx.x == 0) S.t_front = S.t_fused = S.t_bar = S.t_hub = 0ull;
  grid_barrier(P, S, bar, kPhPrologue);
  for (;;) {
    const uint32_t phase = S.phase;
    if (phase == kPhStop || (S.err & kErrFatal)) break;
    if (phase == kPhRelax) relax_phase<ELL>(P, S, B, C, fused);
    else if (phase == kPhRedistMin) redist_min_phase(P);
    else if (phase == kPhRedistMove) redist_move_phase(P);
    else if (phase == kPhApply) lazy_apply_phase(P, S, B, C);
    else if (phase == kPhBig) {
      if constexpr (!ELL) big_phase(P, S, B, C);  // ELL rows hold <= 8 edges: no hubs
    }
    grid_barrier(P, S, bar, phase);
  }
  const uint32_t lane = threadIdx.x & 31;
  uint32_t vals[7] = {C.items, C.stale, C.relax, C.improved, C.local, C.global, C.ovf};
  const int idx[7] = {kStItems, kStStale, kStRelax, kStImproved, kStLocal, kStGlobal, kStOvf};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const uint32_t s = warp_sum(vals[k]);
    if (lane == 0 && s) atomicAdd(&P.stats->v[idx[k]], (unsigned long long)s);
  }
  if (threadIdx.x == 0) {
    if (fused) atomicAdd(&P.stats->v[kStFused], (unsigned long long)fused);
    atomicAdd(&P.stats->v[kStTFrontier], S.t_front);
    atomicAdd(&P.stats->v[kStTFused], S.t_fused);
    atomicAdd(&P.stats->v[kStTBarrier], S.t_bar);
    atomicAdd(&P.stats->v[kStTHub], S.t_hub);
  }
}

// The persistent kernel, one instantiation per adjacency layout (CSR offsets + edge
// array for any graph; ELL-8 rows for graphs of degree at most 8).
extern "C" __global__ void __launch_bounds__(kBlock, 3) og_delta_kernel(Params P) {
  delta_body<false>(P);
}
extern "C" __global__ void __launch_bounds__(kBlock, 3) og_delta_ell_kernel(Params P) {
  delta_body<true>(P);
}

// dist[slot][*] = unreachable for the listed slots (blockIdx.y indexes the slot list).
extern "C" __global__ void og_fill_kernel(uint32_t* dist, uint32_t n, const uint32_t* slots) {
  const uint32_t q = slots ? slots[blockIdx.y] : blockIdx.y;
  uint32_t* d = dist + (size_t)q * n;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // align to 16 bytes for vector stores
  const uint32_t mis = (uint32_t)(((uintptr_t)d >> 2) & 3u);
  const uint32_t headn = mis ? min(n, 4u - mis) : 0u;
  if (i < headn) d[i] = kInf;
  const uint32_t body = (n - headn) / 4u;
  uint4* d4 = reinterpret_cast<uint4*>(d + headn);
  for (size_t k = i; k < body; k += stride) d4[k] = make_uint4(kInf, kInf, kInf, kInf);
  for (size_t k = headn + 4ull * body + i; k < n; k += stride) d[k] = kInf;
}

// Starts the listed queries: dist[src] = 0 and the start vertex in its first bucket
// (the initial state of the Section 3.2 figures: the source at distance 0, alone in its
// bucket).
extern "C" __global__ void og_init_kernel(Params P, const uint32_t* slots, uint32_t nslots) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const uint32_t q = slots ? slots[t] : t;
  const QDesc d = P.qd[q];
  P.dist[(size_t)q * P.n + d.src] = 0u;
  const uint32_t h0 = d.kind == kASTAR ? heuristic(P.xy, P.xy_integral, d.src, d.tx, d.ty) : 0u;
  const uint32_t key0 = d.delta ? bucket_of(0u, h0, d.delta) : 0u;
  uint32_t* cnts = P.counts + (size_t)q * P.B;
  for (uint32_t k = 0; k < P.B; ++k) cnts[k] = 0u;
  cnts[key0 & P.Bmask] = 1u;
  P.ring[((size_t)q * P.B + (key0 & P.Bmask)) * P.cap] = make_uint2(d.src, 0u);
  QState s;
  s.cur = key0;
  s.head = 0;
  s.tail = 1;
  s.active = 1;
  s.ovf_n = 0;
  s.ovf_min = kInf;
  s.ovf_sel = 0;
  s.redist = 0;
  s.ovf_n2 = 0;
  s.ovf_min2 = kInf;
  s.redist_min = kInf;
  s.no_exit = 0;
  s.result = kInf;
  s.aborted = 0;
  s.pad[0] = s.pad[1] = 0;
  P.qs[q] = s;
}

// Graph upload helpers: interleave {neighbor, weight}, validate neighbors, weight range.
extern "C" __global__ void og_interleave_kernel(const uint32_t* nbr, const uint32_t* w,
                                                uint2* adj, size_t m, uint32_t n,
                                                uint32_t* flags /* [0]=bad, [1]=min, [2]=max */) {
  uint32_t bad = 0, mn = kInf, mx = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t v = nbr[i], x = w[i];
    bad |= v >= n;
    mn = min(mn, x);
    mx = max(mx, x);
    adj[i] = make_uint2(v, x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad |= __shfl_xor_sync(FULL, bad, o);
    mn = min(mn, __shfl_xor_sync(FULL, mn, o));
    mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, 1u);
    atomicMin(flags + 1, mn);
    atomicMax(flags + 2, mx);
  }
}

}  // namespace og

namespace og {

// ELL-8 rows from CSR: row v holds v's out-edges in its first deg(v) slots and the
// neighbor marker 0xFFFFFFFF in the rest (only built for graphs of degree <= 8).
extern "C" __global__ void og_ell_kernel(const uint32_t* off, const uint2* adj, uint4* ell,
                                         uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t beg = off[v], end = off[v + 1];
    uint2 e[kEllWidth];
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k)
      e[k] = beg + k < end ? adj[beg + k] : make_uint2(kNone, 0u);
    uint4* r = ell + (size_t)v * 4;
    r[0] = make_uint4(e[0].x, e[0].y, e[1].x, e[1].y);
    r[1] = make_uint4(e[2].x, e[2].y, e[3].x, e[3].y);
    r[2] = make_uint4(e[4].x, e[4].y, e[5].x, e[5].y);
    r[3] = make_uint4(e[6].x, e[6].y, e[7].x, e[7].y);
  }
}

cudaError_t launch_ell(const uint32_t* off, const uint2* adj, uint4* ell, uint32_t n, int sms,
                       cudaStream_t st) {
  og_ell_kernel<<<sms * 8, 256, 0, st>>>(off, adj, ell, n);
  return cudaGetLastError();
}

// Host-side launchers (the kernels above are only launched through these).
cudaError_t launch_delta(const Params& P, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<Params*>(&P)};
  const void* k = P.ell ? (const void*)og_delta_ell_kernel : (const void*)og_delta_kernel;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBlock), args, smem, st);
}

cudaError_t delta_occupancy(int* blocks_per_sm, size_t smem, bool ell) {
  const void* k = ell ? (const void*)og_delta_ell_kernel : (const void*)og_delta_kernel;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBlock, smem);
}

cudaError_t launch_fill(uint32_t* dist, uint32_t n, const uint32_t* slots, uint32_t nslots,
                        int sms, cudaStream_t st) {
  if (nslots == 0) return cudaSuccess;
  const uint32_t per = (n / 4 + 255) / 256;
  uint32_t gx = per < 1 ? 1 : per;
  const uint32_t cap = (uint32_t)sms * 8u;
  if (gx > cap) gx = cap;
  og_fill_kernel<<<dim3(gx, nslots), 256, 0, st>>>(dist, n, slots);
  return cudaGetLastError();
}

cudaError_t launch_init(const Params& P, const uint32_t* slots, uint32_t nslots, cudaStream_t st) {
  if (nslots == 0) return cudaSuccess;
  og_init_kernel<<<(nslots + 127) / 128, 128, 0, st>>>(P, slots, nslots);
  return cudaGetLastError();
}

cudaError_t launch_interleave(const uint32_t* nbr, const uint32_t* w, uint2* adj, size_t m,
                              uint32_t n, uint32_t* flags, int sms, cudaStream_t st) {
  og_interleave_kernel<<<sms * 4, 256, 0, st>>>(nbr, w, adj, m, n, flags);
  return cudaGetLastError();
}

}  // namespace og

// ---- allocation-free entry point ----------------------------------------------------------
// og_sssp_delta_noalloc runs the same round-synchronous kernel as og_sssp_delta, but its
// scratch (query cursor, barrier words, counters, bucket ring and overflow pile) lives in
// the fixed device array below instead of memory the library allocates.  It serves
// callers that cannot call cudaMalloc: code inside a host application whose allocator has
// already claimed the device memory, code on a path where cudaMalloc's implicit device
// synchronisation is not acceptable, and code that must not meet an out-of-memory error
// after start-up.  The array is reserved on every GPU that loads the library, for the
// life of the process.
#include <mutex>

#include "og.h"

namespace og {

constexpr size_t kNoAllocBytes = 64ull << 20;           // scratch array size (64 MiB)
constexpr uint32_t kNoAllocMaxN = 1u << 20;             // largest graph accepted
constexpr size_t kNoAllocHeader = 4096;                 // state words before the arena
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char og_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_occ[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};
}  // namespace

}  // namespace og

extern "C" int og_sssp_delta_noalloc(const uint32_t* offsets, const uint32_t* edges, uint32_t n,
                                     uint64_t m, uint32_t src, uint32_t delta,
                                     uint32_t* dist_out, void* stream) {
  using namespace og;
  if (!offsets || !dist_out || (m && !edges) || n == 0 || src >= n || delta == 0)
    return OG_E_INVALID;
  if (n > kNoAllocMaxN || m >= 0xFFFFFFFFull) return OG_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return OG_E_CUDA;
  }
  const size_t smem = 2 * (size_t)2048 * (sizeof(uint2) + sizeof(uint16_t));
  void* base = nullptr;
  {
    // Set-up, once per device with that device current: the device address of the array
    // (host code only ever sees a host-side stand-in for the symbol).
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, og_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return OG_E_CUDA;
      }
      int occ = 0, sms = 0;
      if (delta_occupancy(&occ, smem, false) != cudaSuccess || occ < 1 ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return OG_E_CUDA;
      }
      g_noalloc_occ[dev] = occ;
      g_noalloc_sms[dev] = sms;
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  // Header: Sync | Stats | QDesc | QState | frontier prefix | ring counters.
  Sync* sync = reinterpret_cast<Sync*>(b);
  Stats* stats = reinterpret_cast<Stats*>(b + 256);
  QDesc* qd = reinterpret_cast<QDesc*>(b + 512);
  QState* qs = reinterpret_cast<QState*>(b + 768);
  uint32_t* pref = reinterpret_cast<uint32_t*>(b + 1024);
  uint32_t* counts = reinterpret_cast<uint32_t*>(b + 2048);
  uint32_t max_w = 0xFFFFFFFFu;  // unknown without a pass over the edges: widest ring
  uint32_t B = kMaxRing;
  if (delta >= max_w / 2) B = 2;
  const uint64_t arena = (kNoAllocBytes - kNoAllocHeader) / sizeof(uint2);
  const uint32_t cap = (uint32_t)(arena / 2 / B);
  const uint32_t ocap = (uint32_t)(arena / 4);
  uint2* ring = reinterpret_cast<uint2*>(b + kNoAllocHeader);
  uint2* ovf = ring + (size_t)B * cap;

  QDesc hq;
  memset(&hq, 0, sizeof(hq));
  hq.src = src;
  hq.dst = kNone;
  hq.delta = delta;
  hq.kind = kSSSP;
  Params P{};
  P.off = offsets;
  P.adj = reinterpret_cast<const uint2*>(edges);
  P.xy = nullptr;
  P.n = n;
  P.dist = dist_out;
  P.qd = qd;
  P.qs = qs;
  P.ring = ring;
  P.counts = counts;
  P.ovf = ovf;
  P.fr_pref = pref;
  P.sync = sync;
  P.stats = stats;
  P.nq = 1;
  P.B = B;
  P.Bmask = B - 1;
  P.cap = cap;
  P.ocap = ocap;
  P.T = 1024;
  P.tile = 128;
  P.bin_cap = 2048;
  P.max_rounds = 0xFFFFFFFFu;
  P.has_astar = 0;
  P.spin_ns = 2000000000ull;
  // Calls share the array: the state words start from zero on every call (two calls
  // that overlap on the GPU would race on it).
  if (cudaMemsetAsync(b, 0, kNoAllocHeader, st) != cudaSuccess ||
      cudaMemcpyAsync(qd, &hq, sizeof(hq), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      launch_fill(dist_out, n, nullptr, 1, g_noalloc_sms[dev], st) != cudaSuccess ||
      launch_init(P, nullptr, 1, st) != cudaSuccess ||
      launch_delta(P, g_noalloc_sms[dev] * g_noalloc_occ[dev], smem, st) != cudaSuccess) {
    cudaGetLastError();
    return OG_E_CUDA;
  }
  Sync hs;
  QState hqs;
  if (cudaMemcpyAsync(&hs, sync, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&hqs, qs, sizeof(hqs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return OG_E_CUDA;
  }
  if (hs.err & kErrTimeout) return OG_E_TIMEOUT;
  if (hqs.aborted) return OG_E_ARENA;
  if (hs.err & kErrSat) return OG_E_OVERFLOW;
  return OG_OK;
}
