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
#include <stddef.h>

#include "og_device.cuh"

namespace og {

struct Smem {
  uint32_t cur[kMaxQ];     // current bucket per query
  uint32_t delta[kMaxQ];
  uint32_t head[kMaxQ];    // frontier start in the current ring slot
  uint32_t pref[kMaxQ + 1];// frontier prefix sums (scratch in the decider)
  uint32_t binN[3];        // CTA-local bin fill counts (a level reads one, fills the
                           // next and clears the third)
  uint32_t obN;            // entries staged in the outbox this round
  uint32_t grab;
  uint32_t last;
  uint32_t phase;
  uint32_t err;
  uint32_t f_active, f_redist, f_pull;
  uint32_t d_err, d_big, d_lz;  // decider: control words read once by thread 0
  uint32_t wtmp[kWarps + 1];
  uint32_t lb_pos[kBlock + 1];  // CTA-wide expansion: edge prefix sums of the entries
  uint32_t lb_beg[kBlock], lb_g[kBlock], lb_q[kBlock];
  unsigned long long t_front, t_fused, t_bar, t_hub;  // per-CTA phase time (thread 0)
};

struct Bins {
  uint2* e[2];
  uint16_t* q[2];
  uint4* ob;     // outbox: {vertex, distance, query, bucket} of later buckets, this round
};

// The CTA-local bin a level fills: its entries, their queries and its fill count; and
// the CTA's outbox, where entries bound for the global buckets wait (ob null: such
// entries go to their buckets at once).
struct BinOut {
  uint2* e;
  uint16_t* q;
  uint32_t* n;
  uint4* ob;
  uint32_t* obn;
};

struct Cnt {
  uint32_t items, stale, relax, improved, local, global, ovf;
};

// Appends the improved vertices of a warp (lanes with ins) to their buckets: the CTA-local
// bin when the bucket is the query's current one and fusion is on, else the ring slot of
// the bucket (warp-aggregated: lanes with the same (query, slot) share one atomicAdd),
// else the overflow pile.  Must be called by all 32 lanes.
__device__ __forceinline__ void insert_warp(const Params& P, Smem& S, const BinOut& O,
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
    if ((int)lane == leader) base = atomicAdd(O.n, (uint32_t)__popc(lm));
    base = __shfl_sync(FULL, base, leader);
    if (dest == 1) {
      const uint32_t pos = base + __popc(lm & lanemask_lt());
      if (pos < P.bin_cap) {
        O.e[pos] = make_uint2(v, nd);
        O.q[pos] = (uint16_t)q;
        C.local++;
      } else {
        dest = 2;  // bin full: the entry goes to the global current bucket
      }
    }
  }
  if (O.ob) {
    // Entries for the global buckets wait in the outbox (one shared-memory atomic per
    // warp), so the warp does not wait for a global append here.
    const unsigned sm = __ballot_sync(FULL, dest >= 2);
    if (sm) {
      const int leader = __ffs(sm) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(O.obn, (uint32_t)__popc(sm));
      base = __shfl_sync(FULL, base, leader);
      if (dest >= 2) {
        const uint32_t pos = base + __popc(sm & lanemask_lt());
        if (pos < kOutbox) {
          O.ob[pos] = make_uint4(v, nd, q, key);
          dest = 0;
        }
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

// Relaxes up to K already-loaded edges per lane: nd = g + w (saturating), atomicMin on
// dist[v]; an improvement is inserted eagerly into bucket floor((nd + h) / Delta).  All K
// atomics are issued before any insert, so a lane keeps K independent memory operations
// in flight instead of paying one round trip per edge.
template <int K>
__device__ __forceinline__ void relax_edges(const Params& P, Smem& S, const BinOut& O,
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
    insert_warp(P, S, O, ins, allow_local, ew[k].x, nd[k], key, q[k], C);
  }
}

// CSR edges: the K neighbor loads are issued together, then relax_edges.
template <int K>
__device__ __forceinline__ void relax_batch(const Params& P, Smem& S, const BinOut& O,
                                            bool allow_local, const bool (&ok)[K],
                                            const uint32_t (&e)[K], const uint32_t (&g)[K],
                                            const uint32_t (&q)[K], Cnt& C) {
  uint2 ew[K];
#pragma unroll
  for (int k = 0; k < K; ++k) ew[k] = ok[k] ? __ldg(P.adj + e[k]) : make_uint2(0u, 0u);
  relax_edges<K>(P, S, O, allow_local, ok, ew, g, q, C);
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
__device__ __forceinline__ void expand_warp(const Params& P, Smem& S, const BinOut& O,
                                            bool allow_local, bool has, uint32_t u,
                                            uint32_t g, uint32_t q, Cnt& C) {
  const uint32_t lane = threadIdx.x & 31;
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
      relax_batch<kHeavyBatch>(P, S, O, allow_local, ok, ee, gg, qq, C);
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
    relax_batch<kLightBatch>(P, S, O, allow_local, ok, ee, gg, qq, C);
  }
}

// Stages entries of later buckets (lanes with bits in gm; their vertex, distance and
// bucket in ew / nd / key) in the CTA's outbox, which reaches the global buckets once at
// the end of the round (flush_outbox), so the level that produced them does not wait for
// a global atomic.  Entries that do not fit go to their buckets directly.  All 32 lanes.
template <bool ASTAR>
__device__ __forceinline__ void stage_later(const Params& P, Smem& S, const Bins& B,
                                            const BinOut& O, unsigned gm,
                                            const uint2 (&ew)[kEllWidth],
                                            const uint32_t (&nd)[kEllWidth], uint32_t q,
                                            bool astar, Cnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t cq = S.cur[q], dl = S.delta[q];
  uint32_t key[kEllWidth];  // the bucket of each staged entry, as expand_rows chose it
#pragma unroll
  for (int k = 0; k < kEllWidth; ++k) {
    const uint32_t h = (ASTAR && astar && ((gm >> k) & 1u))
                           ? heuristic(P.xy, P.xy_integral, ew[k].x, __ldg(&P.qd[q].tx),
                                       __ldg(&P.qd[q].ty))
                           : 0u;
    const uint32_t kk = dl ? bucket_of(nd[k], h, dl) : cq + 1u;
    key[k] = kk < cq ? cq : kk;
  }
  const uint32_t ng = __popc(gm);
  uint32_t incl = ng;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&S.obN, incl);
  base = __shfl_sync(FULL, base, 31);
  uint32_t pos = base + incl - ng;
  unsigned dm = 0;  // entries the outbox could not take
#pragma unroll
  for (int k = 0; k < kEllWidth; ++k) {
    if ((gm >> k) & 1u) {
      if (pos < kOutbox) B.ob[pos] = make_uint4(ew[k].x, nd[k], q, key[k]);
      else dm |= 1u << k;
      ++pos;
    }
  }
  // One entry per lane per pass (selected by index, so insert_warp is expanded once).
  while (__any_sync(FULL, dm != 0u)) {
    const bool has = dm != 0u;
    uint32_t v = 0, dv = 0, kv = 0;
    if (has) {
      const int j = __ffs(dm) - 1;
      dm &= dm - 1u;
#pragma unroll
      for (int k = 0; k < kEllWidth; ++k) {
        if (k == j) {
          v = ew[k].x;
          dv = nd[k];
          kv = key[k];
        }
      }
    }
    const BinOut direct = {O.e, O.q, O.n, nullptr, nullptr};
    insert_warp(P, S, direct, has, false, v, dv, kv, q, C);
  }
}

// Moves the outbox into the global buckets (ring slot or overflow pile, warp-aggregated).
// Called by every thread of the CTA; leaves the outbox empty.
__device__ void flush_outbox(const Params& P, Smem& S, const Bins& B, Cnt& C) {
  __syncthreads();
  const uint32_t n = min(S.obN, kOutbox);
  const uint32_t lim = (n + 31u) & ~31u;
  const BinOut direct = {B.e[0], B.q[0], &S.binN[0], nullptr, nullptr};  // never the bin
  for (uint32_t k = threadIdx.x; k < lim; k += kBlock) {
    const bool has = k < n;
    uint4 en = make_uint4(0, 0, 0, 0);
    if (has) en = B.ob[k];
    insert_warp(P, S, direct, has, false, en.x, en.y, en.w, en.z, C);
  }
  __syncthreads();
  if (threadIdx.x == 0) S.obN = 0;
}

// Relaxes one loaded ELL row per lane (lanes with live; g = the row's vertex distance):
// issues the row's atomicMins, then sends improved vertices of the current bucket to
// the CTA's bin with one warp-wide scan and one shared-memory atomic, and those of later
// buckets to the outbox.  All 32 lanes.
template <bool ASTAR>
__device__ __forceinline__ void relax_row(const Params& P, Smem& S, const Bins& B,
                                          const BinOut& O, bool allow_local, bool live,
                                          const uint2 (&ew)[kEllWidth], uint32_t g,
                                          uint32_t q, Cnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* dq = P.dist + (size_t)q * P.n;
  unsigned okm = 0;
  uint32_t nd[kEllWidth];
#pragma unroll
  for (int k = 0; k < kEllWidth; ++k) {
    const bool ok = live && ew[k].x != kNone;
    okm |= (ok ? 1u : 0u) << k;
    const unsigned long long sum = (unsigned long long)g + ew[k].y;
    nd[k] = sum >= kSat ? kSat : (uint32_t)sum;
    if (ok && sum >= kSat) atomicOr(&P.sync->err, kErrSat);
  }
  if (P.precheck) {
    uint32_t seen[kEllWidth];
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k) seen[k] = ((okm >> k) & 1u) ? ld_cached(dq + ew[k].x) : 0u;
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k)
      if (nd[k] >= seen[k]) okm &= ~(1u << k);
  }
  uint32_t old[kEllWidth];
#pragma unroll
  for (int k = 0; k < kEllWidth; ++k)
    old[k] = ((okm >> k) & 1u) ? atomicMin(dq + ew[k].x, nd[k]) : 0u;
  const uint32_t cq = S.cur[q], dl = S.delta[q];
  // A* (priority g + h): the heuristic is needed only for the improved edges' buckets.
  const bool astar = ASTAR && P.has_astar && live && __ldg(&P.qd[q].kind) == kASTAR;
  unsigned lm = 0, gm = 0;
#pragma unroll
  for (int k = 0; k < kEllWidth; ++k) {
    const bool ins = ((okm >> k) & 1u) && nd[k] < old[k];
    const uint32_t h = (astar && ins) ? heuristic(P.xy, P.xy_integral, ew[k].x,
                                                  __ldg(&P.qd[q].tx), __ldg(&P.qd[q].ty))
                                      : 0u;
    // Delta 0 marks a Bellman-Ford query: the next round's bucket, whatever the distance.
    uint32_t kk = dl ? bucket_of(nd[k], h, dl) : cq + 1u;
    if (ins && kk < cq) {  // only with an inconsistent A* heuristic: clamp, no early exit
      kk = cq;
      P.qs[q].no_exit = 1u;
    }
    const bool loc = ins && allow_local && kk == cq;
    lm |= (loc ? 1u : 0u) << k;
    gm |= ((ins && !loc) ? 1u : 0u) << k;
    if (ins && P.prefetch) prefetch_row(P.ell, P.off, ew[k].x);
  }
  C.relax += __popc(okm);
  C.improved += __popc(lm | gm);
  if (__any_sync(FULL, lm != 0u)) {
    const uint32_t nl = __popc(lm);
    uint32_t incl = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, incl, o);
      if ((int)lane >= o) incl += t;
    }
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(O.n, incl);
    base = __shfl_sync(FULL, base, 31);
    uint32_t pos = base + incl - nl;
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k) {
      if ((lm >> k) & 1u) {
        if (pos < P.bin_cap) {
          O.e[pos] = make_uint2(ew[k].x, nd[k]);
          O.q[pos] = (uint16_t)q;
          C.local++;
        } else {
          gm |= 1u << k;  // bin full: the entry goes to the global current bucket
        }
        ++pos;
      }
    }
  }
  if (__any_sync(FULL, gm != 0u)) stage_later<ASTAR>(P, S, B, O, gm, ew, nd, q, astar, C);
}

// Expands the bucket entries held by a warp (one per lane with has) on the ELL layout:
// the lane reads its vertex's whole row (up to 8 {neighbor, weight} pairs, 64 bytes)
// together with the stale check, then relaxes it (relax_row), so a level costs two
// dependent memory round trips.  All 32 lanes.
template <bool ASTAR>
__device__ __forceinline__ void expand_rows(const Params& P, Smem& S, const Bins& B,
                                            const BinOut& O, bool allow_local, bool has,
                                            uint32_t u, uint32_t g, uint32_t q, Cnt& C) {
  uint2 ew[kEllWidth];
  uint32_t d = 0;
  if (has) {
    C.items++;
    d = __ldcg(P.dist + (size_t)q * P.n + u);
    load_row(P.ell, u, ew);
  } else {
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k) ew[k] = make_uint2(kNone, 0u);
  }
  const bool live = has && d == g;
  if (has && !live) C.stale++;
  relax_row<ASTAR>(P, S, B, O, allow_local, live, ew, g, q, C);
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
__device__ __forceinline__ void expand_cta(const Params& P, Smem& S, const BinOut& O,
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
    relax_batch<kLightBatch>(P, S, O, allow_local, ok, ee, gg, qq, C);
  }
  __syncthreads();  // the lb arrays are refilled by the next call
}

constexpr uint32_t kQStateWords = sizeof(QState) / 4;
static_assert(kQStateWords <= 32 && sizeof(QState) % 4 == 0, "QState fits one warp load");
#define QS_WORD(f) ((uint32_t)(offsetof(QState, f) / 4))

// Run by the CTA that arrives last at a grid barrier, before it releases the others:
// advances every query's bucket cursor and publishes the next phase and frontier.
// Every value a decision depends on is read once -- the control words by thread 0 into
// shared memory, each query's words by lane 0 of its warp and shuffled to the others --
// so a word that changes while the decider runs (the error word, when a waiting CTA
// times out) can never send the lanes of a warp down different paths.  A query's state
// words come in one warp-wide load (every other CTA has arrived: they no longer change).
__device__ void decide(const Params& P, Smem& S, uint32_t done_phase) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Sync* sy = P.sync;
  if (tid == 0) {
    S.d_err = ld_relaxed(&sy->err);
    S.d_big = (uint32_t)(ld_relaxed64(&sy->big_word) >> 32);
    S.d_lz = ld_relaxed(&sy->lz_n);
    S.f_active = 0;
    S.f_redist = 0;
    S.f_pull = 0;
  }
  __syncthreads();
  const uint32_t err = S.d_err;
  const bool fatal = (err & kErrFatal) != 0;
  if (done_phase == kPhRelax && !fatal && S.d_big > 0u) {
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
  if (done_phase == kPhRelax && !fatal && P.lazy && S.d_lz > 0u) {
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
  for (uint32_t q = warp; q < P.nq; q += kWarps) {
    QState* qs = P.qs + q;
    uint32_t* cnts = P.counts + (size_t)q * P.B;
    // The query's state in one round trip: lane i holds word i of its QState.
    const uint32_t snap = lane < kQStateWords
                              ? __ldcg(reinterpret_cast<const uint32_t*>(qs) + lane) : 0u;
    auto F = [&](uint32_t w) -> uint32_t { return __shfl_sync(FULL, snap, (int)w); };
    uint32_t active = F(QS_WORD(active));
    uint32_t size = 0;
    if (active && F(QS_WORD(aborted))) {
      active = 0;
      if (lane == 0) {
        qs->active = 0;
        qs->redist = 0;
        qs->result = kInf;
      }
    }
    if (active && !fatal) {
      uint32_t cur = F(QS_WORD(cur)), head = F(QS_WORD(head)), tail = F(QS_WORD(tail));
      uint32_t redist = F(QS_WORD(redist));
      // A pull phase consumed the frontier of the queries it pulled: for them it ends the
      // round like a relax phase; the others keep their frontier for the relax phase.
      if (done_phase == kPhRelax || (done_phase == kPhPull && F(QS_WORD(pull)))) {
        const uint32_t c = cur & P.Bmask;
        const uint32_t cnt = min(warp_ld(cnts + c), P.cap);
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
          const uint32_t ovf_n = F(QS_WORD(ovf_n)), ovf_min = F(QS_WORD(ovf_min));
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
            tail = min(warp_ld(cnts + (next & P.Bmask)), P.cap);
          }
        }
      } else if (done_phase == kPhRedistMin && redist) {
        const uint32_t nc = F(QS_WORD(redist_min));
        if (nc == kInf) {  // every pile entry was out of date and the ring is empty
          active = 0;
          redist = 0;
          if (lane == 0) qs->ovf_n = 0;
        } else {
          cur = nc;
        }
      } else if (done_phase == kPhRedistMove && redist) {
        const uint32_t sel = F(QS_WORD(ovf_sel)), n2 = F(QS_WORD(ovf_n2));
        const uint32_t min2 = F(QS_WORD(ovf_min2));
        if (lane == 0) {
          qs->ovf_sel = sel ^ 1u;
          qs->ovf_n = n2;
          qs->ovf_min = min2;
        }
        redist = 0;
        head = 0;
        tail = min(warp_ld(cnts + (cur & P.Bmask)), P.cap);
      }
      const QDesc* qd = P.qd + q;
      const uint32_t kind = __ldg(&qd->kind);
      const uint32_t dst = __ldg(&qd->dst);
      if (active && !redist && (kind == kPPSP || kind == kASTAR) && !F(QS_WORD(no_exit))) {
        // Stop rule of Section 6.1 (PPSP): entering bucket i with i * Delta >= the best
        // distance to the target found so far.
        const uint32_t dt = warp_ld(P.dist + (size_t)q * P.n + dst);
        if (dt != kInf && (unsigned long long)cur * __ldg(&qd->delta) >= dt) active = 0;
      }
      const uint32_t res = (!active && dst < P.n) ? warp_ld(P.dist + (size_t)q * P.n + dst) : 0u;
      // Direction optimisation: an SSSP / wBFS query whose frontier exceeds n / pull_div
      // pulls this round instead of pushing.
      const bool pull = P.pull_div && active && !redist && kind == kSSSP &&
                        __ldg(&qd->delta) != 0u && tail - head > P.n / P.pull_div;
      if (lane == 0) {
        qs->cur = cur;
        qs->head = head;
        qs->tail = tail;
        qs->redist = redist;
        qs->active = active;
        qs->pull = pull ? 1u : 0u;
        if (!active) qs->result = res;
        if (active) S.f_active = 1;
        if (redist) S.f_redist = 1;
        if (pull) S.f_pull = 1;
      }
      size = (active && !redist && !pull) ? tail - head : 0u;
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
    if (next == kPhRelax && S.f_pull) next = kPhPull;  // pulls first, then the pushes
    if (next == kPhRelax || next == kPhPull) {
      if (sy->rounds >= P.max_rounds) next = kPhStop;
      else sy->rounds = sy->rounds + 1;
    }
    sy->phase = next;
    sy->work = 0;
    sy->total = S.pref[P.nq];
    sy->any_active = S.f_active;
    P.stats->v[kStRounds] += (next == kPhRelax || next == kPhPull) ? 1ull : 0ull;
    if (done_phase == kPhRedistMove) P.stats->v[kStRedist] += 1ull;
  }
}
#undef QS_WORD

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
    // The acquire that observed the new generation orders these after the decider's
    // writes.
    S.phase = ld_relaxed(&P.sync->phase);
    S.err = ld_relaxed(&P.sync->err);
    S.t_bar += gtimer() - t_in;
  }
  __syncthreads();
  ++bar;
}

// One round for all active queries: frontier pass over the global current buckets, then
// the CTA-local fusion loop (Section 3.3): the CTA's warps drain its local bin together,
// one level per iteration, with block-level synchronisation only.  Entry buffers
// alternate between two bins; their fill counts rotate over three words, so the count a
// level fills was cleared during the level before and one barrier per level suffices.
// On the ELL layout with fusion, entries of later buckets collect in the outbox and
// reach the global buckets at the end of the round.
template <bool ELL, bool ASTAR>
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
    S.binN[2] = 0;
    S.obN = 0;
  }
  __syncthreads();
  const uint32_t total = S.pref[P.nq];
  const bool fuse = P.T != 0;
  const BinOut first = {B.e[0], B.q[0], &S.binN[0], B.ob, &S.obN};
  const uint64_t t_start = tid == 0 ? gtimer() : 0ull;
  // Tiles are claimed one ahead: the claim of the next tile travels while this one is
  // expanded.
  uint32_t nxt = 0;
  if (tid == 0) nxt = atomicAdd(&P.sync->work, P.tile);
  for (;;) {
    if (tid == 0) S.grab = nxt;
    __syncthreads();
    const uint32_t base = S.grab;
    __syncthreads();
    if (base >= total) break;
    if (tid == 0) nxt = atomicAdd(&P.sync->work, P.tile);
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
      if constexpr (ELL) expand_rows<ASTAR>(P, S, B, first, fuse, has, u, g, q, C);
      else expand_cta(P, S, first, fuse, has, u, g, q, C);
    }
    __syncthreads();
    if (S.obN >= kOutbox / 2) flush_outbox(P, S, B, C);  // uniform: read after a barrier
  }
  const uint64_t t_mid = tid == 0 ? gtimer() : 0ull;
  if (tid == 0) S.t_front += t_mid - t_start;
  if (!fuse) {
    flush_outbox(P, S, B, C);
    return;
  }
  int in = 0;    // entry buffer the level reads
  int cin = 0;   // count word of that buffer
  for (;;) {
    __syncthreads();
    if (S.obN >= kOutbox / 2) flush_outbox(P, S, B, C);  // uniform: read after a barrier
    const uint32_t nin = S.binN[cin];
    if (nin == 0) break;
    const int cout = cin == 2 ? 0 : cin + 1;
    // The third count word was read at the top of the previous level and is filled by
    // the next one: clear it now.
    if (tid == 0) S.binN[cout == 2 ? 0 : cout + 1] = 0;
    const uint32_t cnt = min(nin, P.bin_cap);
    const uint32_t lim = (cnt + 31u) & ~31u;
    const BinOut O = {B.e[in ^ 1], B.q[in ^ 1], &S.binN[cout], B.ob, &S.obN};
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
        insert_warp(P, S, O, has, false, en.x, en.y, has ? S.cur[q] : 0u, q, C);
      }
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
      if constexpr (ELL) expand_rows<ASTAR>(P, S, B, O, true, has, en.x, en.y, q, C);
      else expand_warp(P, S, O, true, has, en.x, en.y, q, C);
    }
    in ^= 1;
    cin = cout;
    ++fused;
  }
  flush_outbox(P, S, B, C);
  __syncthreads();
  if (tid == 0) S.t_fused += gtimer() - t_mid;
}

// Overflow redistribution, step 1: the smallest bucket among live pile entries.
__device__ void redist_min_phase(const Params& P) {
  const uint32_t gtid = blockIdx.x * kBlock + threadIdx.x, gstride = gridDim.x * kBlock;
  for (uint32_t q = 0; q < P.nq; ++q) {
    QState* qs = P.qs + q;
    if (!warp_ld(&qs->redist)) continue;
    const uint32_t sel = warp_ld(&qs->ovf_sel);
    const uint32_t n = min(warp_ld(&qs->ovf_n), P.ocap);
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
    if (!warp_ld(&qs->redist)) continue;
    const uint32_t sel = warp_ld(&qs->ovf_sel);
    const uint32_t n = min(warp_ld(&qs->ovf_n), P.ocap);
    const uint32_t cur = warp_ld(&qs->cur);
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
  const BinOut O = {B.e[0], B.q[0], &S.binN[0], nullptr, nullptr};  // hub edges go global
  const uint64_t t_start = tid == 0 ? gtimer() : 0ull;
  for (uint32_t q = tid; q < P.nq; q += kBlock) S.cur[q] = __ldcg(&P.qs[q].cur);
  __syncthreads();
  const uint32_t nsub =
      min(warp_ld(reinterpret_cast<const uint32_t*>(&P.sync->big_word)), P.map_cap) * kBigSubs;
  uint32_t cnext = 0;
  if (lane == 0) cnext = atomicAdd(&P.sync->big_claim, 1u);
  for (;;) {
    const uint32_t c = __shfl_sync(FULL, cnext, 0);
    if (c >= nsub) break;
    // The next piece is claimed now; its number is only needed after this one, so the
    // claim's round trip overlaps the work below.
    if (lane == 0) cnext = atomicAdd(&P.sync->big_claim, 1u);
    // The piece's hub, read warp-uniformly (the loop bounds below enclose full-warp
    // collectives): its slot, then the record's six words in one warp-wide load.
    const uint32_t slot = warp_ld(P.big_map + c / kBigSubs);
    if (slot >= P.big_cap) continue;  // chunk of a hub that did not fit (expanded in place)
    static_assert(sizeof(BigItem) == 6 * sizeof(uint32_t), "BigItem is six words");
    const uint32_t w = lane < 6 ? __ldcg(reinterpret_cast<const uint32_t*>(P.big + slot) + lane)
                                : 0u;
    const uint32_t hg = __shfl_sync(FULL, w, 1), hq = __shfl_sync(FULL, w, 2);
    const uint32_t hb = __shfl_sync(FULL, w, 3), he = __shfl_sync(FULL, w, 4);
    const uint32_t cb = __shfl_sync(FULL, w, 5);
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
      relax_batch<kHeavyBatch>(P, S, O, false, ok, ee, gg, qq, C);
    }
  }
  __syncthreads();
  if (tid == 0) S.t_hub += gtimer() - t_start;
}

// Direction optimisation (the pull direction of Section 4.2's scheduling language): for
// a query whose frontier is large, every vertex not yet settled (its bucket >= the
// current one) scans its in-edges and takes the best distance through a neighbour of
// the current bucket, instead of the frontier pushing along its out-edges.  Each vertex
// is written only by the warp that owns it (no atomics on the destination); an
// improvement is inserted like a pushed one.  The in-edges of a warp's 32 vertices are
// walked together (flattened as in expand_warp), and each edge lowers its owner's best
// candidate with a shared-memory atomicMin.  Every current-bucket vertex acts as a source,
// a superset of the round's frontier, so the result is the push round's or better.
__device__ void pull_phase(const Params& P, Smem& S, const Bins& B, Cnt& C) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t q = tid; q < P.nq; q += kBlock) {
    S.cur[q] = __ldcg(&P.qs[q].cur);
    S.head[q] = __ldcg(&P.qs[q].pull);  // scratch: the query pulls this phase
  }
  if (tid == 0) S.obN = 0;
  __syncthreads();
  const BinOut O = {B.e[0], B.q[0], &S.binN[0], B.ob, &S.obN};  // never the bin
  uint32_t* wbest = S.lb_pos + warp * 32;  // best candidate of each lane's vertex
  const uint32_t gwarp = blockIdx.x * kWarps + warp, nwarp = gridDim.x * kWarps;
  for (uint32_t q = 0; q < P.nq; ++q) {
    if (!S.head[q]) continue;  // uniform: shared memory
    const uint32_t cur = S.cur[q], dl = S.delta[q];
    uint32_t* dq = P.dist + (size_t)q * P.n;
    for (uint32_t v0 = gwarp * 32; v0 < P.n; v0 += nwarp * 32) {
      const uint32_t v = v0 + lane;
      bool has = v < P.n;
      const uint32_t d = has ? __ldcg(dq + v) : 0u;
      if (has && d != kInf && d / dl < cur) has = false;  // settled in an earlier bucket
      uint32_t beg = 0, end = 0;
      if (has) {
        beg = __ldg(P.toff + v);
        end = __ldg(P.toff + v + 1);
      }
      wbest[lane] = has ? d : kInf;
      __syncwarp();
      const uint32_t deg = end - beg;
      uint32_t incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, o);
        if ((int)lane >= o) incl += t;
      }
      const uint32_t total = __shfl_sync(FULL, incl, 31);
      const uint32_t excl = incl - deg;
      for (uint32_t base = 0; base < total; base += 32 * kLightBatch) {
        bool ok[kLightBatch];
        uint32_t own[kLightBatch];
        uint2 iw[kLightBatch];
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
          ok[k] = idx < total;
          own[k] = pos;
          iw[k] = ok[k] ? __ldg(P.tadj + ob + (idx - oe)) : make_uint2(0u, 0u);
        }
        uint32_t du[kLightBatch];
#pragma unroll
        for (int k = 0; k < kLightBatch; ++k) du[k] = ok[k] ? __ldcg(dq + iw[k].x) : kInf;
#pragma unroll
        for (int k = 0; k < kLightBatch; ++k) {
          if (ok[k]) {
            C.relax++;
            if (du[k] != kInf && du[k] / dl == cur) {
              const unsigned long long sum = (unsigned long long)du[k] + iw[k].y;
              atomicMin(wbest + own[k], sum >= kSat ? kSat : (uint32_t)sum);
            }
          }
        }
      }
      __syncwarp();
      const uint32_t best = wbest[lane];
      const bool ins = has && best < d;
      if (ins) {
        if (best >= kSat) atomicOr(&P.sync->err, kErrSat);
        dq[v] = best;
        C.improved++;
      }
      __syncwarp();
      insert_warp(P, S, O, ins, false, v, best, ins ? best / dl : 0u, q, C);
    }
  }
  flush_outbox(P, S, B, C);
}

// The lazy bucket update's reduction (Section 3.1): every vertex marked this round is
// inserted once, into the bucket of its distance now (the minimum of the round's
// updates); its mark is cleared for the next round.
__device__ void lazy_apply_phase(const Params& P, Smem& S, const Bins& B, Cnt& C) {
  const uint32_t tid = threadIdx.x;
  const BinOut O = {B.e[0], B.q[0], &S.binN[0], nullptr, nullptr};  // inserts go global
  for (uint32_t q = tid; q < P.nq; q += kBlock) S.cur[q] = __ldcg(&P.qs[q].cur);
  __syncthreads();
  const uint32_t tn = min(warp_ld(&P.sync->lz_n), P.lz_cap);
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
    insert_warp(P, S, O, has, false, v, d, key, q, C);
  }
}

template <bool ELL, bool ASTAR>
__device__ __forceinline__ void delta_body(const Params& P) {
  extern __shared__ __align__(16) unsigned char og_dyn_smem[];
  __shared__ Smem S;
  Bins B;
  B.e[0] = reinterpret_cast<uint2*>(og_dyn_smem);
  B.e[1] = B.e[0] + P.bin_cap;
  B.q[0] = reinterpret_cast<uint16_t*>(B.e[1] + P.bin_cap);
  B.q[1] = B.q[0] + P.bin_cap;
  B.ob = reinterpret_cast<uint4*>(og_dyn_smem + bins_smem_bytes(P.bin_cap));
  for (uint32_t q = threadIdx.x; q < P.nq; q += kBlock) S.delta[q] = __ldg(&P.qd[q].delta);
  Cnt C = {0, 0, 0, 0, 0, 0, 0};
  uint32_t fused = 0;
  uint32_t bar = 0;
  if (threadIdx.x == 0) S.t_front = S.t_fused = S.t_bar = S.t_hub = 0ull;
  grid_barrier(P, S, bar, kPhPrologue);
  for (;;) {
    const uint32_t phase = S.phase;
    if (phase == kPhStop || (S.err & kErrFatal)) break;
    if (phase == kPhRelax) relax_phase<ELL, ASTAR>(P, S, B, C, fused);
    else if (phase == kPhRedistMin) redist_min_phase(P);
    else if (phase == kPhRedistMove) redist_move_phase(P);
    else if (phase == kPhApply) lazy_apply_phase(P, S, B, C);
    else if (phase == kPhPull) pull_phase(P, S, B, C);
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
// array for any graph; ELL-8 rows for graphs of degree at most 8).  On ELL rows, launches
// with an A* query use their own instantiation, so the heuristic's registers do not
// weigh on the others.
extern "C" __global__ void __launch_bounds__(kBlock, 3) og_delta_kernel(Params P) {
  delta_body<false, true>(P);
}
extern "C" __global__ void __launch_bounds__(kBlock, 3) og_delta_ell_kernel(Params P) {
  delta_body<true, false>(P);
}
extern "C" __global__ void __launch_bounds__(kBlock, 3) og_delta_ell_astar_kernel(Params P) {
  delta_body<true, true>(P);
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
  s.pull = 0;
  s.pad = 0;
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
static const void* delta_kernel_for(bool ell, bool astar) {
  if (!ell) return (const void*)og_delta_kernel;
  return astar ? (const void*)og_delta_ell_astar_kernel : (const void*)og_delta_ell_kernel;
}

cudaError_t launch_delta(const Params& P, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<Params*>(&P)};
  const void* k = delta_kernel_for(P.ell != nullptr, P.has_astar != 0);
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBlock), args, smem, st);
}

// CTAs per SM of the persistent kernel for a layout (the smaller of the two ELL
// instantiations, so one launch shape serves both); also sets its shared-memory limit.
cudaError_t delta_occupancy(int* blocks_per_sm, size_t smem, bool ell) {
  int best = 1 << 30;
  for (int a = 0; a < (ell ? 2 : 1); ++a) {
    const void* k = delta_kernel_for(ell, a == 1);
    cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kBlock, smem);
    if (e != cudaSuccess) return e;
    best = b < best ? b : best;
  }
  *blocks_per_sm = best;
  return cudaSuccess;
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

// The transpose (in-edges) for the pull direction: in-degrees counted with atomicAdd,
// then every edge u -> v scattered to v's in-edge list as {u, weight} (the order within a
// list does not matter: a pull takes the minimum over it).  One warp per source vertex.
extern "C" __global__ void og_indeg_kernel(const uint32_t* off, const uint2* adj, uint32_t n,
                                           uint32_t* deg) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t u = w0; u < n; u += nw)
    for (uint32_t e = off[u] + lane; e < off[u + 1]; e += 32) atomicAdd(deg + adj[e].x, 1u);
}
extern "C" __global__ void og_transpose_kernel(const uint32_t* off, const uint2* adj, uint32_t n,
                                               const uint32_t* toff, uint32_t* cursor,
                                               uint2* tadj) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t u = w0; u < n; u += nw)
    for (uint32_t e = off[u] + lane; e < off[u + 1]; e += 32) {
      const uint2 a = adj[e];
      const uint32_t pos = atomicAdd(cursor + a.x, 1u);
      tadj[toff[a.x] + pos] = make_uint2(u, a.y);
    }
}

cudaError_t launch_indeg(const uint32_t* off, const uint2* adj, uint32_t n, uint32_t* deg, int sms,
                         cudaStream_t st) {
  og_indeg_kernel<<<sms * 8, 256, 0, st>>>(off, adj, n, deg);
  return cudaGetLastError();
}
cudaError_t launch_transpose(const uint32_t* off, const uint2* adj, uint32_t n, const uint32_t* toff,
                             uint32_t* cursor, uint2* tadj, int sms, cudaStream_t st) {
  og_transpose_kernel<<<sms * 8, 256, 0, st>>>(off, adj, n, toff, cursor, tadj);
  return cudaGetLastError();
}

// Checks a caller's device CSR before any kernel walks it: offsets[0] = 0, offsets[n] = m,
// offsets non-decreasing (flags[0] bit 0) and every neighbor < n (bit 1).  Reads only
// offsets[0 .. n] and the m {neighbor, weight} pairs, so a malformed graph is reported
// instead of being followed.
extern "C" __global__ void og_check_csr_kernel(const uint32_t* off, const uint2* adj, uint32_t n,
                                               uint32_t m, uint32_t* flags) {
  uint32_t bad = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)n; i += stride) {
    const uint32_t a = off[i], b = off[i + 1];
    if (a > b) bad |= 1u;
    if (i == 0 && a != 0u) bad |= 1u;
    if (i + 1 == n && b != m) bad |= 1u;
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)m; i += stride)
    if (adj[i].x >= n) bad |= 2u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(FULL, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(flags, bad);
}

cudaError_t launch_check_csr(const uint32_t* off, const uint2* adj, uint32_t n, uint32_t m,
                             uint32_t* flags, int sms, cudaStream_t st) {
  og_check_csr_kernel<<<sms * 4, 256, 0, st>>>(off, adj, n, m, flags);
  return cudaGetLastError();
}

}  // namespace og
