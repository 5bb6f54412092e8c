// Barrier-free Delta-stepping engine: per-warp bucket fusion and per-query completion.
//
// Same method as og_kernels.cu (eager bucket update with bucket fusion, Section 3.3),
// scheduled without grid-wide barriers:
//   * every warp owns a FIFO of entries of the current bucket of one query in shared
//     memory (its "local bucket").  It drains that FIFO with warp-level synchronisation
//     only -- the fused rounds of the paper -- and copies it to the query's global bucket
//     once it holds `threshold` entries, so that other warps can take part;
//   * idle warps claim 32-entry tiles of a query's global current bucket through a CAS
//     on an (epoch, claim) word; appends reserve positions with warp-aggregated
//     atomicAdd and publish each entry with one 64-bit store, a consumer waits for the
//     entry (bounded) and resets the position to the empty marker;
//   * each query counts its outstanding entries of the current bucket (local, global or
//     in flight).  Priority order is kept exactly: a query moves to its next bucket only
//     when that count reaches zero, and the warp that brings it to zero performs the
//     move (next non-empty bucket, overflow redistribution, PPSP / A* stop rule).
// The paper's global round barrier thus becomes a per-query completion event; queries
// of a batch advance independently.
#include "og_device.cuh"

namespace og {

constexpr unsigned long long kEmpty = 0xFFFFFFFFFFFFFFFFull;  // free ring position
constexpr uint32_t kClosed = 0xFFFFFFFFu;                      // claim word: no task

__device__ __forceinline__ unsigned long long pack(uint32_t v, uint32_t d) {
  return ((unsigned long long)d << 32) | v;
}

struct WarpQ {      // the warp's local bucket (FIFO in shared memory); warp-uniform fields
  uint2* buf;
  uint32_t cap, head, size;
  uint32_t q, cur;
};

struct ACnt {
  uint32_t items, stale, relax, improved, local, global, ovf, flushes, fused;
};

// Appends a warp's improved vertices: bucket == cur -> the warp's FIFO (if fusion is on
// and there is room) else the global current bucket; cur < bucket < cur + B -> ring slot
// of the bucket; beyond -> overflow pile.  All 32 lanes call.
// Outstanding-work accounting: an entry that other warps can claim (global current
// bucket) is counted in the query's outstanding count before it is stored -- otherwise a
// consumer could finish it and drive the count to zero first.  Entries kept in the FIFO
// are private and are returned here, to be counted when the batch settles.
__device__ __forceinline__ uint32_t insert_async(const AParams& P, WarpQ& L, bool ins,
                                                 uint32_t v, uint32_t nd, uint32_t key,
                                                 ACnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t q = L.q, cur = L.cur;
  AQState* s = P.aq + q;
  int dest = 0;  // 1 local, 2 ring, 3 overflow
  if (ins) {
    if (key < cur) {  // only with an inconsistent A* heuristic: clamp, disable early exit
      key = cur;
      s->no_exit = 1u;
    }
    dest = (P.T != 0 && key == cur) ? 1 : ((key - cur < P.B) ? 2 : 3);
  }
  uint32_t added = 0;
  const unsigned lm = __ballot_sync(FULL, dest == 1);
  if (lm) {
    const uint32_t room = L.cap - L.size;
    const uint32_t rank = __popc(lm & lanemask_lt());
    if (dest == 1) {
      if (rank < room) {
        L.buf[(L.head + L.size + rank) % L.cap] = make_uint2(v, nd);
        C.local++;
      } else {
        dest = 2;  // FIFO full: the entry goes to the global current bucket
      }
    }
    const uint32_t took = min((uint32_t)__popc(lm), room);
    L.size += took;
    added += took;
  }
  const unsigned rm = __ballot_sync(FULL, dest == 2);
  const unsigned cm = __ballot_sync(FULL, dest == 2 && key == cur);
  uint32_t dep = 0;
  if (cm) {
    if (lane == 0) {
      dep = atomicAdd(&s->work, (uint32_t)__popc(cm));
      __threadfence();
    }
    dep = __shfl_sync(FULL, dep, 0);  // every store below waits for the count
  }
  if (dest == 2) {
    const uint32_t cid = q * P.B + (key & P.Bmask);
    if (q >= P.nq || v >= P.n) report_bad(P.sync, 6u, v, q);
    const unsigned peers = __match_any_sync(rm, cid);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(P.counts + cid, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    uint32_t pos = base + __popc(peers & lanemask_lt());
    asm volatile("" : "+r"(pos) : "r"(dep));
    if (pos < P.cap) {
      st_relaxed64(reinterpret_cast<unsigned long long*>(P.ring + (size_t)cid * P.cap + pos),
                   pack(v, nd));
      C.global++;
    } else {
      dest = 3;
    }
  }
  // counted entries of the current bucket that found their slot full wait in the pile
  added -= __popc(__ballot_sync(FULL, dest == 3 && ((cm >> lane) & 1u)));
  if (dest == 3) {
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
  return added;
}

template <int K>
__device__ __forceinline__ uint32_t relax_edges_async(const AParams& P, WarpQ& L,
                                                      const bool (&ok)[K],
                                                      const uint2 (&ew)[K],
                                                      const uint32_t (&g)[K], ACnt& C,
                                                      uint32_t delta, bool astar, float tx,
                                                      float ty) {
  bool okk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    okk[k] = ok[k];
    if (ok[k] && ew[k].x >= P.n) {
      report_bad(P.sync, 3u, ew[k].x, 0u);
      okk[k] = false;
    }
  }
  uint32_t h[K];
#pragma unroll
  for (int k = 0; k < K; ++k)
    h[k] = (astar && okk[k]) ? heuristic(P.xy, P.xy_integral, ew[k].x, tx, ty) : 0u;
  uint32_t nd[K], old[K];
  uint32_t* dq = P.dist + (size_t)L.q * P.n;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const unsigned long long s = (unsigned long long)g[k] + ew[k].y;
    nd[k] = s >= kSat ? kSat : (uint32_t)s;
    if (okk[k] && s >= kSat) atomicOr(&P.sync->err, kErrSat);
  }
  bool go[K];
#pragma unroll
  for (int k = 0; k < K; ++k) go[k] = okk[k];
  if (P.precheck) {
    uint32_t seen[K];
#pragma unroll
    for (int k = 0; k < K; ++k) seen[k] = okk[k] ? ld_cached(dq + ew[k].x) : 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) go[k] = okk[k] && nd[k] < seen[k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) old[k] = go[k] ? atomicMin(dq + ew[k].x, nd[k]) : 0u;
  if (P.touched) {
    // First reach of a vertex (its distance was unreachable): mark its block, so the
    // slot's row can later be reset block by block (the result is not waited for).
    uint32_t* tb = P.touched + (size_t)L.q * P.tb_words;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (go[k] && old[k] == kInf) {
        const uint32_t b = ew[k].x >> kTouchShift;
        atomicOr(tb + (b >> 5), 1u << (b & 31u));
      }
  }
  uint32_t added = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool ins = go[k] && nd[k] < old[k];
    C.relax += okk[k] ? 1u : 0u;
    C.improved += ins ? 1u : 0u;
    if (ins && P.prefetch) prefetch_row(P.ell, P.off, ew[k].x);
    const uint32_t key = ins ? bucket_of(nd[k], h[k], delta) : 0u;
    added += insert_async(P, L, ins, ew[k].x, nd[k], key, C);
  }
  return added;
}

template <int K>
__device__ __forceinline__ uint32_t relax_async(const AParams& P, WarpQ& L,
                                                const bool (&ok)[K], const uint32_t (&e)[K],
                                                const uint32_t (&g)[K], ACnt& C,
                                                uint32_t delta, bool astar, float tx,
                                                float ty) {
  uint2 ew[K];
#pragma unroll
  for (int k = 0; k < K; ++k) ew[k] = ok[k] ? __ldg(P.adj + e[k]) : make_uint2(0u, 0u);
  return relax_edges_async<K>(P, L, ok, ew, g, C, delta, astar, tx, ty);
}

// Relaxes the out-edges of the entries held by the lanes (query L.q, bucket L.cur).  An
// entry whose vertex has a smaller distance by now is skipped (a newer entry exists).
// Returns the number of current-bucket entries added.
template <bool ELL>
__device__ uint32_t expand_async(const AParams& P, WarpQ& L, bool has, uint32_t u, uint32_t g,
                                 ACnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const QDesc* qd = P.qd + L.q;
  const uint32_t delta = __ldg(&qd->delta);
  const bool astar = P.has_astar && __ldg(&qd->kind) == kASTAR;
  const float tx = astar ? __ldg(&qd->tx) : 0.f, ty = astar ? __ldg(&qd->ty) : 0.f;
  uint32_t beg = 0, end = 0;
  if (has && (u >= P.n || L.q >= P.nq)) {
    report_bad(P.sync, 1u, u, L.q);
    has = false;
  }
  if (ELL) {  // ELL rows: one 64-byte row per lane, no offsets lookup
    uint2 ew[kEllWidth];
    bool live = has;
    uint32_t d = 0;
    if (has) {
      C.items++;
      d = __ldcg(P.dist + (size_t)L.q * P.n + u);
      load_row(P.ell, u, ew);
    } else {
#pragma unroll
      for (int k = 0; k < kEllWidth; ++k) ew[k] = make_uint2(kNone, 0u);
    }
    if (has && d < g) {
      live = false;
      C.stale++;
    }
    bool ok[kEllWidth];
    uint32_t gg[kEllWidth];
#pragma unroll
    for (int k = 0; k < kEllWidth; ++k) {
      ok[k] = live && ew[k].x != kNone;
      gg[k] = g;
    }
    return relax_edges_async<kEllWidth>(P, L, ok, ew, gg, C, delta, astar, tx, ty);
  }
  if (has) {
    C.items++;
    const uint32_t d = __ldcg(P.dist + (size_t)L.q * P.n + u);
    beg = __ldg(P.off + u);
    end = __ldg(P.off + u + 1);
    if (d < g) {
      has = false;
      C.stale++;
      beg = end = 0;
    } else if (end < beg) {
      report_bad(P.sync, 2u, u, beg);
      has = false;
      beg = end = 0;
    }
  }
  uint32_t added = 0;
  const uint32_t deg = end - beg;
  const bool heavy = deg >= 32u;
  unsigned hm = __ballot_sync(FULL, heavy);
  while (hm) {
    const int l = __ffs(hm) - 1;
    hm &= hm - 1;
    const uint32_t hb = __shfl_sync(FULL, beg, l), he = __shfl_sync(FULL, end, l);
    const uint32_t hg = __shfl_sync(FULL, g, l);
    for (uint32_t e0 = hb; e0 < he; e0 += 32 * 4) {
      bool ok[4];
      uint32_t ee[4], gg[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ee[k] = e0 + 32u * k + lane;
        ok[k] = ee[k] < he;
        gg[k] = hg;
      }
      added += relax_async<4>(P, L, ok, ee, gg, C, delta, astar, tx, ty);
    }
  }
  const uint32_t ld = heavy ? 0u : deg;
  uint32_t incl = ld;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  const uint32_t excl = incl - ld;
  for (uint32_t base = 0; base < total; base += 32 * 4) {
    bool ok[4];
    uint32_t ee[4], gg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t idx = base + 32u * k + lane;
      uint32_t pos = 0;  // owner lane: number of lanes whose inclusive sum is <= idx
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const uint32_t x = __shfl_sync(FULL, incl, pos + s - 1);
        if (x <= idx) pos += s;
      }
      const uint32_t ob = __shfl_sync(FULL, beg, pos), oe = __shfl_sync(FULL, excl, pos);
      gg[k] = __shfl_sync(FULL, g, pos);
      ok[k] = idx < total;
      ee[k] = ob + (idx - oe);
    }
    added += relax_async<4>(P, L, ok, ee, gg, C, delta, astar, tx, ty);
  }
  return added;
}

// Ends a query: result, dirty marker (ring positions may still hold entries), and one
// fewer active query.  Whole warp.
__device__ void finish_query(const AParams& P, uint32_t q, bool leaves_entries) {
  const uint32_t lane = threadIdx.x & 31;
  AQState* s = P.aq + q;
  const QDesc* qd = P.qd + q;
  if (lane == 0) {
    const uint32_t dst = __ldg(&qd->dst);
    s->result = dst < P.n ? __ldcg(P.dist + (size_t)q * P.n + dst) : 0u;
    if (leaves_entries || __ldcg(&s->aborted)) s->dirty = 1u;
    s->advances = __ldcg(&s->advances) + 1u;
    s->mode = kMDone;
    __threadfence();
    atomicSub(&P.sync->active, 1u);
  }
  __syncwarp();
}

// Called by the warp whose update brought the query's outstanding count to zero: every
// entry of the current task is done and no other warp holds work of this query.  Moves
// the query to its next task (Section 3.2: the next bucket is the smallest non-empty one;
// Section 6.1: PPSP stops on entering bucket i with i * Delta >= dist(src, dst)).
__device__ void advance(const AParams& P, uint32_t q) {
  const uint32_t lane = threadIdx.x & 31;
  AQState* s = P.aq + q;
  const QDesc* qd = P.qd + q;
  uint32_t* cnts = P.counts + (size_t)q * P.B;
  __threadfence();
  unsigned long long w = 0;
  if (lane == 0) w = atomicExch(&s->word, ((unsigned long long)kClosed << 32) | kClosed);
  w = __shfl_sync(FULL, w, 0);
  const uint32_t epoch = (uint32_t)(w >> 32);
  uint32_t mode = warp_ld(&s->mode), cur = warp_ld(&s->cur);
  for (int guard = 0;; ++guard) {
    if (warp_ld(&s->aborted)) {
      finish_query(P, q, true);
      return;
    }
    uint32_t nmode = mode, ncur = cur, nwork = 0, nlimit = 0;
    bool done = false;
    if (mode == kMRelax) {
      if (lane == 0) cnts[cur & P.Bmask] = 0u;
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
      const uint32_t ovf_n = warp_ld(&s->ovf_n), ovf_min = warp_ld(&s->ovf_min);
      if (ovf_n > 0 && ovf_min <= next) {
        nmode = kMRedistMin;
        nlimit = nwork = min(ovf_n, P.ocap);
        if (lane == 0) {
          s->redist_min = next;
          s->ovf_n2 = 0;
          s->ovf_min2 = kInf;
          s->redists = __ldcg(&s->redists) + 1u;
        }
      } else if (next == kInf) {
        done = true;
      } else {
        ncur = next;
        nmode = kMRelax;
        nwork = min(warp_ld(cnts + (next & P.Bmask)), P.cap);
      }
    } else if (mode == kMRedistMin) {
      const uint32_t nc = warp_ld(&s->redist_min);
      if (nc == kInf) {
        if (lane == 0) s->ovf_n = 0;
        done = true;
      } else {
        ncur = nc;
        nmode = kMRedistMove;
        nlimit = nwork = warp_ld(&s->limit);
      }
    } else {  // kMRedistMove
      if (lane == 0) {
        s->ovf_sel = __ldcg(&s->ovf_sel) ^ 1u;
        s->ovf_n = __ldcg(&s->ovf_n2);
        s->ovf_min = __ldcg(&s->ovf_min2);
      }
      nmode = kMRelax;
      nwork = min(warp_ld(cnts + (cur & P.Bmask)), P.cap);
    }
    const uint32_t kind = __ldg(&qd->kind);
    if (!done && nmode == kMRelax && kind != kSSSP && !warp_ld(&s->no_exit)) {
      const uint32_t dt = warp_ld(P.dist + (size_t)q * P.n + __ldg(&qd->dst));
      if (dt != kInf && (unsigned long long)ncur * __ldg(&qd->delta) >= dt) {
        finish_query(P, q, true);
        return;
      }
    }
    if (done) {
      finish_query(P, q, false);
      return;
    }
    __syncwarp();
    if (lane == 0) {
      s->mode = nmode;
      s->cur = ncur;
      s->work = nwork;
      s->limit = nlimit;
      s->advances = s->advances + 1u;
    }
    __syncwarp();
    mode = nmode;
    cur = ncur;
    if (nwork == 0 && guard < 8) continue;  // nothing to claim: move on at once
    break;
  }
  if (lane == 0) {
    __threadfence();
    st_release64(&s->word, (unsigned long long)(epoch + 1) << 32);
  }
  __syncwarp();
}

// Adds delta (two's complement) to a query's outstanding count; advances the query if
// it reached zero.  Every lane fences before lane 0 settles: the lanes' earlier stores
// (a consumed ring position reset to free, entries appended) must be visible before the
// count can reach zero, because reaching zero lets the query advance and reuse the ring
// slot; a reset arriving after a new entry in the reused slot would erase that entry.
__device__ __forceinline__ void settle(const AParams& P, uint32_t q, uint32_t delta) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t zero = 0;
  if (q >= P.nq) {
    if (lane == 0) report_bad(P.sync, 8u, q, delta);
    return;
  }
  __threadfence();
  __syncwarp();
  if (lane == 0 && delta != 0) {
    const uint32_t old = atomicAdd(&P.aq[q].work, delta);
    zero = (old + delta == 0u) ? 1u : 0u;
  }
  zero = __shfl_sync(FULL, zero, 0);
  if (zero) advance(P, q);
}

// Copies the warp's FIFO, except the `keep` oldest entries (its next batch), to the
// query's global current bucket, where idle warps can claim them.
__device__ void flush_local(const AParams& P, WarpQ& L, ACnt& C, uint32_t keep = 0) {
  const uint32_t lane = threadIdx.x & 31;
  if (L.size <= keep) return;
  __syncwarp();
  if (L.q >= P.nq || L.size > L.cap) {
    if (lane == 0) report_bad(P.sync, 9u, L.q, L.size);
    L.size = 0;
    L.head = 0;
    return;
  }
  AQState* s = P.aq + L.q;
  const uint32_t cid = L.q * P.B + (L.cur & P.Bmask);
  const uint32_t nmove = L.size - keep;
  const uint32_t first = (L.head + keep) % L.cap;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(P.counts + cid, nmove);
  base = __shfl_sync(FULL, base, 0);
  uint32_t spilled = 0;
  for (uint32_t i = lane; i < nmove; i += 32) {
    const uint2 en = L.buf[(first + i) % L.cap];
    const uint32_t pos = base + i;
    if (pos < P.cap) {
      st_relaxed64(reinterpret_cast<unsigned long long*>(P.ring + (size_t)cid * P.cap + pos),
                   pack(en.x, en.y));
    } else {
      const uint32_t sel = __ldcg(&s->ovf_sel);
      const uint32_t op = atomicAdd(&s->ovf_n, 1u);
      atomicMin(&s->ovf_min, L.cur);
      if (op < P.ocap) {
        P.ovf[((size_t)L.q * 2 + sel) * P.ocap + op] = en;
      } else {
        s->aborted = 1u;
        atomicOr(&P.sync->err, kErrArena);
      }
      ++spilled;
    }
  }
  spilled = warp_sum(spilled);
  C.flushes++;
  L.size = keep;
  __syncwarp();
  if (spilled) settle(P, L.q, 0u - spilled);  // spilled entries wait in the overflow pile
}

// Redistribution task on pile entries [start, start + k): step 1 records the smallest
// live bucket, step 2 moves live entries of the new ring window into the ring.
__device__ void redist_task(const AParams& P, uint32_t q, uint32_t mode, uint32_t cur,
                            uint32_t start, uint32_t k) {
  const uint32_t lane = threadIdx.x & 31;
  AQState* s = P.aq + q;
  const QDesc* qd = P.qd + q;
  const bool astar = __ldg(&qd->kind) == kASTAR;
  const uint32_t delta = __ldg(&qd->delta);
  const uint32_t sel = __ldcg(&s->ovf_sel);
  const uint2* pile = P.ovf + ((size_t)q * 2 + sel) * P.ocap;
  uint32_t best = kInf;
  bool live = lane < k;
  if (live && start + lane >= P.ocap) {
    report_bad(P.sync, 5u, start + lane, q);
    live = false;
  }
  uint2 en = make_uint2(0u, 0u);
  if (live) {
    en = __ldcg(pile + start + lane);
    if (en.x >= P.n) {
      report_bad(P.sync, 7u, en.x, start + lane);
      live = false;
    }
  }
  if (live) {
    if (__ldcg(P.dist + (size_t)q * P.n + en.x) >= en.y) {
      const uint32_t h =
          astar ? heuristic(P.xy, P.xy_integral, en.x, __ldg(&qd->tx), __ldg(&qd->ty)) : 0u;
      const uint32_t key = max(bucket_of(en.y, h, delta), mode == kMRedistMove ? cur : 0u);
      if (mode == kMRedistMin) {
        best = key;
      } else {
        bool to_pile = true;
        if (key - cur < P.B) {
          const uint32_t cid = q * P.B + (key & P.Bmask);
          const uint32_t pos = atomicAdd(P.counts + cid, 1u);
          if (pos < P.cap) {
            st_relaxed64(
                reinterpret_cast<unsigned long long*>(P.ring + (size_t)cid * P.cap + pos),
                pack(en.x, en.y));
            to_pile = false;
          }
        }
        if (to_pile) {
          const uint32_t pos = atomicAdd(&s->ovf_n2, 1u);
          atomicMin(&s->ovf_min2, key);
          if (pos < P.ocap) {
            P.ovf[((size_t)q * 2 + (sel ^ 1u)) * P.ocap + pos] = en;
          } else {
            s->aborted = 1u;
            atomicOr(&P.sync->err, kErrArena);
          }
        }
      }
    }
  }
  if (mode == kMRedistMin) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL, best, o));
    if (lane == 0 && best != kInf) atomicMin(&s->redist_min, best);
  }
  __syncwarp();
  settle(P, q, 0u - k);
}

// Claims up to 32 entries of some query's current task.  The warp looks at 32 queries at
// a time, starting at query `rot` (lane i at rot + i): every lane reads its query's claim
// word, and those that are open also read the task's limit, so a round of the search
// costs three round trips however many of the 32 queries are finished or idle.  The open
// queries with entries left are then tried in lane order by compare-and-swap on their
// claim words (a lane that loses its compare-and-swap reads its query again; eight
// attempts per group of 32); the claim is broadcast to the warp.
__device__ bool claim(const AParams& P, uint32_t& rot, uint32_t& q, uint32_t& mode,
                      uint32_t& cur, uint32_t& start, uint32_t& k) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t a0 = 0; a0 < P.nq; a0 += 32) {
    const uint32_t qq = (rot + a0 + lane) % P.nq;
    AQState* s = P.aq + qq;
    unsigned long long w = 0ull;
    uint32_t c = 0, m = 0, cu = 0, lim = 0;
    if (a0 + lane < P.nq) {
      w = ld_acquire64(&s->word);
      c = (uint32_t)w;
      if (c != kClosed) {
        m = __ldcg(&s->mode);
        cu = __ldcg(&s->cur);
        lim = m == kMRelax ? min(__ldcg(P.counts + (size_t)qq * P.B + (cu & P.Bmask)), P.cap)
                           : __ldcg(&s->limit);
      }
    }
    for (int tries = 0; tries < 8; ++tries) {
      const unsigned open = __ballot_sync(FULL, a0 + lane < P.nq && c != kClosed && c < lim);
      if (!open) break;
      const int l = __ffs(open) - 1;
      uint32_t got = 0;
      if ((int)lane == l) {
        got = atomicCAS(&s->word, w, w + min(32u, lim - c)) == w ? 1u : 0u;
        if (!got) {  // another warp moved the word first: look at the query again
          w = ld_acquire64(&s->word);
          c = (uint32_t)w;
          if (c != kClosed) {
            m = __ldcg(&s->mode);
            cu = __ldcg(&s->cur);
            lim = m == kMRelax
                      ? min(__ldcg(P.counts + (size_t)qq * P.B + (cu & P.Bmask)), P.cap)
                      : __ldcg(&s->limit);
          }
        }
      }
      if (__shfl_sync(FULL, got, l)) {
        q = __shfl_sync(FULL, qq, l);
        mode = __shfl_sync(FULL, m, l);
        cur = __shfl_sync(FULL, cu, l);
        start = __shfl_sync(FULL, c, l);
        k = __shfl_sync(FULL, min(32u, lim - c), l);
        rot = q;
        return true;
      }
    }
  }
  return false;
}

template <bool ELL>
__device__ __forceinline__ void async_body(const AParams& P) {
  extern __shared__ __align__(16) unsigned char og_async_smem[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpQ L;
  L.buf = reinterpret_cast<uint2*>(og_async_smem) + (size_t)warp * P.lq_cap;
  L.cap = P.lq_cap;
  L.head = 0;
  L.size = 0;
  L.q = 0;
  L.cur = 0;
  ACnt C = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t rot = (blockIdx.x * kWarps + warp) % max(P.nq, 1u);
  uint64_t idle_t0 = 0;
  uint32_t backoff = 32, batches = 0, last_beat = 0;
  bool stop = false;
  const uint64_t deadline = P.budget_ns ? warp_now() + P.budget_ns : 0ull;
  for (;;) {
    if (L.size) {
      // Fused processing of the warp's own bucket: no synchronisation beyond the warp.
      const uint32_t k = min(32u, L.size);
      uint32_t v = 0, d = 0;
      const bool has = lane < k;
      __syncwarp();  // FIFO entries written by other lanes are visible
      if (has) {
        const uint2 en = L.buf[(L.head + lane) % L.cap];
        v = en.x;
        d = en.y;
      }
      __syncwarp();
      L.head = (L.head + k) % L.cap;
      L.size -= k;
      const uint32_t added = expand_async<ELL>(P, L, has, v, d, C);
      C.fused++;
      settle(P, L.q, added - k);
      if (L.size && L.size >= P.T) flush_local(P, L, C, 32u);
      if ((++batches & 63u) == 0 && lane == 0) atomicAdd(&P.sync->progress, 1u);
      if ((batches & 15u) == 0) {
        if (warp_ld(&P.sync->err) & kErrFatal) break;
        if (deadline && warp_now() > deadline) {
          flush_local(P, L, C);
          stop = true;
        }
      }
      continue;
    }
    if (stop) break;
    uint32_t q, mode, cur, start, k;
    if (claim(P, rot, q, mode, cur, start, k)) {
      idle_t0 = 0;
      backoff = 32;
      if ((++batches & 63u) == 0 && lane == 0) atomicAdd(&P.sync->progress, 1u);
      if (mode == kMRelax) {
        uint32_t v = 0, d = 0;
        bool has = lane < k;
        if (has && (q >= P.nq || start + lane >= P.cap)) {
          report_bad(P.sync, 4u, start + lane, q);
          has = false;
        }
        if (has) {
          unsigned long long* p = reinterpret_cast<unsigned long long*>(
              P.ring + ((size_t)q * P.B + (cur & P.Bmask)) * P.cap + start + lane);
          unsigned long long x = ld_relaxed64(p);
          const uint64_t t0 = gtimer();
          uint32_t spins = 0;
          while ((uint32_t)x == 0xFFFFFFFFu) {  // reserved, not yet written
            if ((++spins & 63u) == 0 && gtimer() - t0 > P.spin_ns) {
              P.sync->timeout_at = 2u;
              // Where the wait gave up, for the error message (the timer slots of the
              // statistics are unused by this engine): query and position, bucket and
              // its append count, the claim word, the query's cursor / mode / count.
              const AQState* aq = P.aq + q;
              const unsigned long long where = ((unsigned long long)q << 32) | (start + lane);
              if (atomicCAS(&P.stats->v[kStTFrontier], 0ull, where) == 0ull) {
                P.stats->v[kStTFused] =
                    ((unsigned long long)cur << 32) |
                    __ldcg(P.counts + (size_t)q * P.B + (cur & P.Bmask));
                P.stats->v[kStTBarrier] = ld_relaxed64(&aq->word);
                P.stats->v[kStTHub] = ((unsigned long long)__ldcg(&aq->cur) << 32) |
                                      ((unsigned long long)__ldcg(&aq->mode) << 28) |
                                      (__ldcg(&aq->work) & 0x0FFFFFFFu);
              }
              atomicOr(&P.sync->err, kErrTimeout);
              break;
            }
            x = ld_relaxed64(p);
          }
          if ((uint32_t)x != 0xFFFFFFFFu) {
            st_relaxed64(p, kEmpty);
            v = (uint32_t)x;
            d = (uint32_t)(x >> 32);
          } else {
            has = false;
          }
        }
        L.q = q;
        L.cur = cur;
        const uint32_t added = expand_async<ELL>(P, L, has, v, d, C);
        settle(P, q, added - k);
        if (L.size && L.size >= P.T) flush_local(P, L, C, 32u);
      } else {
        redist_task(P, q, mode, cur, start, k);
      }
      if (deadline && warp_now() > deadline) {
        flush_local(P, L, C);
        stop = true;
      }
      continue;
    }
    // Nothing to claim: finished, stopped, or waiting for other warps to publish work.
    // Every test below is warp-uniform (one lane reads, all lanes decide alike).
    if (warp_ld(&P.sync->active) == 0u) break;
    if (warp_ld(&P.sync->err) & kErrFatal) break;
    const uint64_t now = warp_now();
    if (deadline && now > deadline) break;
    // Time out only when no warp has reported progress for the whole limit: a healthy
    // run may keep its work in a few warps' local buckets for a long time.
    const uint32_t beat = warp_ld(&P.sync->progress);
    if (idle_t0 == 0 || beat != last_beat) {
      idle_t0 = now;
      last_beat = beat;
    } else if (now - idle_t0 > P.spin_ns) {
      if (lane == 0) {
        P.sync->timeout_at = 1u;
        atomicOr(&P.sync->err, kErrTimeout);
      }
      break;
    }
    __nanosleep(backoff);
    backoff = min(backoff * 2u, 1024u);
  }
  // Leave nothing in the FIFO (a fatal error may stop a warp with local entries).
  const uint32_t vals[9] = {C.items, C.stale, C.relax, C.improved, C.local, C.global,
                            C.ovf, C.flushes, C.fused};
  const int idx[9] = {kStItems, kStStale, kStRelax, kStImproved, kStLocal, kStGlobal, kStOvf,
                      kStFlush, kStFused};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint32_t x = vals[i];  // flushes and fused batches are warp-uniform counts
    const uint32_t s = (i >= 7) ? x : warp_sum(x);
    if (lane == 0 && s) atomicAdd(&P.stats->v[idx[i]], (unsigned long long)s);
  }
}

extern "C" __global__ void __launch_bounds__(kBlock) og_async_kernel(AParams P) {
  async_body<false>(P);
}
extern "C" __global__ void __launch_bounds__(kBlock) og_async_ell_kernel(AParams P) {
  async_body<true>(P);
}

// Starts the listed queries: dist[src] = 0 and the start vertex as the only entry of its
// first bucket (the initial state of the Section 3.2 figures).
extern "C" __global__ void og_async_init_kernel(AParams P, const uint32_t* slots,
                                                uint32_t nslots) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const uint32_t q = slots ? slots[t] : t;
  const QDesc d = P.qd[q];
  P.dist[(size_t)q * P.n + d.src] = 0u;
  if (P.touched) {
    const uint32_t b = d.src >> kTouchShift;
    atomicOr(P.touched + (size_t)q * P.tb_words + (b >> 5), 1u << (b & 31u));
  }
  const uint32_t h0 = d.kind == kASTAR ? heuristic(P.xy, P.xy_integral, d.src, d.tx, d.ty) : 0u;
  const uint32_t key0 = bucket_of(0u, h0, d.delta);
  uint32_t* cnts = P.counts + (size_t)q * P.B;
  for (uint32_t k = 0; k < P.B; ++k) cnts[k] = 0u;
  cnts[key0 & P.Bmask] = 1u;
  st_relaxed64(reinterpret_cast<unsigned long long*>(
                   P.ring + ((size_t)q * P.B + (key0 & P.Bmask)) * P.cap),
               pack(d.src, 0u));
  AQState s;
  s.word = 0ull;
  s.mode = kMRelax;
  s.cur = key0;
  s.work = 1;
  s.limit = 0;
  s.ovf_n = 0;
  s.ovf_min = kInf;
  s.ovf_sel = 0;
  s.ovf_n2 = 0;
  s.ovf_min2 = kInf;
  s.redist_min = kInf;
  s.no_exit = 0;
  s.result = kInf;
  s.aborted = 0;
  s.dirty = 0;
  s.advances = 0;
  s.redists = 0;
  P.aq[q] = s;
  __threadfence();
  atomicAdd(&P.sync->active, 1u);
}

// Resets the distance rows of the listed slots to unreachable, only in the blocks their
// touched bitmaps mark, and clears those bitmaps (blockIdx.y indexes the slot list).  A
// warp takes one bitmap word at a time and fills each marked block of kTouchBlock
// vertices with 16-byte stores.
extern "C" __global__ void og_touch_reset_kernel(uint32_t* dist, uint32_t n, uint32_t* touched,
                                                 uint32_t tb_words, const uint32_t* slots) {
  const uint32_t q = slots[blockIdx.y];
  uint32_t* d = dist + (size_t)q * n;
  uint32_t* tb = touched + (size_t)q * tb_words;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t wpb = blockDim.x >> 5;
  for (uint32_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < tb_words; i += gridDim.x * wpb) {
    uint32_t word = 0;
    if (lane == 0) {
      word = tb[i];
      if (word) tb[i] = 0u;
    }
    word = __shfl_sync(FULL, word, 0);
    while (word) {
      const uint32_t bit = (uint32_t)(__ffs(word) - 1);
      word &= word - 1u;
      const size_t v0 = ((size_t)i * 32u + bit) << kTouchShift;
      // kTouchBlock = 256 vertices: 8 per lane, in two 16-byte stores when the block is
      // whole and 16-byte aligned, else word by word.
      const size_t end = min((size_t)n, v0 + kTouchBlock);
      const bool vec = end == v0 + kTouchBlock && (((uintptr_t)(d + v0)) & 15u) == 0;
      if (vec) {
        uint4* p = reinterpret_cast<uint4*>(d + v0);
        p[lane] = make_uint4(kInf, kInf, kInf, kInf);
        p[lane + 32] = make_uint4(kInf, kInf, kInf, kInf);
      } else {
        for (size_t v = v0 + lane; v < end; v += 32) d[v] = kInf;
      }
    }
  }
}

cudaError_t launch_touch_reset(uint32_t* dist, uint32_t n, uint32_t* touched, uint32_t tb_words,
                               const uint32_t* slots, uint32_t nslots, int sms, cudaStream_t st) {
  if (nslots == 0) return cudaSuccess;
  uint32_t gx = (tb_words + 7u) / 8u;
  const uint32_t cap = (uint32_t)sms * 2u;
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  og_touch_reset_kernel<<<dim3(gx, nslots), 256, 0, st>>>(dist, n, touched, tb_words, slots);
  return cudaGetLastError();
}

cudaError_t launch_async(const AParams& P, int grid, size_t smem, cudaStream_t st) {
  if (P.ell) og_async_ell_kernel<<<grid, kBlock, smem, st>>>(P);
  else og_async_kernel<<<grid, kBlock, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t async_occupancy(int* blocks_per_sm, size_t smem, bool ell) {
  const void* k = ell ? (const void*)og_async_ell_kernel : (const void*)og_async_kernel;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBlock, smem);
}

cudaError_t launch_async_init(const AParams& P, const uint32_t* slots, uint32_t nslots,
                              cudaStream_t st) {
  if (nslots == 0) return cudaSuccess;
  og_async_init_kernel<<<(nslots + 127) / 128, 128, 0, st>>>(P, slots, nslots);
  return cudaGetLastError();
}

}  // namespace og
