// Device side of approximate unweighted set cover (Section 6.1, "Approximate Set Cover"),
// with the sets of the graph's set system (set v = adjacency list of v, entries counted
// with multiplicity) bucketed by their number of uncovered elements.  The highest
// non-empty bucket j is worked off in steps; a step is
//   A  pack: every member drops its covered elements (into the other element buffer)
//      and counts the rest, D; D = 0 leaves, D < t_j moves to the bucket of D, the
//      others are active and claim each of their elements with an atomicMin of
//      ((~step) << 32 | priority): the smallest priority wins, and a claim of an earlier
//      step never matches this step's key;
//   B  count: an active set counts the elements whose claim is its own key; with at
//      least tau_j it joins the cover (step_out = step) and marks all its elements
//      covered, otherwise it stays in bucket j for the next step.
// Sets with fewer than `hub` residual elements are handled 32 to a warp (a warp owns all
// their elements, so each phase needs no grid-wide count); larger sets have their
// elements split into 256-element chunks over every warp of the grid, which needs one
// more grid barrier after the pack (A2: classify, claim) and after the count (C: join,
// cover, move).  One cooperative persistent launch; phases are separated by a bounded
// grid barrier whose last arriver decides the next phase (sc_decide).
#include <stddef.h>

#include "og_device.cuh"

#include "og_setcover.cuh"

namespace og {

namespace {

struct ScSmem {
  uint32_t phase, err, last;
  uint32_t j, step, csel, band, tj, tauj;
  uint32_t ns;        // small members of the current lists
  uint32_t nl;        // large members
  uint32_t tl;        // elements of the large members (the step's element space)
  uint32_t gn;        // gather: entries of the band's current buffer
  unsigned long long t_bar, t_a, t_b, t_g;  // per-CTA phase time (thread 0)
};

struct ScCnt {
  uint32_t items, scanned, moved, chosen;
};

enum LMode : int { kLPack = 0, kLClaim = 1, kLCount = 2, kLCover = 3 };

__device__ __forceinline__ uint32_t gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ uint32_t nwarps() { return gridDim.x * (blockDim.x >> 5); }

__device__ __forceinline__ uint32_t next_store(uint32_t s) { return s == 1u ? 2u : 1u; }

__device__ __forceinline__ unsigned long long claim_key(uint32_t step, uint32_t pri) {
  return ((unsigned long long)(0xFFFFFFFFu - step) << 32) | pri;
}

// Element o of a set whose elements start at `base` in storage s.
__device__ __forceinline__ uint32_t elem(const ScParams& P, uint32_t base, uint32_t s, uint32_t o) {
  return s == 0u ? __ldg(&P.adj[base + o].x) : __ldcg(P.pk[s - 1u] + base + o);
}

// Bucket of a residual size d >= 1: the largest j with t[j] <= d.
__device__ __forceinline__ uint32_t bucket_of_size(const ScParams& P, uint32_t d) {
  uint32_t lo = 0, hi = P.nb - 1u;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1u) / 2u;
    if (__ldg(P.t + mid) <= d) lo = mid;
    else hi = mid - 1u;
  }
  return lo;
}

__device__ __forceinline__ uint32_t warp_incl(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// X: per-lane first element of the lane's set, non-decreasing over lanes, X of lane 0 = 0.
// Returns the largest lane k with X_k <= e (the set holding element e).  All lanes call.
__device__ __forceinline__ uint32_t find_set(uint32_t X, uint32_t e) {
  uint32_t k = 0;
#pragma unroll
  for (uint32_t s = 16; s > 0; s >>= 1) {
    const uint32_t x = __shfl_sync(FULL, X, k + s);
    if (x <= e) k += s;
  }
  return k;
}

// Lanes with equal keys form contiguous runs (keys never decrease over the lanes).  For
// the lanes with flag set: the rank of this lane among the flagged lanes of its run, the
// number of flagged lanes in the run, and the run's first lane.  All lanes call.
struct Run {
  uint32_t rank, count, head;
};
__device__ __forceinline__ Run run_of(bool flag, uint32_t key) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(FULL, key, 1);
  const unsigned heads = __ballot_sync(FULL, lane == 0u || prev != key);
  const unsigned fl = __ballot_sync(FULL, flag);
  const unsigned le = (lane == 31u) ? FULL : ((2u << lane) - 1u);
  const uint32_t head = 31u - (uint32_t)__clz(heads & le);
  const unsigned above = heads & ~le;
  const unsigned below_next = above ? ((1u << (__ffs(above) - 1)) - 1u) : FULL;
  const unsigned run = below_next & ~((1u << head) - 1u);
  Run r;
  r.rank = __popc(fl & run & lanemask_lt());
  r.count = __popc(fl & run);
  r.head = head;
  return r;
}

// Appends (bucket j, set v) to band j / 16 (lanes with ok).  All lanes call.
__device__ __forceinline__ void band_insert(const ScParams& P, bool ok, uint32_t j, uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t b = j / kScBand;
  if (ok && b >= P.nbands) report_bad(P.sync, 50u, j, v);
  ok = ok && b < P.nbands;
  const unsigned m = __match_any_sync(FULL, ok ? b : (0x80000000u | lane));
  const uint32_t leader = (uint32_t)__ffs(m) - 1u;
  uint32_t at = 0;
  if (ok && lane == leader) at = atomicAdd(P.bcnt + b, (uint32_t)__popc(m));
  at = __shfl_sync(FULL, at, leader);
  if (!ok) return;
  atomicMax(P.bmax + b, j);
  const uint32_t pos = at + (uint32_t)__popc(m & lanemask_lt());
  const uint32_t cap = __ldg(P.bcap + b);
  if (pos >= cap) {
    report_bad(P.sync, 51u, b, pos);
    return;
  }
  const uint32_t sel = __ldcg(P.bsel + b);
  P.bl[__ldg(P.bbase + b) + (unsigned long long)sel * cap + pos] =
      ((unsigned long long)j << 32) | v;
}

// Appends set v (lanes with ok) with residual d and length word lw to member lists sel:
// small (d < hub) or large (with its range in the element space).  All lanes call.
__device__ __forceinline__ void list_insert(const ScParams& P, uint32_t sel, bool ok, uint32_t v,
                                            uint32_t lw, uint32_t d) {
  const uint32_t lane = threadIdx.x & 31;
  const bool small = d < P.hub;
  {
    const bool f = ok && small;
    const unsigned m = __ballot_sync(FULL, f);
    if (m) {
      const uint32_t leader = (uint32_t)__ffs(m) - 1u;
      uint32_t at = 0;
      if (lane == leader) at = atomicAdd(&P.ss->ns[sel], (uint32_t)__popc(m));
      at = __shfl_sync(FULL, at, leader);
      if (f) {
        const uint32_t pos = at + (uint32_t)__popc(m & lanemask_lt());
        if (pos >= P.n) {
          report_bad(P.sync, 52u, v, pos);
        } else {
          const ScList& L = P.sm[sel];
          L.id[pos] = v;
          L.lw[pos] = lw;
          L.dn[pos] = 0u;
          L.wn[pos] = 0u;
        }
      }
    }
  }
  {
    const bool f = ok && !small;
    const unsigned m = __ballot_sync(FULL, f);
    if (m) {
      const uint32_t x = f ? d : 0u;
      const uint32_t incl = warp_incl(x);
      const uint32_t tot = __shfl_sync(FULL, incl, 31);
      const uint32_t leader = (uint32_t)__ffs(m) - 1u;
      unsigned long long old = 0;
      if (lane == leader)
        old = atomicAdd(&P.ss->bw[sel],
                        ((unsigned long long)__popc(m) << kScCntShift) | (unsigned long long)tot);
      old = __shfl_sync(FULL, old, leader);
      if (f) {
        const unsigned long long pos = (old >> kScCntShift) + (unsigned long long)__popc(m & lanemask_lt());
        const unsigned long long start = (old & kScTotMask) + (incl - x);
        if (pos >= P.lg_cap || start + x > 0xFFFFFFFFull) {
          report_bad(P.sync, 53u, v, (uint32_t)pos);
        } else {
          const ScList& L = P.lg[sel];
          L.id[pos] = v;
          L.lw[pos] = lw;
          L.dn[pos] = 0u;
          L.wn[pos] = 0u;
          L.st[pos] = (uint32_t)start;
        }
      }
    }
  }
}

// End of a set's step: join (step_out), move down (band list), stay (next member lists)
// or leave (nothing left).  d: residual found by this step's pack, now in storage s.
__device__ __forceinline__ void settle(const ScParams& P, const ScSmem& S, bool valid, uint32_t v,
                                       uint32_t d, uint32_t s, bool act, bool win, ScCnt& C) {
  const bool move = valid && d > 0u && !act;
  const bool stay = valid && act && !win;
  const uint32_t nlw = d | (s << kScLenBits);
  if (valid && win) {
    P.step_out[v] = S.step;
    ++C.chosen;
  }
  uint32_t jb = 0;
  if (move) {
    jb = bucket_of_size(P, d);
    P.len[v] = nlw;
    ++C.moved;
  }
  band_insert(P, move, jb, v);
  list_insert(P, S.csel ^ 1u, stay, v, nlw, d);
}

// ---- small sets: 32 members per warp --------------------------------------------------

// Phase A for members [32 g, 32 g + 32) of the small list: pack, classify, claim.
__device__ void small_a(const ScParams& P, const ScSmem& S, uint32_t g, ScCnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const ScList& Lc = P.sm[S.csel];
  const uint32_t i = g * 32u + lane;
  const bool valid = i < S.ns;
  uint32_t v = 0, lw = 0, base = 0;
  if (valid) {
    v = __ldcg(Lc.id + i);
    lw = __ldcg(Lc.lw + i);
    base = __ldg(P.off + v);
    ++C.items;
  }
  const uint32_t L = lw & kScLenMask, store = lw >> kScLenBits, dst = next_store(store);
  uint32_t I = warp_incl(L);
  const uint32_t X = I - L, T = __shfl_sync(FULL, I, 31);
  for (uint32_t it = 0; it < T; it += 32u) {
    const uint32_t e = it + lane;
    const bool ok = e < T;
    const uint32_t k = find_set(X, e);
    const uint32_t kb = __shfl_sync(FULL, base, k), ks = __shfl_sync(FULL, store, k);
    const uint32_t kx = __shfl_sync(FULL, X, k), kl = __shfl_sync(FULL, L, k);
    uint32_t u = 0;
    bool keep = false;
    if (ok) {
      u = elem(P, kb, ks, e - kx);
      keep = __ldcg(P.cov + u) == 0;
      ++C.scanned;
    }
    const Run r = run_of(keep, k);
    uint32_t at = 0;
    if (lane == r.head && r.count) at = atomicAdd(Lc.dn + g * 32u + k, r.count);
    at = __shfl_sync(FULL, at, r.head);
    if (keep) {
      const uint32_t pos = at + r.rank;
      if (pos < kl) P.pk[next_store(ks) - 1u][kb + pos] = u;
      else report_bad(P.sync, 56u, kb, pos);
    }
  }
  __syncwarp();
  const uint32_t D = valid ? __ldcg(Lc.dn + i) : 0u;
  const bool act = valid && D >= S.tj;
  const unsigned long long key = act ? claim_key(S.step, __ldg(P.pri + v)) : 0ull;
  const uint32_t La = act ? D : 0u;
  I = warp_incl(La);
  const uint32_t Xa = I - La, Ta = __shfl_sync(FULL, I, 31);
  for (uint32_t it = 0; it < Ta; it += 32u) {
    const uint32_t e = it + lane;
    const uint32_t k = find_set(Xa, e);
    const uint32_t kb = __shfl_sync(FULL, base, k), kd = __shfl_sync(FULL, dst, k);
    const uint32_t kx = __shfl_sync(FULL, Xa, k);
    const unsigned long long kk = __shfl_sync(FULL, key, k);
    if (e < Ta) {
      const uint32_t u = __ldcg(P.pk[kd - 1u] + kb + e - kx);
      atomicMin(P.claim + u, kk);
    }
  }
}

// Phase B for members [32 g, 32 g + 32) of the small list: count received elements,
// join or stay, cover, move.
__device__ void small_b(const ScParams& P, const ScSmem& S, uint32_t g, ScCnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const ScList& Lc = P.sm[S.csel];
  const uint32_t i = g * 32u + lane;
  const bool valid = i < S.ns;
  uint32_t v = 0, lw = 0, base = 0, D = 0;
  if (valid) {
    v = __ldcg(Lc.id + i);
    lw = __ldcg(Lc.lw + i);
    base = __ldg(P.off + v);
    D = __ldcg(Lc.dn + i);
  }
  const uint32_t dst = next_store(lw >> kScLenBits);
  const bool act = valid && D >= S.tj;
  const unsigned long long key = act ? claim_key(S.step, __ldg(P.pri + v)) : 0ull;
  const uint32_t La = act ? D : 0u;
  const uint32_t I = warp_incl(La);
  const uint32_t Xa = I - La, Ta = __shfl_sync(FULL, I, 31);
  for (uint32_t it = 0; it < Ta; it += 32u) {
    const uint32_t e = it + lane;
    const uint32_t k = find_set(Xa, e);
    const uint32_t kb = __shfl_sync(FULL, base, k), kd = __shfl_sync(FULL, dst, k);
    const uint32_t kx = __shfl_sync(FULL, Xa, k);
    const unsigned long long kk = __shfl_sync(FULL, key, k);
    bool hit = false;
    if (e < Ta) hit = __ldcg(P.claim + __ldcg(P.pk[kd - 1u] + kb + e - kx)) == kk;
    const Run r = run_of(hit, k);
    if (lane == r.head && r.count) atomicAdd(Lc.wn + g * 32u + k, r.count);
  }
  __syncwarp();
  const uint32_t W = act ? __ldcg(Lc.wn + i) : 0u;
  const bool win = act && W >= S.tauj;
  const uint32_t Lw = win ? D : 0u;
  const uint32_t Iw = warp_incl(Lw);
  const uint32_t Xw = Iw - Lw, Tw = __shfl_sync(FULL, Iw, 31);
  for (uint32_t it = 0; it < Tw; it += 32u) {
    const uint32_t e = it + lane;
    const uint32_t k = find_set(Xw, e);
    const uint32_t kb = __shfl_sync(FULL, base, k), kd = __shfl_sync(FULL, dst, k);
    const uint32_t kx = __shfl_sync(FULL, Xw, k);
    if (e < Tw) P.cov[__ldcg(P.pk[kd - 1u] + kb + e - kx)] = 1;
  }
  settle(P, S, valid, v, D, dst, act, win, C);
}

// ---- large sets: 256-element chunks over the whole grid --------------------------------

__device__ void large_chunk(const ScParams& P, const ScSmem& S, uint32_t c, int mode, ScCnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const ScList& Lc = P.lg[S.csel];
  const uint32_t cb = c * kScChunk;  // < S.tl
  // the member holding element cb: the last one starting at or before it
  uint32_t lo = 0, hi = S.nl - 1u;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1u) / 2u;
    if (__ldcg(Lc.st + mid) <= cb) lo = mid;
    else hi = mid - 1u;
  }
  const uint32_t i0 = lo;
  // lane l describes member i0 + l
  const uint32_t il = i0 + lane;
  const bool lv = il < S.nl;
  const uint32_t st = lv ? __ldcg(Lc.st + il) : 0xFFFFFFFFu;
  const uint32_t X = lane == 0u ? 0u : (lv ? st - cb : 0xFFFFFFFFu);
  const uint32_t Y = lane == 0u ? cb - st : 0u;  // element cb's offset inside member i0
  uint32_t v = 0, lw = 0, base = 0, D = 0, W = 0;
  unsigned long long key = 0;
  if (lv && X < kScChunk) {
    v = __ldcg(Lc.id + il);
    lw = __ldcg(Lc.lw + il);
    base = __ldg(P.off + v);
    if (mode != kLPack) D = __ldcg(Lc.dn + il);
    if (mode == kLCover) W = __ldcg(Lc.wn + il);
    if (mode == kLClaim || mode == kLCount) key = claim_key(S.step, __ldg(P.pri + v));
    if (mode == kLPack && Y == 0u) ++C.items;
  }
  const uint32_t L = lw & kScLenMask, store = lw >> kScLenBits;
  const uint32_t lim = S.tl - cb;  // elements of the space from cb on
  for (uint32_t it = 0; it < kScChunk; it += 32u) {
    const uint32_t e = it + lane;
    const bool ok = e < lim;
    const uint32_t k = find_set(X, e);
    const uint32_t kb = __shfl_sync(FULL, base, k), ks = __shfl_sync(FULL, store, k);
    const uint32_t kx = __shfl_sync(FULL, X, k), ky = __shfl_sync(FULL, Y, k);
    const uint32_t kl = __shfl_sync(FULL, L, k), kd = __shfl_sync(FULL, D, k);
    const uint32_t o = e - kx + ky;  // offset inside member i0 + k
    if (mode == kLPack) {
      uint32_t u = 0;
      bool keep = false;
      if (ok) {
        if (o < kl) {
          u = elem(P, kb, ks, o);
          keep = __ldcg(P.cov + u) == 0;
          ++C.scanned;
        } else {
          report_bad(P.sync, 57u, c, o);
        }
      }
      const Run r = run_of(keep, k);
      uint32_t at = 0;
      if (lane == r.head && r.count) at = atomicAdd(Lc.dn + i0 + k, r.count);
      at = __shfl_sync(FULL, at, r.head);
      if (keep) {
        const uint32_t pos = at + r.rank;
        if (pos < kl) P.pk[next_store(ks) - 1u][kb + pos] = u;
        else report_bad(P.sync, 58u, kb, pos);
      }
    } else if (mode == kLClaim) {
      const unsigned long long kk = __shfl_sync(FULL, key, k);
      if (ok && kd >= S.tj && o < kd)
        atomicMin(P.claim + __ldcg(P.pk[next_store(ks) - 1u] + kb + o), kk);
    } else if (mode == kLCount) {
      const unsigned long long kk = __shfl_sync(FULL, key, k);
      bool hit = false;
      if (ok && kd >= S.tj && o < kd)
        hit = __ldcg(P.claim + __ldcg(P.pk[next_store(ks) - 1u] + kb + o)) == kk;
      const Run r = run_of(hit, k);
      if (lane == r.head && r.count) atomicAdd(Lc.wn + i0 + k, r.count);
    } else {
      const uint32_t kw = __shfl_sync(FULL, W, k);
      if (ok && kd >= S.tj && kw >= S.tauj && o < kd)
        P.cov[__ldcg(P.pk[next_store(ks) - 1u] + kb + o)] = 1;
    }
  }
}

__device__ __forceinline__ uint32_t chunks(uint32_t tl) {
  return tl / kScChunk + ((tl % kScChunk) ? 1u : 0u);
}

// Phase C, per large member: join or stay, move.
__device__ void large_settle(const ScParams& P, const ScSmem& S, ScCnt& C) {
  const uint32_t lane = threadIdx.x & 31;
  const ScList& Lc = P.lg[S.csel];
  for (uint32_t b0 = gwarp() * 32u; b0 < S.nl; b0 += nwarps() * 32u) {
    const uint32_t i = b0 + lane;
    const bool valid = i < S.nl;
    uint32_t v = 0, lw = 0, D = 0, W = 0;
    if (valid) {
      v = __ldcg(Lc.id + i);
      lw = __ldcg(Lc.lw + i);
      D = __ldcg(Lc.dn + i);
      W = __ldcg(Lc.wn + i);
    }
    const bool act = valid && D >= S.tj;
    const bool win = act && W >= S.tauj;
    settle(P, S, valid, v, D, next_store(lw >> kScLenBits), act, win, C);
  }
}

// ---- phases ----------------------------------------------------------------------------

__device__ void gather_phase(const ScParams& P, const ScSmem& S) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t b = S.band;
  const uint32_t cap = __ldg(P.bcap + b);
  const uint32_t sel = __ldcg(P.bsel + b);
  const uint32_t cnt = min(S.gn, cap);
  const unsigned long long* src = P.bl + __ldg(P.bbase + b) + (unsigned long long)sel * cap;
  unsigned long long* dst = P.bl + __ldg(P.bbase + b) + (unsigned long long)(sel ^ 1u) * cap;
  for (uint32_t b0 = gwarp() * 32u; b0 < cnt; b0 += nwarps() * 32u) {
    const uint32_t i = b0 + lane;
    const bool ok = i < cnt;
    const unsigned long long e = ok ? __ldcg(src + i) : 0ull;
    const uint32_t j = (uint32_t)(e >> 32), v = (uint32_t)e;
    const bool mem = ok && j == S.j;
    const bool keep = ok && !mem;
    const unsigned m = __ballot_sync(FULL, keep);
    if (m) {
      const uint32_t leader = (uint32_t)__ffs(m) - 1u;
      uint32_t at = 0;
      if (lane == leader) at = atomicAdd(&P.ss->gcnt, (uint32_t)__popc(m));
      at = __shfl_sync(FULL, at, leader);
      const uint32_t jm = __reduce_max_sync(FULL, keep ? j : 0u);
      if (lane == leader) atomicMax(&P.ss->gmax, jm);
      if (keep) {
        const uint32_t pos = at + (uint32_t)__popc(m & lanemask_lt());
        if (pos < cap) dst[pos] = e;
        else report_bad(P.sync, 59u, b, pos);
      }
    }
    const uint32_t lw = mem ? __ldcg(P.len + v) : 0u;
    list_insert(P, S.csel, mem, v, lw, lw & kScLenMask);
  }
}

__device__ void phase_a(const ScParams& P, const ScSmem& S, ScCnt& C) {
  const uint32_t G = (S.ns + 31u) / 32u, K = S.nl ? chunks(S.tl) : 0u;
  for (uint32_t u = gwarp(); u < G + K; u += nwarps()) {
    if (u < G) small_a(P, S, u, C);
    else large_chunk(P, S, u - G, kLPack, C);
  }
}

__device__ void phase_a2(const ScParams& P, const ScSmem& S, ScCnt& C) {
  const uint32_t K = S.nl ? chunks(S.tl) : 0u;
  for (uint32_t u = gwarp(); u < K; u += nwarps()) large_chunk(P, S, u, kLClaim, C);
}

__device__ void phase_b(const ScParams& P, const ScSmem& S, ScCnt& C) {
  const uint32_t G = (S.ns + 31u) / 32u, K = S.nl ? chunks(S.tl) : 0u;
  for (uint32_t u = gwarp(); u < G + K; u += nwarps()) {
    if (u < G) small_b(P, S, u, C);
    else large_chunk(P, S, u - G, kLCount, C);
  }
}

__device__ void phase_c(const ScParams& P, const ScSmem& S, ScCnt& C) {
  const uint32_t K = S.nl ? chunks(S.tl) : 0u;
  for (uint32_t u = gwarp(); u < K; u += nwarps()) large_chunk(P, S, u, kLCover, C);
  large_settle(P, S, C);
}

// The decider's view of ScState: lane i loads word i in one round trip (every other CTA
// has arrived, so no word changes any more; the error word rides in lane 31), and each
// field is taken from its lane by a shuffle, so every lane sees the same value (lane 0
// also rewrites some of these words, and the lanes of a warp are not guaranteed to run in
// lockstep: a lane reading a word itself could see the new value while the others saw the
// old one, decide differently and leave the others waiting in a collective).
constexpr uint32_t kScStateWords = sizeof(ScState) / 4;
static_assert(kScStateWords <= 31 && sizeof(ScState) % 8 == 0,
              "ScState and the error word fit one warp load");
#define SS_WORD(f) ((uint32_t)(offsetof(ScState, f) / 4))

// Run by warp 0 of the CTA that arrives last at a grid barrier: the next phase.  Every
// value a decision depends on is warp-uniform: the state block is read once (snapshot),
// the band arrays through ballots.
__device__ void sc_decide(const ScParams& P, uint32_t done) {
  const uint32_t lane = threadIdx.x & 31;
  ScState* ss = P.ss;
  const uint32_t snap = lane < kScStateWords
                            ? __ldcg(reinterpret_cast<const uint32_t*>(ss) + lane)
                            : (lane == 31 ? ld_relaxed(&P.sync->err) : 0u);
  auto F = [&](uint32_t w) -> uint32_t { return __shfl_sync(FULL, snap, (int)w); };
  const bool fatal = (F(31) & kErrFatal) != 0u;
  uint32_t next = kScStop;
  auto large_n = [&](uint32_t sel) -> uint32_t {  // entries of large member list sel
    const uint32_t lo = F(SS_WORD(bw) + 2 * sel), hi = F(SS_WORD(bw) + 2 * sel + 1);
    return (uint32_t)((((unsigned long long)hi << 32) | lo) >> kScCntShift);
  };
  // The highest non-empty band at or below `from`; its largest bucket is gathered next.
  auto transition = [&](int from) -> uint32_t {
    const uint32_t gathers = F(SS_WORD(gathers));
    for (int top = from; top >= 0; top -= 32) {
      const int b = top - (int)lane;
      const bool ne = b >= 0 && __ldcg(P.bcnt + b) > 0u;
      const unsigned m = __ballot_sync(FULL, ne);
      if (m) {
        const int bb = top - (__ffs(m) - 1);
        if (lane == 0) {
          ss->band = (uint32_t)bb;
          ss->j = __ldcg(P.bmax + bb);
          ss->gmax = 0u;
          ss->gcnt = 0u;
          ss->ns[0] = ss->ns[1] = 0u;
          ss->bw[0] = ss->bw[1] = 0ull;
          ss->gathers = gathers + 1u;
        }
        return kScGather;
      }
    }
    return kScStop;
  };
  // A step either adds a set to the cover or empties its bucket (every member leaves or
  // moves down), so a run takes at most n + nb steps; more means a broken invariant.
  auto start_step = [&]() -> uint32_t {
    const uint32_t s = F(SS_WORD(step)) + 1u;
    const uint32_t j = F(SS_WORD(j));
    if ((unsigned long long)s > (unsigned long long)P.n + P.nb + 1ull) {
      if (lane == 0) report_bad(P.sync, 63u, s, j);
      return kScStop;
    }
    if (lane == 0) {
      ss->step = s;
      P.stats->v[kStRounds] += 1ull;
    }
    return kScA;
  };
  if (!fatal) {
    const uint32_t c = F(SS_WORD(csel)) & 1u;
    switch (done) {
      case kScPrologue:
        next = transition((int)P.nbands - 1);
        break;
      case kScGather: {
        const uint32_t b = F(SS_WORD(band));
        const uint32_t gcnt = F(SS_WORD(gcnt)), gmax = F(SS_WORD(gmax));
        if (lane == 0) {
          P.bsel[b] = __ldcg(P.bsel + b) ^ 1u;
          P.bcnt[b] = gcnt;
          P.bmax[b] = gmax;
        }
        if (F(SS_WORD(ns) + c) + large_n(c) == 0u) {
          const uint32_t j = F(SS_WORD(j));
          if (lane == 0) report_bad(P.sync, 54u, j, b);
          next = kScStop;
        } else {
          next = start_step();
        }
        break;
      }
      case kScA:
        next = large_n(c) ? kScA2 : kScB;
        break;
      case kScA2:
        next = kScB;
        break;
      case kScB:
      case kScC: {
        if (done == kScB && large_n(c)) {
          next = kScC;
          break;
        }
        const uint32_t x = c ^ 1u;
        if (F(SS_WORD(ns) + x) + large_n(x) > 0u) {
          if (lane == 0) {
            ss->csel = x;
            ss->ns[c] = 0u;
            ss->bw[c] = 0ull;
          }
          next = start_step();
        } else {
          next = transition((int)F(SS_WORD(band)));
        }
        break;
      }
      default:
        next = kScStop;
    }
  }
  __syncwarp();
  if (lane == 0) P.sync->phase = next;
}
#undef SS_WORD

// Bounded grid barrier: the last CTA to arrive runs sc_decide and releases the others,
// who give up after spin_ns or on a fatal error.
__device__ void sc_barrier(const ScParams& P, ScSmem& S, uint32_t& bar, uint32_t done) {
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
    if (threadIdx.x < 32) sc_decide(P, done);
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
    // decider's writes, so they can be issued together.
    S.phase = ld_relaxed(&P.sync->phase);
    S.err = ld_relaxed(&P.sync->err);
    const ScState* ss = P.ss;
    S.j = __ldcg(&ss->j);
    S.step = __ldcg(&ss->step);
    S.csel = __ldcg(&ss->csel) & 1u;
    S.band = __ldcg(&ss->band);
    S.ns = min(__ldcg(&ss->ns[S.csel]), P.n);
    const unsigned long long bw = __ldcg(&ss->bw[S.csel]);
    S.nl = (uint32_t)min(bw >> kScCntShift, (unsigned long long)P.lg_cap);
    S.tl = (uint32_t)min(bw & kScTotMask, 0xFFFFFFFFull);
    const uint32_t jj = S.j < P.nb ? S.j : 0u;
    S.tj = P.nb ? __ldg(P.t + jj) : 1u;
    S.tauj = P.nb ? __ldg(P.tau + jj) : 1u;
    S.gn = S.band < P.nbands ? __ldcg(P.bcnt + S.band) : 0u;
    S.t_bar += gtimer() - t_in;
  }
  __syncthreads();
  ++bar;
}

}  // namespace

extern "C" __global__ void __launch_bounds__(kBlock, 4) og_setcover_kernel(ScParams P) {
  __shared__ ScSmem S;
  ScCnt C = {0, 0, 0, 0};
  uint32_t bar = 0;
  if (threadIdx.x == 0) S.t_bar = S.t_a = S.t_b = S.t_g = 0ull;
  sc_barrier(P, S, bar, kScPrologue);
  for (;;) {
    const uint32_t phase = S.phase;
    if (phase == kScStop || (S.err & kErrFatal)) break;
    const uint64_t t0 = threadIdx.x == 0 ? gtimer() : 0ull;
    if (phase == kScGather) gather_phase(P, S);
    else if (phase == kScA) phase_a(P, S, C);
    else if (phase == kScA2) phase_a2(P, S, C);
    else if (phase == kScB) phase_b(P, S, C);
    else if (phase == kScC) phase_c(P, S, C);
    if (threadIdx.x == 0) {
      const uint64_t dt = gtimer() - t0;
      if (phase == kScGather) S.t_g += dt;
      else if (phase == kScA || phase == kScA2) S.t_a += dt;
      else S.t_b += dt;
    }
    sc_barrier(P, S, bar, phase);
  }
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t vals[4] = {C.items, C.scanned, C.chosen, C.moved};
  const int idx[4] = {kStItems, kStRelax, kStImproved, kStGlobal};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t s = warp_sum(vals[q]);
    if (lane == 0 && s) atomicAdd(&P.stats->v[idx[q]], (unsigned long long)s);
  }
  if (threadIdx.x == 0) {
    atomicAdd(&P.stats->v[kStTBarrier], S.t_bar);
    atomicAdd(&P.stats->v[kStTFrontier], S.t_a);
    atomicAdd(&P.stats->v[kStTFused], S.t_b);
    atomicAdd(&P.stats->v[kStTHub], S.t_g);
  }
}

// Per set: residual = degree (storage 0), nothing covered or claimed, not chosen; the
// priority is checked to be a permutation; sets are counted per first band.
extern "C" __global__ void og_setcover_init_kernel(ScParams P) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t b0 = blockIdx.x * blockDim.x; b0 < P.n; b0 += stride) {
    const uint32_t v = b0 + threadIdx.x;
    const bool ok = v < P.n;
    uint32_t deg = 0;
    if (ok) {
      deg = __ldg(P.off + v + 1) - __ldg(P.off + v);
      P.len[v] = deg;
      P.cov[v] = 0;
      P.claim[v] = 0xFFFFFFFFFFFFFFFFull;
      P.step_out[v] = 0u;
      const uint32_t p = __ldg(P.pri + v);
      if (p >= P.n) {
        report_bad(P.sync, kScBadPriority, v, p);
      } else {
        const uint32_t bit = 1u << (p & 31u);
        if (atomicOr(P.seen + (p >> 5), bit) & bit) report_bad(P.sync, kScBadPriority, v, p);
      }
    }
    const bool live = ok && deg > 0u && P.nb > 0u;
    const uint32_t b = live ? bucket_of_size(P, deg) / kScBand : 0u;
    const unsigned m = __match_any_sync(FULL, live ? b : (0x80000000u | lane));
    if (live && lane == (uint32_t)__ffs(m) - 1u) {
      if (b < P.nbands) atomicAdd(P.hist + b, (uint32_t)__popc(m));
      else report_bad(P.sync, 61u, v, b);
    }
  }
}

// Band capacities (sets whose first band is at or above b) and buffer offsets.
extern "C" __global__ void og_setcover_plan_kernel(ScParams P) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t* cap = const_cast<uint32_t*>(P.bcap);
  unsigned long long* base = const_cast<unsigned long long*>(P.bbase);
  uint32_t suffix = 0;
  for (uint32_t b = P.nbands; b-- > 0;) {
    suffix += P.hist[b];
    cap[b] = suffix;
  }
  unsigned long long acc = 0;
  for (uint32_t b = 0; b < P.nbands; ++b) {
    base[b] = acc;
    acc += 2ull * cap[b];
  }
  if (acc > P.bl_entries) report_bad(P.sync, 62u, (uint32_t)(acc >> 32), (uint32_t)acc);
}

// Every set with elements goes to the band of its first bucket (buffer 0).
extern "C" __global__ void og_setcover_fill_kernel(ScParams P) {
  if (ld_relaxed(&P.sync->err) & kErrFatal) return;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t b0 = blockIdx.x * blockDim.x; b0 < P.n; b0 += stride) {
    const uint32_t v = b0 + threadIdx.x;
    const bool ok = v < P.n;
    const uint32_t deg = ok ? __ldg(P.off + v + 1) - __ldg(P.off + v) : 0u;
    const bool live = deg > 0u && P.nb > 0u;
    band_insert(P, live, live ? bucket_of_size(P, deg) : 0u, v);
  }
}

extern "C" __global__ void og_setcover_iota_kernel(uint32_t* p, uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    p[v] = v;
}

cudaError_t setcover_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, og_setcover_kernel, kBlock,
                                                       0);
}

cudaError_t launch_setcover(const ScParams& P, int grid, cudaStream_t st) {
  void* args[] = {const_cast<ScParams*>(&P)};
  return cudaLaunchCooperativeKernel((const void*)og_setcover_kernel, dim3(grid), dim3(kBlock),
                                     args, 0, st);
}

cudaError_t launch_setcover_prep(const ScParams& P, uint32_t* iota, int sms, cudaStream_t st) {
  if (iota) og_setcover_iota_kernel<<<sms * 4, 256, 0, st>>>(iota, P.n);
  og_setcover_init_kernel<<<sms * 4, 256, 0, st>>>(P);
  og_setcover_plan_kernel<<<1, 32, 0, st>>>(P);
  og_setcover_fill_kernel<<<sms * 4, 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace og
