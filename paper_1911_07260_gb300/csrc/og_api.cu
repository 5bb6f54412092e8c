// Host side of libog: the C ABI declared in include/og.h.
//
// Every call validates its arguments on the host, stages query descriptors through
// pinned memory, and runs the Delta-stepping kernels of og_kernels.cu on the caller's
// stream.  Scratch (bucket rings, overflow piles, query cursors) is owned by the graph
// (single queries, batches) or by a server, grown on demand and reused across calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "og.h"
#include "og_internal.cuh"
#include "og_kcore.cuh"
#include "og_setcover.cuh"

namespace og {
cudaError_t launch_delta(const Params& P, int grid, size_t smem, cudaStream_t st);
cudaError_t delta_occupancy(int* blocks_per_sm, size_t smem, bool ell);
cudaError_t launch_ell(const uint32_t* off, const uint2* adj, uint4* ell, uint32_t n, int sms,
                       cudaStream_t st);
cudaError_t launch_fill(uint32_t* dist, uint32_t n, const uint32_t* slots, uint32_t nslots,
                        int sms, cudaStream_t st);
cudaError_t launch_init(const Params& P, const uint32_t* slots, uint32_t nslots,
                        cudaStream_t st);
cudaError_t launch_interleave(const uint32_t* nbr, const uint32_t* w, uint2* adj, size_t m,
                              uint32_t n, uint32_t* flags, int sms, cudaStream_t st);
cudaError_t launch_check_csr(const uint32_t* off, const uint2* adj, uint32_t n, uint32_t m,
                             uint32_t* flags, int sms, cudaStream_t st);
cudaError_t launch_indeg(const uint32_t* off, const uint2* adj, uint32_t n, uint32_t* deg, int sms,
                         cudaStream_t st);
cudaError_t launch_transpose(const uint32_t* off, const uint2* adj, uint32_t n, const uint32_t* toff,
                             uint32_t* cursor, uint2* tadj, int sms, cudaStream_t st);
cudaError_t launch_async(const AParams& P, int grid, size_t smem, cudaStream_t st);
cudaError_t async_occupancy(int* blocks_per_sm, size_t smem, bool ell);
cudaError_t launch_async_init(const AParams& P, const uint32_t* slots, uint32_t nslots,
                              cudaStream_t st);
cudaError_t launch_touch_reset(uint32_t* dist, uint32_t n, uint32_t* touched, uint32_t tb_words,
                               const uint32_t* slots, uint32_t nslots, int sms, cudaStream_t st);
cudaError_t kcore_occupancy(int* blocks_per_sm);
cudaError_t launch_kcore(const KParams& P, int grid, cudaStream_t st);
cudaError_t launch_kcore_init(const uint32_t* off, uint32_t* prio, uint32_t n, int sms,
                              cudaStream_t st);
cudaError_t setcover_occupancy(int* blocks_per_sm);
cudaError_t launch_setcover(const ScParams& P, int grid, cudaStream_t st);
cudaError_t launch_setcover_prep(const ScParams& P, uint32_t* iota, int sms, cudaStream_t st);
cudaError_t launch_pack_adj(const uint32_t* off_old, const uint2* adj_old,
                            const uint32_t* off_new, const uint32_t* src_of,
                            const uint32_t* new_of, uint2* adj_new, uint32_t n, int sms,
                            cudaStream_t st);
cudaError_t launch_perm_rows(uint32_t* rows, uint32_t n, uint32_t nrows, const uint2* mv,
                             uint32_t nmv, bool to_user, uint32_t* tmp, int sms,
                             cudaStream_t st);
}  // namespace og

using namespace og;

namespace {

thread_local char g_cuda_msg[512] = "";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? OG_E_OOM : OG_E_CUDA;
}

#define CK(x)                                          \
  do {                                                 \
    cudaError_t _e = (x);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #x);   \
  } while (0)

#define TRY(x)                    \
  do {                            \
    int _r = (x);                 \
    if (_r != OG_OK) return _r;   \
  } while (0)

// Status of a finished persistent launch from the error word it left in Sync: a failed
// internal bounds check first (its code, value and context go to the message), then a
// bounded wait that gave up, then a query that ran out of bucket space where the arena
// cannot grow (arena_out), then a saturated distance.  Every entry point that runs the
// round engine maps its launches through this one function.
int launch_status(uint32_t err, uint32_t bad_code, uint32_t bad_val, uint32_t bad_aux,
                  bool arena_out) {
  if (err & kErrBounds) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "check %u failed: value %u, context %u",
             bad_code, bad_val, bad_aux);
    return OG_E_INTERNAL;
  }
  if (err & kErrTimeout) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "grid barrier wait gave up");
    return OG_E_TIMEOUT;
  }
  if (arena_out) return OG_E_ARENA;
  if (err & kErrSat) return OG_E_OVERFLOW;
  return OG_OK;
}

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t b) {
    if (b <= bytes && p) return OG_OK;
    release();
    cudaError_t e = cudaMalloc(&p, b ? b : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "cudaMalloc");
    }
    bytes = b;
    return OG_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

struct HBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t b) {
    if (b <= bytes && p) return OG_OK;
    release();
    cudaError_t e = cudaMallocHost(&p, b ? b : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "cudaMallocHost");
    }
    bytes = b;
    return OG_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Device scratch of one launch configuration (grown on demand, reused across calls).
struct Workspace {
  DBuf dist, ring, counts, ovf, qs, qd, pref, sync, stats, slots, aq, big, bmap;
  DBuf stouched;  // server: touched-block bitmaps of the slots' distance rows
  DBuf permtmp;   // staging of the moved entries when rows change vertex order
  DBuf kprio, kcnt, ktouched, klist, kring, kcounts, klossy, kstate;  // k-core
  DBuf lzbits, lzlist;  // lazy bucket update
  DBuf sclad, sclen, scpk, sccov, scclaim, scseen, scmeta, scbase, scbl, scsm, sclg, scstate,
      scpri, scout;  // set cover
  HBuf h_qd, h_qs, h_sync, h_stats, h_slots, h_aq, h_kstate;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // Barrier-free engine: ring positions must read "free" (all ones) before use.  Entries
  // [0, clean_upto) of the ring are known free except the listed dirty ranges.
  uint64_t clean_upto = 0;
  std::vector<std::pair<uint64_t, uint64_t>> dirty;
  void* ring_ptr = nullptr;
  void release() {
    for (DBuf* b : {&dist, &ring, &counts, &ovf, &qs, &qd, &pref, &sync, &stats, &slots, &aq,
                    &stouched, &permtmp, &big, &bmap, &kprio, &kcnt, &ktouched, &klist, &kring, &kcounts, &klossy,
                    &kstate, &lzbits, &lzlist, &sclad, &sclen, &scpk, &sccov, &scclaim, &scseen,
                    &scmeta, &scbase, &scbl, &scsm, &sclg, &scstate, &scpri, &scout})
      b->release();
    for (HBuf* b : {&h_qd, &h_qs, &h_sync, &h_stats, &h_slots, &h_aq, &h_kstate}) b->release();
    clean_upto = 0;
    dirty.clear();
    ring_ptr = nullptr;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    e0 = e1 = nullptr;
  }
  int events() {
    if (!e0) CK(cudaEventCreate(&e0));
    if (!e1) CK(cudaEventCreate(&e1));
    return OG_OK;
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

uint32_t pow2_floor(double x) {
  if (!(x >= 1.0)) return 1u;
  if (x >= 2147483648.0) return 1u << 31;
  uint32_t p = 1;
  while ((double)p * 2.0 <= x) p <<= 1;
  return p;
}

uint32_t pow2_ceil(uint64_t x) {
  uint32_t p = 1;
  while (p < x && p < (1u << 31)) p <<= 1;
  return p;
}

constexpr uint32_t kDefaultFusion = 1024;
constexpr int kEllWidthHost = 8;
constexpr uint32_t kTileSparse = 32;    // frontier tile, average degree <= 8
constexpr uint32_t kTileDense = 256;    // frontier tile, denser graphs
constexpr uint32_t kBinCap = 2048;
constexpr uint32_t kDefaultHub = 4096;      // out-degree from which a vertex is a hub
constexpr uint32_t kHubSlots = 65536;       // hubs listed per round
constexpr uint32_t kHubChunks = 1u << 20;   // 1024-edge hub chunks per round
constexpr uint32_t kKcoreHub = 256;         // k-core: default hub out-degree
constexpr uint32_t kSetcoverHub = 32;       // set cover: residual size of a large set
constexpr int kSetcoverBps = 4;             // set cover: default CTAs per SM
constexpr int kKcoreBps = 2;                // k-core: default CTAs per SM
constexpr uint64_t kDefaultSpinNs = 2000000000ull;
// Hot-first packing: the n / kHotDiv vertices of largest degree move to ids [0, n / kHotDiv),
// in order of degree, when the graph has at least kHotMinN vertices and those vertices
// hold at least half of the edges (a power-law degree distribution; a road network's top
// eighth holds ~15%).
constexpr uint32_t kHotDiv = 8;
constexpr uint32_t kHotMinN = 1u << 20;

}  // namespace

struct og_graph {
  uint32_t n = 0;
  uint64_t m = 0;
  uint32_t min_w = 0, max_w = 0;
  double mean_w = 0.0;
  uint32_t* off = nullptr;
  uint2* adj = nullptr;
  uint4* ell = nullptr;      // ELL-8 rows when every degree is <= 8
  uint32_t* toff = nullptr;  // transpose (in-edges), built the first time a pull is asked for
  uint2* tadj = nullptr;
  uint32_t max_deg = 0;
  float2* xy = nullptr;
  std::vector<float> h_xy;   // host copy: target coordinates of A* queries
  bool xy_integral = false;
  og_config cfg{};
  Workspace ws;
  int sms = 0;
  int occ = 0;
  int occ_async = 0;
  int occ_l[2] = {0, 0};        // round engine: CTAs per SM for CSR / ELL
  int occ_async_l[2] = {0, 0};  // barrier-free engine
  // Vertex order on the device.  Empty h_pi: the user's ids.  Otherwise device id x holds
  // user vertex h_pi[x] and user vertex v has device id h_dev[v]; every id crossing the
  // boundary goes through them, every per-vertex array through the moved list mv
  // ({device id, user id} of the nmv vertices whose ids differ; og_order.cu).
  std::vector<uint32_t> h_pi, h_dev;
  uint2* mv = nullptr;
  uint32_t nmv = 0;
  uint32_t servers = 0;         // live servers: their slots hold rows in the device order
};

struct og_server {
  og_graph* g = nullptr;
  og_config cfg{};
  cudaStream_t stream = nullptr;
  uint32_t slots = 0, B = 0, cap = 0, ocap = 0;
  Workspace ws;
  std::vector<QDesc> hq;
  std::vector<uint64_t> tags;
  std::vector<uint8_t> state;   // 0 free, 1 admitted (not started), 2 running, 3 finished
  std::vector<uint32_t> results;
  std::vector<uint32_t> free_list;
  std::vector<uint32_t> pending;
  std::deque<uint32_t> done;
  bool started = false;
};

namespace {

uint32_t default_delta(const og_graph* g) {
  const double avg_deg = g->n ? (double)g->m / g->n : 0.0;
  const double mw = g->mean_w > 0 ? g->mean_w : 1.0;
  // Low-degree, large-diameter graphs want a wide bucket for parallelism; dense
  // small-diameter graphs a narrow one for work efficiency (Section 6.2, Delta selection).
  return avg_deg <= 8.0 ? pow2_floor(16.0 * mw) : pow2_floor(std::max(1.0, mw / 4.0));
}

// Effective schedule: explicit call config, then graph default, then library default.
og_config resolve(const og_graph* g, const og_config* user) {
  og_config d;
  og_config_default(&d);
  og_config r = d;
  auto pick32 = [](uint32_t a, uint32_t b, uint32_t c) { return a ? a : (b ? b : c); };
  auto pick64 = [](uint64_t a, uint64_t b, uint64_t c) { return a ? a : (b ? b : c); };
  const og_config z{};
  const og_config& u = user ? *user : z;
  r.delta = pick32(u.delta, g->cfg.delta, default_delta(g));
  r.fusion_threshold = pick32(u.fusion_threshold, g->cfg.fusion_threshold, kDefaultFusion);
  // Sparse graphs: small tiles spread a narrow frontier over many CTAs, whose fused loops
  // then carry the work; dense graphs: a tile of one entry per thread amortises the
  // claim and the degree scan of the CTA-wide expansion.
  const uint32_t tile = (g->n && (double)g->m / g->n > 8.0) ? kTileDense : kTileSparse;
  r.expand_tile = pick32(u.expand_tile, g->cfg.expand_tile, tile);
  r.blocks_per_sm = pick32(u.blocks_per_sm, g->cfg.blocks_per_sm, 0);
  r.ring_buckets = pick32(u.ring_buckets, g->cfg.ring_buckets, 0);
  r.hub_degree = pick32(u.hub_degree, g->cfg.hub_degree, kDefaultHub);
  r.bucket_update = pick32(u.bucket_update, g->cfg.bucket_update, OG_UPDATE_EAGER);
  r.spin_limit_ns = pick64(u.spin_limit_ns, g->cfg.spin_limit_ns, kDefaultSpinNs);
  r.arena_entries = pick64(u.arena_entries, g->cfg.arena_entries, 0);
  r.engine = u.engine ? u.engine : g->cfg.engine;
  r.pull_divisor = u.pull_divisor ? u.pull_divisor : g->cfg.pull_divisor;
  r.precheck = u.precheck ? u.precheck : g->cfg.precheck;
  r.layout = u.layout ? u.layout : g->cfg.layout;
  // layout 0 stays "automatic": the round engine picks its ELL row path (two dependent
  // round trips per fused level instead of three, measured faster) on graphs with ELL
  // rows when no A* query is in the launch, CSR otherwise (run_chunk_rounds).
  r.prefetch = u.prefetch ? u.prefetch : (g->cfg.prefetch ? g->cfg.prefetch : OG_PREFETCH_OFF);
  if (r.layout == OG_LAYOUT_ELL && !g->ell) r.layout = OG_LAYOUT_CSR;
  if (!r.precheck)
    r.precheck = (g->n && (double)g->m / g->n > 8.0) ? OG_PRECHECK_ON : OG_PRECHECK_OFF;
  return r;
}

// Default bucket arena per query: large enough that buckets rarely spill into the
// overflow pile (a spill costs two grid-wide redistribution passes) -- 48n entries for
// dense graphs, 12n otherwise -- within 60% of the free device memory shared by the nq
// queries of a launch, and at least 6n entries.
uint64_t default_arena(const og_graph* g, uint32_t nq) {
  const uint64_t lo = std::max<uint64_t>(6ull * g->n, 1ull << 16);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return lo;
  }
  const uint64_t budget = (uint64_t)((double)fr * 0.6) / sizeof(uint2) / std::max(1u, nq);
  // Dense graphs have large buckets spread over many materialised slots.
  const uint64_t want = (g->n && (double)g->m / g->n > 8.0 ? 48ull : 12ull) * g->n;
  return std::max(lo, std::min<uint64_t>(want, budget));
}

uint32_t ring_size(const og_graph* g, const og_config& c, uint32_t min_delta) {
  if (c.ring_buckets) {
    uint32_t b = pow2_ceil(c.ring_buckets);
    return std::max(2u, std::min<uint32_t>(b, kMaxRing));
  }
  // Enough materialised buckets that one relaxation never jumps past the ring.
  const uint64_t span = (uint64_t)g->max_w / std::max(1u, min_delta) + 2;
  return std::max(2u, std::min<uint32_t>(pow2_ceil(span), kMaxRing));
}

int occupancy(og_graph* g, size_t smem, bool ell) {
  if (!g->occ_l[ell]) {
    int dev = 0, b = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
    CK(delta_occupancy(&b, smem, ell));
    if (b < 1) {
      snprintf(g_cuda_msg, sizeof(g_cuda_msg), "persistent kernel does not fit on an SM");
      return OG_E_CUDA;
    }
    g->occ_l[ell] = b;
  }
  g->occ = g->occ_l[ell];
  return OG_OK;
}

struct RunOut {
  uint32_t err = 0;
  uint64_t restarts = 0;
};

// The in-edge lists of the graph (for pull rounds), built on the device the first time a
// pull is asked for and kept with the graph: in-degrees, their prefix sums (on the
// host), then a scatter of every edge.
int ensure_transpose(og_graph* g, cudaStream_t st) {
  if (g->toff) return OG_OK;
  const uint32_t n = g->n;
  uint32_t* toff = nullptr;
  uint32_t* cur = nullptr;
  uint2* tadj = nullptr;
  std::vector<uint32_t> h(n + 1, 0u);
  int dev = 0;
  auto fail = [&](cudaError_t e, const char* what) {
    if (toff) cudaFree(toff);
    if (cur) cudaFree(cur);
    if (tadj) cudaFree(tadj);
    return cuda_fail(e, what);
  };
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && !g->sms)
    e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(e, "device query");
  if ((e = cudaMalloc(&toff, sizeof(uint32_t) * ((size_t)n + 1))) != cudaSuccess ||
      (e = cudaMalloc(&cur, sizeof(uint32_t) * (size_t)n)) != cudaSuccess ||
      (e = cudaMalloc(&tadj, sizeof(uint2) * std::max<uint64_t>(1, g->m))) != cudaSuccess)
    return fail(e, "transpose allocation");
  if ((e = cudaMemsetAsync(cur, 0, sizeof(uint32_t) * (size_t)n, st)) != cudaSuccess ||
      (e = launch_indeg(g->off, g->adj, n, cur, g->sms, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h.data(), cur, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "in-degrees");
  uint32_t run = 0;
  for (uint32_t v = 0; v < n; ++v) {
    const uint32_t x = h[v];
    h[v] = run;
    run += x;
  }
  h[n] = run;
  if ((e = cudaMemcpyAsync(toff, h.data(), sizeof(uint32_t) * ((size_t)n + 1),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(cur, 0, sizeof(uint32_t) * (size_t)n, st)) != cudaSuccess ||
      (e = launch_transpose(g->off, g->adj, n, toff, cur, tadj, g->sms, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "transpose");
  cudaFree(cur);
  g->toff = toff;
  g->tadj = tadj;
  return OG_OK;
}

// Round-synchronous engine: up to kMaxQ queries in one persistent launch, regrowing the
// arena when a query runs out of bucket space.  dist_dev: nq*n device words (query i at
// + i*n).
int run_chunk_rounds(og_graph* g, Workspace& ws, const QDesc* qd, uint32_t nq, const og_config& c,
              uint32_t* dist_dev, uint32_t* d_out, Stats* acc, RunOut* ro, cudaStream_t st) {
  const size_t smem = delta_smem_bytes(kBinCap);
  uint32_t min_delta = 0xFFFFFFFFu;
  bool astar = false;
  for (uint32_t i = 0; i < nq; ++i) {
    if (qd[i].kind != kBF) min_delta = std::min(min_delta, qd[i].delta);  // BF: 2 buckets
    astar |= qd[i].kind == kASTAR;
  }
  // The lazy bucket update marks vertices instead of inserting them: CSR kernel only.
  // An automatic layout takes the ELL rows when they exist and no A* query is in the
  // launch (on ELL rows the A* heuristic costs a dependent load after the atomics).
  const bool ell = g->ell && c.bucket_update != OG_UPDATE_LAZY &&
                   (c.layout == OG_LAYOUT_ELL || (c.layout == 0 && !astar));
  TRY(occupancy(g, smem, ell));
  const uint32_t B = ring_size(g, c, min_delta);
  uint64_t entries = c.arena_entries ? c.arena_entries : default_arena(g, nq);
  TRY(ws.events());
  TRY(ws.h_qd.ensure(sizeof(QDesc) * nq));
  TRY(ws.h_qs.ensure(sizeof(QState) * nq));
  TRY(ws.h_sync.ensure(sizeof(Sync)));
  TRY(ws.h_stats.ensure(sizeof(Stats)));
  memcpy(ws.h_qd.p, qd, sizeof(QDesc) * nq);
  std::vector<uint32_t> pending(nq);
  for (uint32_t i = 0; i < nq; ++i) pending[i] = i;

  for (int attempt = 0;; ++attempt) {
    const uint64_t cap64 = std::max<uint64_t>(64, entries / 2 / B);
    const uint64_t ocap64 = std::max<uint64_t>(64, entries / 4);
    if (cap64 >= 0xFFFFFFF0ull || ocap64 >= 0xFFFFFFF0ull) return OG_E_ARENA;
    const uint32_t cap = (uint32_t)cap64, ocap = (uint32_t)ocap64;
    const uint32_t np = (uint32_t)pending.size();
    TRY(ws.ring.ensure(sizeof(uint2) * (size_t)nq * B * cap));
    TRY(ws.counts.ensure(sizeof(uint32_t) * (size_t)nq * B));
    TRY(ws.ovf.ensure(sizeof(uint2) * (size_t)nq * 2 * ocap));
    TRY(ws.qs.ensure(sizeof(QState) * nq));
    TRY(ws.qd.ensure(sizeof(QDesc) * nq));
    TRY(ws.pref.ensure(sizeof(uint32_t) * (nq + 1)));
    TRY(ws.sync.ensure(sizeof(Sync)));
    TRY(ws.stats.ensure(sizeof(Stats)));
    TRY(ws.slots.ensure(sizeof(uint32_t) * nq));
    TRY(ws.h_slots.ensure(sizeof(uint32_t) * nq));
    memcpy(ws.h_slots.p, pending.data(), sizeof(uint32_t) * np);
    const uint32_t big_cap = g->max_deg >= c.hub_degree ? kHubSlots : 0u;
    if (big_cap) {
      TRY(ws.big.ensure(sizeof(BigItem) * big_cap));
      TRY(ws.bmap.ensure(sizeof(uint32_t) * kHubChunks));
    }

    Params P{};
    P.off = g->off;
    P.adj = g->adj;
    P.ell = ell ? g->ell : nullptr;
    P.xy = g->xy;
    P.n = g->n;
    P.xy_integral = g->xy_integral ? 1u : 0u;
    P.dist = dist_dev;
    P.qd = ws.qd.as<QDesc>();
    P.qs = ws.qs.as<QState>();
    P.ring = ws.ring.as<uint2>();
    P.counts = ws.counts.as<uint32_t>();
    P.ovf = ws.ovf.as<uint2>();
    P.fr_pref = ws.pref.as<uint32_t>();
    P.sync = ws.sync.as<Sync>();
    P.stats = ws.stats.as<Stats>();
    P.big = big_cap ? ws.big.as<BigItem>() : nullptr;
    P.big_map = big_cap ? ws.bmap.as<uint32_t>() : nullptr;
    P.big_cap = big_cap;
    P.map_cap = big_cap ? kHubChunks : 0u;
    P.hub_min = c.hub_degree;
    P.nq = nq;
    P.B = B;
    P.Bmask = B - 1;
    P.cap = cap;
    P.ocap = ocap;
    P.T = c.fusion_threshold == OG_FUSION_OFF ? 0u : c.fusion_threshold;
    P.tile = std::max<uint32_t>(32, (c.expand_tile + 31) / 32 * 32);
    P.bin_cap = kBinCap;
    P.max_rounds = 0xFFFFFFFFu;
    P.has_astar = astar ? 1u : 0u;
    P.precheck = c.precheck == OG_PRECHECK_ON ? 1u : 0u;
    P.prefetch = c.prefetch == OG_PREFETCH_OFF ? 0u : 1u;
    P.spin_ns = c.spin_limit_ns;
    if (c.pull_divisor && c.bucket_update != OG_UPDATE_LAZY) {
      TRY(ensure_transpose(g, st));
      P.pull_div = c.pull_divisor;
      P.toff = g->toff;
      P.tadj = g->tadj;
    }
    if (c.bucket_update == OG_UPDATE_LAZY) {  // marks instead of inserts; no fusion
      const uint32_t words = (g->n + 31) / 32;
      // One mark per (vertex, query) and round; at most 2^28 marks a round (2 GB).
      const uint32_t lz_cap = (uint32_t)std::min<uint64_t>((uint64_t)nq * g->n, 1ull << 28);
      TRY(ws.lzbits.ensure(sizeof(uint32_t) * (size_t)nq * words));
      TRY(ws.lzlist.ensure(sizeof(uint2) * (size_t)lz_cap));
      CK(cudaMemsetAsync(ws.lzbits.p, 0, sizeof(uint32_t) * (size_t)nq * words, st));
      P.lazy = 1u;
      P.T = 0u;
      P.lz_words = words;
      P.lz_bits = ws.lzbits.as<uint32_t>();
      P.lz_list = ws.lzlist.as<uint2>();
      P.lz_cap = lz_cap;
    }

    CK(cudaMemcpyAsync(ws.qd.p, ws.h_qd.p, sizeof(QDesc) * nq, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws.slots.p, ws.h_slots.p, sizeof(uint32_t) * np,
                       cudaMemcpyHostToDevice, st));
    if (attempt == 0) CK(cudaMemsetAsync(ws.qs.p, 0, sizeof(QState) * nq, st));
    CK(cudaMemsetAsync(ws.sync.p, 0, sizeof(Sync), st));
    CK(cudaMemsetAsync(ws.stats.p, 0, sizeof(Stats), st));
    CK(launch_fill(dist_dev, g->n, ws.slots.as<uint32_t>(), np, g->sms, st));
    CK(launch_init(P, ws.slots.as<uint32_t>(), np, st));
    const int bps = c.blocks_per_sm ? std::min<int>((int)c.blocks_per_sm, g->occ) : g->occ;
    CK(cudaEventRecord(ws.e0, st));
    CK(launch_delta(P, g->sms * bps, smem, st));
    CK(cudaEventRecord(ws.e1, st));
    ws.clean_upto = 0;  // this engine leaves entries in the ring: none of it reads "free"
    ws.dirty.clear();
    CK(cudaMemcpyAsync(ws.h_sync.p, ws.sync.p, sizeof(Sync), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ws.h_stats.p, ws.stats.p, sizeof(Stats), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ws.h_qs.p, ws.qs.p, sizeof(QState) * nq, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ws.e0, ws.e1));
    const Stats* hs = ws.h_stats.as<Stats>();
    for (int k = 0; k < 16; ++k) acc->v[k] += hs->v[k];
    acc->v[15] += (unsigned long long)(ms * 1.0e6);  // kernel ns (slot 15)
    const Sync* hy = ws.h_sync.as<Sync>();
    const QState* hq = ws.h_qs.as<QState>();
    ro->err |= hy->err & ~(uint32_t)kErrArena;
    // Fatal errors end the call here; saturation is reported once every chunk has run,
    // and an exhausted arena is regrown below.
    TRY(launch_status(hy->err & kErrFatal, hy->bad_code, hy->bad_val, hy->bad_aux, false));
    pending.clear();
    for (uint32_t i = 0; i < nq; ++i)
      if (hq[i].aborted) pending.push_back(i);
    for (uint32_t i = 0; i < nq; ++i)
      if (!hq[i].aborted && d_out)
        d_out[i] = (qd[i].kind == kPPSP || qd[i].kind == kASTAR) ? hq[i].result : 0u;
    if (pending.empty()) break;
    // Some queries ran out of bucket space: rerun just those with twice the arena.
    if (attempt >= 6) return OG_E_ARENA;
    entries *= 2;
    ro->restarts++;
  }
  return OG_OK;
}

constexpr uint32_t kLocalQueue = 512;  // per-warp FIFO entries (barrier-free engine)

int occupancy_async(og_graph* g, size_t smem, bool ell) {
  if (!g->occ_async_l[ell]) {
    int dev = 0, b = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
    CK(async_occupancy(&b, smem, ell));
    if (b < 1) {
      snprintf(g_cuda_msg, sizeof(g_cuda_msg), "persistent kernel does not fit on an SM");
      return OG_E_CUDA;
    }
    g->occ_async_l[ell] = b;
  }
  g->occ_async = g->occ_async_l[ell];
  return OG_OK;
}

// Makes ring entries [0, need) read "free" before a barrier-free launch: the part never
// used since allocation, and the regions of queries that stopped with entries left.
int clean_ring(Workspace& ws, uint64_t need, cudaStream_t st) {
  if (ws.ring_ptr != ws.ring.p) {
    ws.ring_ptr = ws.ring.p;
    ws.clean_upto = 0;
    ws.dirty.clear();
  }
  for (const auto& r : ws.dirty) {
    const uint64_t lo = r.first, hi = std::min(r.second, ws.clean_upto);
    if (hi > lo)
      CK(cudaMemsetAsync(ws.ring.as<uint2>() + lo, 0xFF, sizeof(uint2) * (hi - lo), st));
  }
  ws.dirty.clear();
  if (need > ws.clean_upto) {
    CK(cudaMemsetAsync(ws.ring.as<uint2>() + ws.clean_upto, 0xFF,
                       sizeof(uint2) * (need - ws.clean_upto), st));
    ws.clean_upto = need;
  }
  return OG_OK;
}

AParams async_params(const og_graph* g, Workspace& ws, uint32_t* dist, uint32_t nq, uint32_t B,
                     uint32_t cap, uint32_t ocap, const og_config& c, bool astar) {
  AParams P{};
  P.off = g->off;
  P.adj = g->adj;
  P.ell = (c.layout == OG_LAYOUT_ELL) ? g->ell : nullptr;
  P.xy = g->xy;
  P.n = g->n;
  P.xy_integral = g->xy_integral ? 1u : 0u;
  P.dist = dist;
  P.qd = ws.qd.as<QDesc>();
  P.aq = ws.aq.as<AQState>();
  P.ring = ws.ring.as<uint2>();
  P.counts = ws.counts.as<uint32_t>();
  P.ovf = ws.ovf.as<uint2>();
  P.sync = ws.sync.as<Sync>();
  P.stats = ws.stats.as<Stats>();
  P.nq = nq;
  P.B = B;
  P.Bmask = B - 1;
  P.cap = cap;
  P.ocap = ocap;
  P.T = c.fusion_threshold == OG_FUSION_OFF ? 0u : c.fusion_threshold;
  P.lq_cap = kLocalQueue;
  P.has_astar = astar ? 1u : 0u;
  P.precheck = c.precheck == OG_PRECHECK_ON ? 1u : 0u;
  P.prefetch = c.prefetch == OG_PREFETCH_OFF ? 0u : 1u;
  P.spin_ns = c.spin_limit_ns;
  P.budget_ns = 0;
  return P;
}

// Barrier-free engine: up to kMaxQ queries in one launch; queries that ran out of bucket
// space rerun with twice the arena.
int run_chunk_async(og_graph* g, Workspace& ws, const QDesc* qd, uint32_t nq,
                    const og_config& c, uint32_t* dist_dev, uint32_t* d_out, Stats* acc,
                    RunOut* ro, cudaStream_t st) {
  const size_t smem = (size_t)kWarps * kLocalQueue * sizeof(uint2);
  const bool ell = c.layout == OG_LAYOUT_ELL && g->ell;
  TRY(occupancy_async(g, smem, ell));
  uint32_t min_delta = 0xFFFFFFFFu;
  bool astar = false;
  for (uint32_t i = 0; i < nq; ++i) {
    min_delta = std::min(min_delta, qd[i].delta);
    astar |= qd[i].kind == kASTAR;
  }
  const uint32_t B = ring_size(g, c, min_delta);
  uint64_t entries = c.arena_entries ? c.arena_entries : default_arena(g, nq);
  TRY(ws.events());
  TRY(ws.h_qd.ensure(sizeof(QDesc) * nq));
  TRY(ws.h_aq.ensure(sizeof(AQState) * nq));
  TRY(ws.h_sync.ensure(sizeof(Sync)));
  TRY(ws.h_stats.ensure(sizeof(Stats)));
  memcpy(ws.h_qd.p, qd, sizeof(QDesc) * nq);
  std::vector<uint32_t> pending(nq);
  for (uint32_t i = 0; i < nq; ++i) pending[i] = i;
  for (int attempt = 0;; ++attempt) {
    const uint64_t cap64 = std::max<uint64_t>(64, entries / 2 / B);
    const uint64_t ocap64 = std::max<uint64_t>(64, entries / 4);
    if (cap64 >= 0xFFFFFFF0ull || ocap64 >= 0xFFFFFFF0ull) return OG_E_ARENA;
    const uint32_t cap = (uint32_t)cap64, ocap = (uint32_t)ocap64;
    const uint32_t np = (uint32_t)pending.size();
    const uint64_t ring_entries = (uint64_t)nq * B * cap;
    TRY(ws.ring.ensure(sizeof(uint2) * ring_entries));
    TRY(ws.counts.ensure(sizeof(uint32_t) * (size_t)nq * B));
    TRY(ws.ovf.ensure(sizeof(uint2) * (size_t)nq * 2 * ocap));
    TRY(ws.aq.ensure(sizeof(AQState) * nq));
    TRY(ws.qd.ensure(sizeof(QDesc) * nq));
    TRY(ws.sync.ensure(sizeof(Sync)));
    TRY(ws.stats.ensure(sizeof(Stats)));
    TRY(ws.slots.ensure(sizeof(uint32_t) * nq));
    TRY(ws.h_slots.ensure(sizeof(uint32_t) * nq));
    memcpy(ws.h_slots.p, pending.data(), sizeof(uint32_t) * np);
    TRY(clean_ring(ws, ring_entries, st));
    AParams P = async_params(g, ws, dist_dev, nq, B, cap, ocap, c, astar);
    CK(cudaMemcpyAsync(ws.qd.p, ws.h_qd.p, sizeof(QDesc) * nq, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws.slots.p, ws.h_slots.p, sizeof(uint32_t) * np,
                       cudaMemcpyHostToDevice, st));
    if (attempt == 0) CK(cudaMemsetAsync(ws.aq.p, 0, sizeof(AQState) * nq, st));
    CK(cudaMemsetAsync(ws.sync.p, 0, sizeof(Sync), st));
    CK(cudaMemsetAsync(ws.stats.p, 0, sizeof(Stats), st));
    CK(launch_fill(dist_dev, g->n, ws.slots.as<uint32_t>(), np, g->sms, st));
    CK(launch_async_init(P, ws.slots.as<uint32_t>(), np, st));
    const int bps = c.blocks_per_sm ? std::min<int>((int)c.blocks_per_sm, g->occ_async)
                                    : g->occ_async;
    CK(cudaEventRecord(ws.e0, st));
    CK(launch_async(P, g->sms * bps, smem, st));
    CK(cudaEventRecord(ws.e1, st));
    CK(cudaMemcpyAsync(ws.h_sync.p, ws.sync.p, sizeof(Sync), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ws.h_stats.p, ws.stats.p, sizeof(Stats), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ws.h_aq.p, ws.aq.p, sizeof(AQState) * nq, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ws.e0, ws.e1));
    const Stats* hs = ws.h_stats.as<Stats>();
    for (int k = 0; k < 16; ++k) acc->v[k] += hs->v[k];
    acc->v[15] += (unsigned long long)(ms * 1.0e6);
    const Sync* hy = ws.h_sync.as<Sync>();
    const AQState* ha = ws.h_aq.as<AQState>();
    ro->err |= hy->err & ~(uint32_t)kErrArena;
    if (hy->err & kErrBounds) {
      snprintf(g_cuda_msg, sizeof(g_cuda_msg), "internal check %u failed (value %u, context %u)",
               hy->bad_code, hy->bad_val, hy->bad_aux);
      return OG_E_INTERNAL;
    }
    const uint64_t per_q = (uint64_t)B * cap;
    for (uint32_t i = 0; i < nq; ++i)
      if (ha[i].dirty || ha[i].mode != kMDone)
        ws.dirty.emplace_back(i * per_q, (i + 1) * per_q);
    if (hy->err & kErrTimeout) {
      int len = snprintf(g_cuda_msg, sizeof(g_cuda_msg), "wait %u gave up;", hy->timeout_at);
      for (uint32_t i = 0; i < nq && len < 400; ++i)
        if (ha[i].mode != kMDone)
          len += snprintf(g_cuda_msg + len, sizeof(g_cuda_msg) - len,
                          " q%u mode %u cur %u work %u claim %u", i, ha[i].mode, ha[i].cur,
                          ha[i].work, (uint32_t)ha[i].word);
      return OG_E_TIMEOUT;
    }
    pending.clear();
    for (uint32_t i = 0; i < nq; ++i) {
      if (ha[i].aborted) {
        pending.push_back(i);
        continue;
      }
      acc->v[kStRounds] += ha[i].advances;
      acc->v[kStRedist] += ha[i].redists;
      if (d_out) d_out[i] = qd[i].kind == kSSSP ? 0u : ha[i].result;
    }
    if (pending.empty()) break;
    if (attempt >= 6) return OG_E_ARENA;
    entries *= 2;
    ro->restarts++;
  }
  return OG_OK;
}

int run_chunk(og_graph* g, Workspace& ws, const QDesc* qd, uint32_t nq, const og_config& c,
              uint32_t* dist_dev, uint32_t* d_out, Stats* acc, RunOut* ro, cudaStream_t st) {
  bool bf = false;
  for (uint32_t i = 0; i < nq; ++i) bf |= qd[i].kind == kBF;
  // Bellman-Ford rounds and the lazy bucket update need the round engine.
  if (c.engine == OG_ENGINE_ASYNC && !bf && c.bucket_update != OG_UPDATE_LAZY)
    return run_chunk_async(g, ws, qd, nq, c, dist_dev, d_out, acc, ro, st);
  return run_chunk_rounds(g, ws, qd, nq, c, dist_dev, d_out, acc, ro, st);
}

void export_stats(const Stats& s, uint64_t restarts, og_stats* out) {
  if (!out) return;
  memset(out, 0, sizeof(*out));
  out->rounds = s.v[kStRounds];
  out->fused_iters = s.v[kStFused];
  out->items = s.v[kStItems];
  out->stale = s.v[kStStale];
  out->relax = s.v[kStRelax];
  out->improved = s.v[kStImproved];
  out->local_inserts = s.v[kStLocal];
  out->global_inserts = s.v[kStGlobal];
  out->overflow_inserts = s.v[kStOvf];
  out->redistributions = s.v[kStRedist];
  out->restarts = restarts;
  out->kernel_ns = s.v[15];
  out->flushes = s.v[kStFlush];
  out->t_frontier_ns = s.v[kStTFrontier];
  out->t_fused_ns = s.v[kStTFused];
  out->t_barrier_ns = s.v[kStTBarrier];
  out->t_hub_ns = s.v[kStTHub];
}

// Device id of user vertex v, and user id of device vertex x (the graph's vertex order).
uint32_t dev_id(const og_graph* g, uint32_t v) { return g->h_dev.empty() ? v : g->h_dev[v]; }
uint32_t user_id(const og_graph* g, uint32_t x) { return g->h_pi.empty() ? x : g->h_pi[x]; }

// Brings nrows per-vertex rows of n words (device memory) from the device order to the
// user's (to_user) or back; a no-op in the user's order.
int perm_rows(og_graph* g, Workspace& ws, uint32_t* rows, uint32_t nrows, bool to_user,
              cudaStream_t st) {
  if (g->nmv == 0 || nrows == 0) return OG_OK;
  // Up to 16 rows at a time, so the staging of the moved entries stays small (the
  // launches of one stream run in order, so the next group reuses it safely).
  constexpr uint32_t kGroup = 16;
  const uint32_t group = std::min(nrows, kGroup);
  TRY(ws.permtmp.ensure(sizeof(uint32_t) * (size_t)g->nmv * group));
  for (uint32_t r0 = 0; r0 < nrows; r0 += group)
    CK(launch_perm_rows(rows + (size_t)r0 * g->n, g->n, std::min(group, nrows - r0), g->mv,
                        g->nmv, to_user, ws.permtmp.as<uint32_t>(), g->sms, st));
  return OG_OK;
}

// Device copy of the coordinates in the device order (the host copy stays in the user's).
int upload_coords(og_graph* g, cudaStream_t st) {
  if (!g->xy || g->h_xy.empty()) return OG_OK;
  std::vector<float> d;
  const float* src = g->h_xy.data();
  if (!g->h_pi.empty()) {
    d.resize(g->h_xy.size());
    for (uint32_t x = 0; x < g->n; ++x) {
      d[2 * (size_t)x] = g->h_xy[2 * (size_t)g->h_pi[x]];
      d[2 * (size_t)x + 1] = g->h_xy[2 * (size_t)g->h_pi[x] + 1];
    }
    src = d.data();
  }
  CK(cudaMemcpyAsync(g->xy, src, sizeof(float) * g->h_xy.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return OG_OK;
}

// The hot-first order of a graph in the user's ids with degrees deg: the K = n / kHotDiv
// vertices of largest degree (ties: the smaller id) take device ids 0, 1, ..., K - 1 in
// that order, and the other vertices below K take the ids the hot vertices left, in
// increasing order on both sides.  pi[x] = user vertex at device id x, dev = its inverse;
// hot_edges = the edges the K vertices hold.
void hot_first(const std::vector<uint32_t>& deg, std::vector<uint32_t>& pi,
               std::vector<uint32_t>& dev, uint64_t* hot_edges) {
  const uint32_t n = (uint32_t)deg.size(), K = n / kHotDiv;
  pi.resize(n);
  dev.resize(n);
  for (uint32_t v = 0; v < n; ++v) pi[v] = v;
  *hot_edges = 0;
  if (K == 0) {
    dev = pi;
    return;
  }
  std::vector<uint32_t> idx(pi);
  auto hotter = [&](uint32_t a, uint32_t b) { return deg[a] != deg[b] ? deg[a] > deg[b] : a < b; };
  std::nth_element(idx.begin(), idx.begin() + (K - 1), idx.end(), hotter);
  std::sort(idx.begin(), idx.begin() + K, hotter);
  std::vector<char> hot(n, 0);
  for (uint32_t i = 0; i < K; ++i) {
    hot[idx[i]] = 1;
    *hot_edges += deg[idx[i]];
  }
  for (uint32_t i = 0; i < K; ++i) pi[i] = idx[i];
  uint32_t c = 0;  // next id below K that is not hot
  for (uint32_t h = K; h < n; ++h) {
    if (!hot[h]) continue;  // pi[h] = h already
    while (hot[c]) ++c;     // as many such ids below K as hot ids at or above it
    pi[h] = c++;
  }
  for (uint32_t x = 0; x < n; ++x) dev[pi[x]] = x;
}

// Puts the graph in the hot-first order (packed) or back in the user's.  The adjacency
// and offsets are rebuilt on the device from the current ones (og_pack_adj_kernel), the
// ELL rows and coordinates follow, and a transpose is dropped (rebuilt when asked for).
// OG_ORDER_AUTO packs only a large skewed graph.  OG_E_BUSY while a server uses the
// graph; on OG_E_OOM the graph is unchanged.
int set_order(og_graph* g, uint32_t order, cudaStream_t st) {
  const uint32_t n = g->n;
  const bool cur = !g->h_pi.empty();
  const bool pack = order != OG_ORDER_USER;
  if (pack == cur) return OG_OK;  // hot-first (of the same graph) or the user's already
  if (order == OG_ORDER_AUTO && n < kHotMinN) return OG_OK;  // too small to pack
  std::vector<uint32_t> off(n + 1);
  CK(cudaMemcpyAsync(off.data(), g->off, sizeof(uint32_t) * (n + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // src_of[x]: current id of the vertex that gets new id x; new_of: current id -> new id.
  std::vector<uint32_t> pi, dev;
  std::vector<uint2> mv;
  const std::vector<uint32_t>* src_of;
  const std::vector<uint32_t>* new_of;
  if (pack) {
    std::vector<uint32_t> deg(n);
    for (uint32_t v = 0; v < n; ++v) deg[v] = off[v + 1] - off[v];
    uint64_t hot_edges = 0;
    hot_first(deg, pi, dev, &hot_edges);
    if (order == OG_ORDER_AUTO && !(n >= kHotMinN && 2 * hot_edges >= g->m)) return OG_OK;
    for (uint32_t x = 0; x < n; ++x)
      if (pi[x] != x) mv.push_back(make_uint2(x, pi[x]));
    if (mv.empty()) return OG_OK;  // the user's order is hot-first already
    src_of = &pi;
    new_of = &dev;
  } else {
    src_of = &g->h_dev;
    new_of = &g->h_pi;
  }
  if (g->servers) return OG_E_BUSY;
  std::vector<uint32_t> offn(n + 1);
  offn[0] = 0;
  for (uint32_t x = 0; x < n; ++x) {
    const uint32_t u = (*src_of)[x];
    offn[x + 1] = offn[x] + (off[u + 1] - off[u]);
  }
  uint32_t *d_off = nullptr, *d_src = nullptr, *d_new = nullptr;
  uint2 *d_adj = nullptr, *d_mv = nullptr;
  auto undo = [&](int code) {
    for (void* p : {(void*)d_off, (void*)d_src, (void*)d_new, (void*)d_adj, (void*)d_mv})
      if (p) cudaFree(p);
    cudaGetLastError();
    return code;
  };
  if (cudaMalloc(&d_off, sizeof(uint32_t) * (n + 1)) != cudaSuccess ||
      cudaMalloc(&d_src, sizeof(uint32_t) * n) != cudaSuccess ||
      cudaMalloc(&d_new, sizeof(uint32_t) * n) != cudaSuccess ||
      cudaMalloc(&d_adj, sizeof(uint2) * (g->m ? g->m : 1)) != cudaSuccess ||
      (pack && cudaMalloc(&d_mv, sizeof(uint2) * mv.size()) != cudaSuccess))
    return undo(OG_E_OOM);
  cudaError_t e = cudaMemcpyAsync(d_off, offn.data(), sizeof(uint32_t) * (n + 1),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_src, src_of->data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_new, new_of->data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && pack)
    e = cudaMemcpyAsync(d_mv, mv.data(), sizeof(uint2) * mv.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_pack_adj(g->off, g->adj, d_off, d_src, d_new, d_adj, n, g->sms, st);
  if (e == cudaSuccess && g->ell) e = launch_ell(d_off, d_adj, g->ell, n, g->sms, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return undo(cuda_fail(e, "vertex order"));
  cudaFree(d_src);
  cudaFree(d_new);
  cudaFree(g->off);
  cudaFree(g->adj);
  g->off = d_off;
  g->adj = d_adj;
  if (g->toff) cudaFree(g->toff);
  if (g->tadj) cudaFree(g->tadj);
  g->toff = nullptr;
  g->tadj = nullptr;
  if (g->mv) cudaFree(g->mv);
  g->mv = pack ? d_mv : nullptr;
  g->nmv = pack ? (uint32_t)mv.size() : 0u;
  if (pack) {
    g->h_pi.swap(pi);
    g->h_dev.swap(dev);
  } else {
    g->h_pi.clear();
    g->h_dev.clear();
  }
  return upload_coords(g, st);
}

int make_desc(const og_graph* g, const og_query& q, const og_config& c, QDesc* d) {
  if (q.src >= g->n) return OG_E_INVALID;
  memset(d, 0, sizeof(*d));
  d->src = dev_id(g, q.src);
  d->dst = kNone;
  switch (q.kind) {
    case OG_Q_SSSP:
      d->kind = kSSSP;
      d->delta = q.delta ? q.delta : c.delta;
      break;
    case OG_Q_WBFS:
      if (g->m && g->min_w == 0) return OG_E_INVALID;  // wBFS needs positive weights
      d->kind = kSSSP;
      d->delta = 1;
      break;
    case OG_Q_PPSP:
    case OG_Q_ASTAR:
      if (q.dst >= g->n) return OG_E_INVALID;
      if (q.kind == OG_Q_ASTAR && !g->xy) return OG_E_INVALID;
      d->kind = q.kind == OG_Q_PPSP ? kPPSP : kASTAR;
      d->dst = dev_id(g, q.dst);
      if (q.kind == OG_Q_ASTAR) {  // host coordinates stay in the user's order
        d->tx = g->h_xy[2 * (size_t)q.dst];
        d->ty = g->h_xy[2 * (size_t)q.dst + 1];
      }
      d->delta = q.delta ? q.delta : c.delta;
      break;
    case OG_Q_BF:
      d->kind = kBF;
      d->delta = 0;  // no buckets by distance: one bucket per round
      return OG_OK;
    default:
      return OG_E_INVALID;
  }
  if (d->delta == 0) return OG_E_INVALID;
  return OG_OK;
}

int run_queries(og_graph* g, const og_query* qv, uint32_t nq, const og_config* ucfg,
                uint32_t* dist_out, uint32_t* d_out, og_stats* stats, cudaStream_t st) {
  if (!g || !qv || nq == 0) return OG_E_INVALID;
  const og_config c = resolve(g, ucfg);
  std::vector<QDesc> qd(nq);
  for (uint32_t i = 0; i < nq; ++i) TRY(make_desc(g, qv[i], c, &qd[i]));
  const bool dev_out = dist_out && is_device_ptr(dist_out);
  Stats acc;
  memset(&acc, 0, sizeof(acc));
  RunOut ro;
  for (uint32_t base = 0; base < nq; base += kMaxQ) {
    const uint32_t k = std::min<uint32_t>(kMaxQ, nq - base);
    uint32_t* ddist;
    if (dev_out) {
      ddist = dist_out + (size_t)base * g->n;
    } else {
      TRY(g->ws.dist.ensure(sizeof(uint32_t) * (size_t)k * g->n));
      ddist = g->ws.dist.as<uint32_t>();
    }
    TRY(run_chunk(g, g->ws, qd.data() + base, k, c, ddist, d_out ? d_out + base : nullptr,
                  &acc, &ro, st));
    if (dist_out) TRY(perm_rows(g, g->ws, ddist, k, true, st));
    if (dist_out && !dev_out) {
      CK(cudaMemcpyAsync(dist_out + (size_t)base * g->n, ddist,
                         sizeof(uint32_t) * (size_t)k * g->n, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  export_stats(acc, ro.restarts, stats);
  return launch_status(ro.err & kErrSat, 0, 0, 0, false);
}

}  // namespace

extern "C" {

int og_version(void) { return 100; }

const char* og_strerror(int code) {
  switch (code) {
    case OG_OK: return "ok";
    case OG_E_INVALID: return "invalid argument";
    case OG_E_OOM: return "out of memory";
    case OG_E_CUDA: return "CUDA runtime error";
    case OG_E_OVERFLOW: return "distance overflow (saturated at 0xFFFFFFFE)";
    case OG_E_TIMEOUT: return "bounded device wait timed out";
    case OG_E_BUSY: return "no free slot";
    case OG_E_ARENA: return "bucket arena exhausted";
    case OG_E_INTERNAL: return "internal consistency check failed";
    default: return "unknown error";
  }
}

const char* og_last_cuda_error(void) { return g_cuda_msg; }

void og_config_default(og_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->fusion_threshold = kDefaultFusion;
  c->hub_degree = kDefaultHub;
  c->spin_limit_ns = kDefaultSpinNs;
}

int og_graph_upload(const uint64_t* offsets, const uint32_t* neighbors, const uint32_t* weights,
                    uint32_t n, uint64_t m, void* stream, og_graph** out) {
  if (!out) return OG_E_INVALID;
  *out = nullptr;
  if (!offsets || n == 0 || n == 0xFFFFFFFFu) return OG_E_INVALID;
  if (m && (!neighbors || !weights)) return OG_E_INVALID;
  if (offsets[0] != 0 || offsets[n] != m || m >= 0xFFFFFFFFull) return OG_E_INVALID;
  for (uint32_t i = 0; i < n; ++i)
    if (offsets[i + 1] < offsets[i]) return OG_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  og_graph* g = new (std::nothrow) og_graph();
  if (!g) return OG_E_OOM;
  g->n = n;
  g->m = m;
  auto fail = [&](int code) {
    og_graph_free(g);
    return code;
  };
  std::vector<uint32_t> off32(n + 1);
  for (uint32_t i = 0; i <= n; ++i) off32[i] = (uint32_t)offsets[i];
  double wsum = 0.0;
  for (uint64_t e = 0; e < m; ++e) wsum += weights[e];
  g->mean_w = m ? wsum / (double)m : 1.0;
  cudaError_t e;
  if ((e = cudaMalloc(&g->off, sizeof(uint32_t) * (n + 1))) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMalloc offsets"));
  if ((e = cudaMalloc(&g->adj, sizeof(uint2) * (m ? m : 1))) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMalloc adjacency"));
  if ((e = cudaMemcpyAsync(g->off, off32.data(), sizeof(uint32_t) * (n + 1),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(cuda_fail(e, "copy offsets"));
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* tmp = nullptr;
  uint32_t* flags = nullptr;
  if (m) {
    if ((e = cudaMalloc(&tmp, sizeof(uint32_t) * 2 * m)) != cudaSuccess)
      return fail(cuda_fail(e, "cudaMalloc staging"));
    if ((e = cudaMalloc(&flags, sizeof(uint32_t) * 4)) != cudaSuccess) {
      cudaFree(tmp);
      return fail(cuda_fail(e, "cudaMalloc flags"));
    }
    const uint32_t init[4] = {0u, 0xFFFFFFFFu, 0u, 0u};
    uint32_t hflags[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(tmp, neighbors, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp + m, weights, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_interleave(tmp, tmp + m, g->adj, m, n, flags, g->sms, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    cudaFree(flags);
    if (e != cudaSuccess) return fail(cuda_fail(e, "upload adjacency"));
    if (hflags[0]) return fail(OG_E_INVALID);  // a neighbor id >= n
    g->min_w = hflags[1];
    g->max_w = hflags[2];
    for (uint32_t i = 0; i < n; ++i)
      g->max_deg = std::max<uint32_t>(g->max_deg, (uint32_t)(offsets[i + 1] - offsets[i]));
    if (g->max_deg <= (uint32_t)kEllWidthHost) {
      // Low-degree graph: also keep one 64-byte row per vertex (no offsets lookup).
      if ((e = cudaMalloc(&g->ell, sizeof(uint4) * 4 * (size_t)n)) != cudaSuccess) {
        g->ell = nullptr;
        cudaGetLastError();
      } else if ((e = launch_ell(g->off, g->adj, g->ell, n, g->sms, st)) != cudaSuccess ||
                 (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        return fail(cuda_fail(e, "build ELL rows"));
      }
    }
  } else {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_fail(e, "upload"));
  }
  og_config_default(&g->cfg);
  g->cfg.fusion_threshold = 0;
  g->cfg.expand_tile = 0;
  g->cfg.spin_limit_ns = 0;
  if (m) {
    // A large power-law graph is packed hot-first; without the memory for the rebuild it
    // stays in the user's order.
    const int rc = set_order(g, OG_ORDER_AUTO, st);
    if (rc != OG_OK && rc != OG_E_OOM) return fail(rc);
  }
  *out = g;
  return OG_OK;
}

int og_graph_set_coords(og_graph* g, const float* xy, void* stream) {
  if (!g || !xy) return OG_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<float> h(2 * (size_t)g->n);
  if (is_device_ptr(xy)) {
    CK(cudaMemcpyAsync(h.data(), xy, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else {
    memcpy(h.data(), xy, sizeof(float) * h.size());
  }
  bool integral = true;
  for (float v : h) {
    if (!std::isfinite(v)) return OG_E_INVALID;
    if (std::fabs(v) >= 16777216.0f || std::floor(v) != v) integral = false;
  }
  if (!g->xy) {
    cudaError_t e = cudaMalloc(&g->xy, sizeof(float2) * g->n);
    if (e != cudaSuccess) {
      g->xy = nullptr;
      return cuda_fail(e, "cudaMalloc coords");
    }
  }
  g->xy_integral = integral;
  g->h_xy.swap(h);
  return upload_coords(g, st);
}

int og_graph_set_order(og_graph* g, uint32_t order, void* stream) {
  if (!g || order > OG_ORDER_USER) return OG_E_INVALID;
  if (!g->m) return OG_OK;
  return set_order(g, order, (cudaStream_t)stream);
}

int og_hot_first_order(const uint32_t* degrees, uint32_t n, uint32_t* device_to_user,
                       uint64_t* hot_edges) {
  if (!degrees || !device_to_user || n == 0) return OG_E_INVALID;
  std::vector<uint32_t> deg(degrees, degrees + n), pi, dev;
  uint64_t he = 0;
  hot_first(deg, pi, dev, &he);
  memcpy(device_to_user, pi.data(), sizeof(uint32_t) * n);
  if (hot_edges) *hot_edges = he;
  return OG_OK;
}

int og_graph_get_order(const og_graph* g, uint32_t* order, uint32_t* moved) {
  if (!g) return OG_E_INVALID;
  if (order) *order = g->h_pi.empty() ? OG_ORDER_USER : OG_ORDER_HOT_FIRST;
  if (moved) *moved = g->nmv;
  return OG_OK;
}

int og_graph_info(const og_graph* g, uint32_t* n, uint64_t* m, uint32_t* min_w,
                  uint32_t* max_w) {
  if (!g) return OG_E_INVALID;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (min_w) *min_w = g->min_w;
  if (max_w) *max_w = g->max_w;
  return OG_OK;
}

int og_graph_set_config(og_graph* g, const og_config* cfg) {
  if (!g || !cfg) return OG_E_INVALID;
  g->cfg = *cfg;
  return OG_OK;
}

int og_graph_get_config(const og_graph* g, og_config* cfg) {
  if (!g || !cfg) return OG_E_INVALID;
  *cfg = resolve(g, nullptr);
  return OG_OK;
}

void og_graph_free(og_graph* g) {
  if (!g) return;
  g->ws.release();
  if (g->off) cudaFree(g->off);
  if (g->adj) cudaFree(g->adj);
  if (g->ell) cudaFree(g->ell);
  if (g->xy) cudaFree(g->xy);
  if (g->toff) cudaFree(g->toff);
  if (g->tadj) cudaFree(g->tadj);
  if (g->mv) cudaFree(g->mv);
  delete g;
}

int og_query_run(og_graph* g, const og_query* q, const og_config* cfg, uint32_t* dist_out,
                 uint32_t* d_out, og_stats* stats, void* stream) {
  if (!g || !q) return OG_E_INVALID;
  return run_queries(g, q, 1, cfg, dist_out, d_out, stats, (cudaStream_t)stream);
}

int og_sssp_delta(og_graph* g, uint32_t src, uint32_t delta, uint32_t* dist_out, void* stream) {
  if (!dist_out) return OG_E_INVALID;
  og_query q{OG_Q_SSSP, src, 0, delta};
  return og_query_run(g, &q, nullptr, dist_out, nullptr, nullptr, stream);
}

int og_wbfs(og_graph* g, uint32_t src, uint32_t* dist_out, void* stream) {
  if (!dist_out) return OG_E_INVALID;
  og_query q{OG_Q_WBFS, src, 0, 1};
  return og_query_run(g, &q, nullptr, dist_out, nullptr, nullptr, stream);
}

int og_sssp_bellman_ford(og_graph* g, uint32_t src, uint32_t* dist_out, og_stats* stats,
                         void* stream) {
  if (!dist_out) return OG_E_INVALID;
  og_query q{OG_Q_BF, src, 0, 0};
  return og_query_run(g, &q, nullptr, dist_out, nullptr, stats, stream);
}

int og_kcore(og_graph* g, uint32_t mode, const og_config* ucfg, uint32_t* core_out,
             og_stats* stats, void* stream) {
  if (!g || !core_out || mode > OG_KCORE_EAGER) return OG_E_INVALID;
  const og_config c = resolve(g, ucfg);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = g->ws;
  const uint32_t n = g->n;
  if (!g->sms) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
  }
  int occ = 0;
  CK(kcore_occupancy(&occ));
  if (occ < 1) return OG_E_CUDA;
  // CTAs per SM: the caller's, else 2 -- peeling rounds are short and barrier-bound, and
  // fewer CTAs reach the grid barrier sooner (R-MAT-24: 56.0 ms at 2, 58.4 ms at 4).  The
  // graph's stored schedule is tuned for Delta-stepping and is not used here.
  const int want = (ucfg && ucfg->blocks_per_sm) ? (int)ucfg->blocks_per_sm : kKcoreBps;
  const int bps = std::max(1, std::min(want, occ));
  const bool dev_out = is_device_ptr(core_out);
  uint32_t* prio = core_out;
  if (!dev_out) {
    TRY(ws.kprio.ensure(sizeof(uint32_t) * (size_t)n));
    prio = ws.kprio.as<uint32_t>();
  }
  // Window buckets: arena_entries vertex ids in all (default 4n, at least 1024 a bucket).
  const uint64_t entries = c.arena_entries ? c.arena_entries : 4ull * n;
  const uint64_t cap64 = std::max<uint64_t>(1024, entries / kKRing);
  if (cap64 >= 0xFFFFFFF0ull) return OG_E_INVALID;
  TRY(ws.kcnt.ensure(sizeof(uint32_t) * (size_t)n));
  TRY(ws.ktouched.ensure(2 * sizeof(uint32_t) * (size_t)n));
  TRY(ws.klist.ensure(2 * sizeof(uint32_t) * (size_t)n));
  TRY(ws.kring.ensure(sizeof(uint32_t) * (size_t)kKRing * cap64));
  TRY(ws.kcounts.ensure(sizeof(uint32_t) * kKRing));
  TRY(ws.klossy.ensure(sizeof(uint32_t) * kKRing));
  TRY(ws.kstate.ensure(sizeof(KState)));
  TRY(ws.sync.ensure(sizeof(Sync)));
  TRY(ws.stats.ensure(sizeof(Stats)));
  TRY(ws.h_sync.ensure(sizeof(Sync)));
  TRY(ws.h_stats.ensure(sizeof(Stats)));
  TRY(ws.h_kstate.ensure(sizeof(KState)));
  TRY(ws.events());
  KParams P{};
  P.off = g->off;
  P.adj = g->adj;
  P.n = n;
  P.prio = prio;
  P.cnt = ws.kcnt.as<uint32_t>();
  P.touched[0] = ws.ktouched.as<uint32_t>();
  P.touched[1] = P.touched[0] + n;
  P.list[0] = ws.klist.as<uint32_t>();
  P.list[1] = P.list[0] + n;
  P.ring = ws.kring.as<uint32_t>();
  P.counts = ws.kcounts.as<uint32_t>();
  P.lossy = ws.klossy.as<uint32_t>();
  P.sync = ws.sync.as<Sync>();
  P.ks = ws.kstate.as<KState>();
  P.stats = ws.stats.as<Stats>();
  // Hubs (out-degree >= hub_degree) are split over every warp after the round's peel.
  // Unset by the caller, the threshold is lower than for Delta-stepping, and the graph's
  // stored schedule (tuned for Delta-stepping) is not used: a peeling round has one
  // frontier and no fused levels, so moving its long adjacency lists to the balanced hub
  // pass costs little (R-MAT-24, lazy: 60.2 ms at 4096, 49.4 ms at 256).
  const uint32_t hub_min = (ucfg && ucfg->hub_degree) ? ucfg->hub_degree : kKcoreHub;
  const uint32_t hub_cap = g->max_deg >= hub_min ? kHubSlots : 0u;
  if (hub_cap) {
    TRY(ws.big.ensure(sizeof(BigItem) * hub_cap));
    TRY(ws.bmap.ensure(sizeof(uint32_t) * kHubChunks));
  }
  P.hub = hub_cap ? ws.big.as<BigItem>() : nullptr;
  P.hub_map = hub_cap ? ws.bmap.as<uint32_t>() : nullptr;
  P.hub_cap = hub_cap;
  P.map_cap = hub_cap ? kHubChunks : 0u;
  P.hub_min = hub_min;
  P.cap = (uint32_t)cap64;
  P.eager = mode == OG_KCORE_EAGER ? 1u : 0u;
  P.tile = std::max<uint32_t>(kBlock, (c.expand_tile + kBlock - 1) / kBlock * kBlock);
  P.spin_ns = c.spin_limit_ns;
  CK(cudaMemsetAsync(P.cnt, 0, sizeof(uint32_t) * (size_t)n, st));
  CK(cudaMemsetAsync(P.counts, 0, sizeof(uint32_t) * kKRing, st));
  CK(cudaMemsetAsync(P.lossy, 0, sizeof(uint32_t) * kKRing, st));
  CK(cudaMemsetAsync(P.ks, 0, sizeof(KState), st));
  CK(cudaMemsetAsync(P.sync, 0, sizeof(Sync), st));
  CK(cudaMemsetAsync(P.stats, 0, sizeof(Stats), st));
  CK(launch_kcore_init(g->off, prio, n, g->sms, st));
  CK(cudaEventRecord(ws.e0, st));
  CK(launch_kcore(P, g->sms * bps, st));
  CK(cudaEventRecord(ws.e1, st));
  CK(cudaMemcpyAsync(ws.h_sync.p, P.sync, sizeof(Sync), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ws.h_stats.p, P.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ws.h_kstate.p, P.ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
  TRY(perm_rows(g, ws, prio, 1, true, st));
  if (!dev_out)
    CK(cudaMemcpyAsync(core_out, prio, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ws.e0, ws.e1));
  const Sync* hy = ws.h_sync.as<Sync>();
  const KState* hk = ws.h_kstate.as<KState>();
  Stats acc = *ws.h_stats.as<Stats>();
  acc.v[15] = (unsigned long long)(ms * 1.0e6);
  acc.v[kStFused] = hk->levels;
  acc.v[kStRedist] = hk->refills;
  acc.v[kStFlush] = hk->scans;
  export_stats(acc, 0, stats);
  if (hy->err & kErrBounds) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "check %u failed: value %u, context %u",
             hy->bad_code, hy->bad_val, hy->bad_aux);
    return OG_E_INTERNAL;
  }
  if (hy->err & kErrTimeout) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "grid barrier wait gave up");
    return OG_E_TIMEOUT;
  }
  return OG_OK;
}

int og_setcover(og_graph* g, uint32_t eps_ppm, const uint32_t* priority, const og_config* ucfg,
                uint32_t* step_out, og_stats* stats, void* stream) {
  if (!g || !step_out || eps_ppm > 1000000u) return OG_E_INVALID;
  if (g->max_deg > kScLenMask || g->m >= (1ull << 32)) return OG_E_INVALID;
  const og_config c = resolve(g, ucfg);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = g->ws;
  const uint32_t n = g->n;
  const uint64_t m = g->m;
  if (!g->sms) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
  }
  int occ = 0;
  CK(setcover_occupancy(&occ));
  if (occ < 1) return OG_E_CUDA;
  // CTAs per SM: the caller's, else 4 -- a step's phases are short, and more resident
  // warps hide more of their dependent gathers (R-MAT-24: 106.1 ms at 1, 82.5 ms at 2,
  // 75.0 ms at 4).
  const int want = (ucfg && ucfg->blocks_per_sm) ? (int)ucfg->blocks_per_sm : kSetcoverBps;
  const int bps = std::max(1, std::min(want, occ));
  // The bucket ladder t_0 = 1, t_(j+1) = t_j + max(1, floor(t_j * eps)) until it passes
  // the largest set, and the received count a set of bucket j needs to join,
  // ceil(t_j / (1 + eps)), both in integers.
  std::vector<uint32_t> lad(1, 1u);
  while (lad.back() <= g->max_deg) {
    const uint64_t t = lad.back();
    const uint64_t inc = std::max<uint64_t>(1, t * eps_ppm / 1000000ull);
    lad.push_back((uint32_t)(t + inc));
    if (lad.size() > (size_t)kScMaxBuckets + 1) return OG_E_INVALID;
  }
  const uint32_t nb = (uint32_t)lad.size() - 1u;
  for (uint32_t j = 0; j < nb; ++j)
    lad.push_back((uint32_t)(((uint64_t)lad[j] * 1000000ull + 1000000ull + eps_ppm - 1) /
                             (1000000ull + eps_ppm)));
  const uint32_t nbands = (nb + kScBand - 1) / kScBand;
  uint32_t hub = (ucfg && ucfg->hub_degree) ? ucfg->hub_degree : kSetcoverHub;
  hub = std::min(std::max(hub, kScMinHub), kScMaxHub);
  const uint32_t lg_cap = (uint32_t)std::min<uint64_t>(n, m / hub + 1);
  // band lists: each set enters each band at most once, sum (first band + 1) <= n + m/16
  const uint64_t bl_entries = 2ull * ((uint64_t)n + m / kScBand + nbands + 1);
  const bool dev_out = is_device_ptr(step_out);
  // In a packed vertex order the priorities are staged in the workspace and permuted
  // there; the caller's buffer is never written.
  const bool packed = g->nmv != 0;
  const bool dev_pri = priority && is_device_ptr(priority) && !packed;
  TRY(ws.sclad.ensure(sizeof(uint32_t) * lad.size()));
  TRY(ws.sclen.ensure(sizeof(uint32_t) * (size_t)n));
  TRY(ws.scpk.ensure(2 * sizeof(uint32_t) * (size_t)std::max<uint64_t>(m, 1)));
  TRY(ws.sccov.ensure((size_t)n));
  TRY(ws.scclaim.ensure(sizeof(unsigned long long) * (size_t)n));
  TRY(ws.scseen.ensure(sizeof(uint32_t) * (size_t)((n + 31) / 32)));
  TRY(ws.scmeta.ensure(5 * sizeof(uint32_t) * (size_t)std::max(nbands, 1u)));
  TRY(ws.scbase.ensure(sizeof(unsigned long long) * (size_t)std::max(nbands, 1u)));
  TRY(ws.scbl.ensure(sizeof(unsigned long long) * (size_t)bl_entries));
  TRY(ws.scsm.ensure(8 * sizeof(uint32_t) * (size_t)n));
  TRY(ws.sclg.ensure(10 * sizeof(uint32_t) * (size_t)lg_cap));
  TRY(ws.scstate.ensure(sizeof(ScState)));
  if (!dev_pri) TRY(ws.scpri.ensure(sizeof(uint32_t) * (size_t)n));
  if (!dev_out) TRY(ws.scout.ensure(sizeof(uint32_t) * (size_t)n));
  TRY(ws.sync.ensure(sizeof(Sync)));
  TRY(ws.stats.ensure(sizeof(Stats)));
  TRY(ws.h_sync.ensure(sizeof(Sync)));
  TRY(ws.h_stats.ensure(sizeof(Stats)));
  TRY(ws.h_kstate.ensure(sizeof(ScState)));
  TRY(ws.events());
  ScParams P{};
  P.off = g->off;
  P.adj = g->adj;
  P.n = n;
  P.pri = dev_pri ? priority : ws.scpri.as<uint32_t>();
  P.step_out = dev_out ? step_out : ws.scout.as<uint32_t>();
  P.len = ws.sclen.as<uint32_t>();
  P.pk[0] = ws.scpk.as<uint32_t>();
  P.pk[1] = P.pk[0] + std::max<uint64_t>(m, 1);
  P.cov = ws.sccov.as<uint8_t>();
  P.claim = ws.scclaim.as<unsigned long long>();
  P.t = ws.sclad.as<uint32_t>();
  P.tau = P.t + nb + 1;
  P.nb = nb;
  P.nbands = nbands;
  P.bl = ws.scbl.as<unsigned long long>();
  uint32_t* meta = ws.scmeta.as<uint32_t>();
  const uint32_t nbm = std::max(nbands, 1u);
  P.hist = meta;
  P.bcap = meta + nbm;
  P.bcnt = meta + 2 * nbm;
  P.bsel = meta + 3 * nbm;
  P.bmax = meta + 4 * nbm;
  P.bbase = ws.scbase.as<unsigned long long>();
  P.bl_entries = bl_entries;
  P.seen = ws.scseen.as<uint32_t>();
  uint32_t* sm = ws.scsm.as<uint32_t>();
  uint32_t* lg = ws.sclg.as<uint32_t>();
  for (int q = 0; q < 2; ++q) {
    uint32_t* a = sm + (size_t)q * 4 * n;
    P.sm[q] = ScList{a, a + n, a + 2 * (size_t)n, a + 3 * (size_t)n, nullptr};
    uint32_t* b = lg + (size_t)q * 5 * lg_cap;
    P.lg[q] = ScList{b, b + lg_cap, b + 2 * (size_t)lg_cap, b + 3 * (size_t)lg_cap,
                     b + 4 * (size_t)lg_cap};
  }
  P.lg_cap = lg_cap;
  P.hub = hub;
  P.sync = ws.sync.as<Sync>();
  P.ss = ws.scstate.as<ScState>();
  P.stats = ws.stats.as<Stats>();
  P.spin_ns = c.spin_limit_ns;
  CK(cudaMemcpyAsync(ws.sclad.p, lad.data(), sizeof(uint32_t) * lad.size(),
                     cudaMemcpyHostToDevice, st));
  if (priority && !dev_pri)
    CK(cudaMemcpyAsync(ws.scpri.p, priority, sizeof(uint32_t) * (size_t)n,
                       cudaMemcpyDefault, st));
  if (packed && !priority)  // the identity in user ids is pi in device ids
    CK(cudaMemcpyAsync(ws.scpri.p, g->h_pi.data(), sizeof(uint32_t) * (size_t)n,
                       cudaMemcpyHostToDevice, st));
  else if (packed)
    TRY(perm_rows(g, ws, ws.scpri.as<uint32_t>(), 1, false, st));
  CK(cudaMemsetAsync(meta, 0, 5 * sizeof(uint32_t) * (size_t)nbm, st));
  CK(cudaMemsetAsync(P.seen, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32), st));
  CK(cudaMemsetAsync(P.ss, 0, sizeof(ScState), st));
  CK(cudaMemsetAsync(P.sync, 0, sizeof(Sync), st));
  CK(cudaMemsetAsync(P.stats, 0, sizeof(Stats), st));
  CK(cudaEventRecord(ws.e0, st));
  CK(launch_setcover_prep(P, (priority || packed) ? nullptr : ws.scpri.as<uint32_t>(), g->sms,
                          st));
  CK(launch_setcover(P, g->sms * bps, st));
  CK(cudaEventRecord(ws.e1, st));
  CK(cudaMemcpyAsync(ws.h_sync.p, P.sync, sizeof(Sync), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ws.h_stats.p, P.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ws.h_kstate.p, P.ss, sizeof(ScState), cudaMemcpyDeviceToHost, st));
  TRY(perm_rows(g, ws, P.step_out, 1, true, st));
  if (!dev_out)
    CK(cudaMemcpyAsync(step_out, P.step_out, sizeof(uint32_t) * (size_t)n,
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ws.e0, ws.e1));
  const Sync* hy = ws.h_sync.as<Sync>();
  const ScState* hs = ws.h_kstate.as<ScState>();
  Stats acc = *ws.h_stats.as<Stats>();
  acc.v[15] = (unsigned long long)(ms * 1.0e6);
  acc.v[kStFused] = hs->gathers;
  export_stats(acc, 0, stats);
  if (hy->err & kErrBounds) {
    if (hy->bad_code == kScBadPriority) {
      snprintf(g_cuda_msg, sizeof(g_cuda_msg),
               "priority of set %u (%u) is out of range or repeated",
               hy->bad_val < n ? user_id(g, hy->bad_val) : hy->bad_val, hy->bad_aux);
      return OG_E_INVALID;
    }
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "check %u failed: value %u, context %u",
             hy->bad_code, hy->bad_val, hy->bad_aux);
    return OG_E_INTERNAL;
  }
  if (hy->err & kErrTimeout) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "grid barrier wait gave up");
    return OG_E_TIMEOUT;
  }
  return OG_OK;
}

int og_ppsp(og_graph* g, uint32_t src, uint32_t dst, uint32_t delta, uint32_t* d_out,
            void* stream) {
  if (!d_out) return OG_E_INVALID;
  og_query q{OG_Q_PPSP, src, dst, delta};
  return og_query_run(g, &q, nullptr, nullptr, d_out, nullptr, stream);
}

int og_astar(og_graph* g, uint32_t src, uint32_t dst, const float* coords, uint32_t delta,
             uint32_t* d_out, void* stream) {
  if (!g || !d_out) return OG_E_INVALID;
  if (coords) TRY(og_graph_set_coords(g, coords, stream));
  og_query q{OG_Q_ASTAR, src, dst, delta};
  return og_query_run(g, &q, nullptr, nullptr, d_out, nullptr, stream);
}

int og_batch_run(og_graph* g, const og_query* q, uint32_t nq, const og_config* cfg,
                 uint32_t* dist_out, uint32_t* d_out, og_stats* stats, void* stream) {
  return run_queries(g, q, nq, cfg, dist_out, d_out, stats, (cudaStream_t)stream);
}

// ---- serving ------------------------------------------------------------------------------

int og_server_create(og_graph* g, uint32_t max_slots, const og_config* cfg, void* stream,
                     og_server** out) {
  if (!g || !out) return OG_E_INVALID;
  *out = nullptr;
  og_server* s = new (std::nothrow) og_server();
  if (!s) return OG_E_OOM;
  s->g = g;
  s->cfg = resolve(g, cfg);
  // The server's barrier-free engine runs CSR unless its caller asks for ELL rows (a
  // layout tuned for the graph's round engine does not carry over).
  s->cfg.layout = (cfg && cfg->layout == OG_LAYOUT_ELL && g->ell) ? OG_LAYOUT_ELL : OG_LAYOUT_CSR;
  if (s->cfg.bucket_update == OG_UPDATE_LAZY) {  // the server runs the barrier-free engine
    delete s;
    return OG_E_INVALID;
  }
  s->stream = (cudaStream_t)stream;
  const uint32_t B = ring_size(g, s->cfg, s->cfg.delta);
  const uint64_t entries = s->cfg.arena_entries
                               ? s->cfg.arena_entries
                               : std::max<uint64_t>((uint64_t)g->n / 2, 1ull << 20);
  const uint64_t per_slot = sizeof(uint32_t) * (uint64_t)g->n + sizeof(uint2) * entries +
                            sizeof(AQState) + sizeof(QDesc) + 64;
  uint32_t slots = max_slots;
  if (!slots) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return OG_E_CUDA;
    }
    slots = (uint32_t)std::min<uint64_t>(kMaxQ, (uint64_t)(fr / 2) / per_slot);
    if (!slots) {
      delete s;
      return OG_E_OOM;
    }
  }
  if (slots > (uint32_t)kMaxQ) slots = kMaxQ;
  s->slots = slots;
  s->B = B;
  s->cap = (uint32_t)std::max<uint64_t>(64, entries / 2 / B);
  s->ocap = (uint32_t)std::max<uint64_t>(64, entries / 4);
  Workspace& ws = s->ws;
  int r = OG_OK;
  const uint32_t tbw = touch_words(g->n);
  if (r == OG_OK) r = ws.dist.ensure(sizeof(uint32_t) * (size_t)slots * g->n);
  if (r == OG_OK) r = ws.stouched.ensure(sizeof(uint32_t) * (size_t)slots * tbw);
  if (r == OG_OK) r = ws.ring.ensure(sizeof(uint2) * (size_t)slots * B * s->cap);
  if (r == OG_OK) r = ws.counts.ensure(sizeof(uint32_t) * (size_t)slots * B);
  if (r == OG_OK) r = ws.ovf.ensure(sizeof(uint2) * (size_t)slots * 2 * s->ocap);
  if (r == OG_OK) r = ws.aq.ensure(sizeof(AQState) * slots);
  if (r == OG_OK) r = ws.qd.ensure(sizeof(QDesc) * slots);
  if (r == OG_OK) r = ws.sync.ensure(sizeof(Sync));
  if (r == OG_OK) r = ws.stats.ensure(sizeof(Stats));
  if (r == OG_OK) r = ws.slots.ensure(sizeof(uint32_t) * slots);
  if (r == OG_OK) r = ws.h_qd.ensure(sizeof(QDesc) * slots);
  if (r == OG_OK) r = ws.h_aq.ensure(sizeof(AQState) * slots);
  if (r == OG_OK) r = ws.h_sync.ensure(sizeof(Sync));
  if (r == OG_OK) r = ws.h_slots.ensure(sizeof(uint32_t) * slots);
  if (r == OG_OK) r = ws.events();
  // A slot without a query must offer nothing to claim: all-ones makes its claim word
  // closed.  The bucket counters start at zero.  (Device memory comes back uncleared
  // from an earlier server; zeroed states read as an open word over stale counters, and
  // idle warps then waited for entries that were never written.)
  if (r == OG_OK &&
      cudaMemsetAsync(ws.aq.p, 0xFF, sizeof(AQState) * slots, s->stream) != cudaSuccess)
    r = OG_E_CUDA;
  if (r == OG_OK && cudaMemsetAsync(ws.counts.p, 0, sizeof(uint32_t) * (size_t)slots * B,
                                    s->stream) != cudaSuccess)
    r = OG_E_CUDA;
  if (r == OG_OK && cudaMemsetAsync(ws.sync.p, 0, sizeof(Sync), s->stream) != cudaSuccess)
    r = OG_E_CUDA;
  // Every slot's distance row starts unreachable, once: afterwards a slot is reset only
  // in the blocks its last query reached (touched bitmap), when a new query is admitted.
  if (r == OG_OK && cudaMemsetAsync(ws.stouched.p, 0, sizeof(uint32_t) * (size_t)slots * tbw,
                                    s->stream) != cudaSuccess)
    r = OG_E_CUDA;
  if (r == OG_OK) {
    int dev = 0;
    if (!g->sms && (cudaGetDevice(&dev) != cudaSuccess ||
                    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) !=
                        cudaSuccess))
      r = OG_E_CUDA;
    else if (launch_fill(ws.dist.as<uint32_t>(), g->n, nullptr, slots, g->sms, s->stream) !=
             cudaSuccess)
      r = OG_E_CUDA;
  }
  if (r == OG_OK) r = clean_ring(ws, (uint64_t)slots * B * s->cap, s->stream);
  if (r == OG_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) r = OG_E_CUDA;
  if (r != OG_OK) {
    og_server_free(s);
    return r;
  }
  s->hq.assign(slots, QDesc{});
  s->tags.assign(slots, 0);
  s->state.assign(slots, 0);
  s->results.assign(slots, kInf);
  for (uint32_t i = slots; i > 0; --i) s->free_list.push_back(i - 1);
  s->g->servers++;
  *out = s;
  return OG_OK;
}

int og_server_submit(og_server* s, const og_query* q, uint64_t tag) {
  if (!s || !q) return OG_E_INVALID;
  if (s->free_list.empty()) return OG_E_BUSY;
  if (q->kind == OG_Q_BF) return OG_E_INVALID;  // the server runs the barrier-free engine
  QDesc d;
  TRY(make_desc(s->g, *q, s->cfg, &d));
  const uint32_t slot = s->free_list.back();
  s->free_list.pop_back();
  s->hq[slot] = d;
  s->tags[slot] = tag;
  s->state[slot] = 1;
  s->pending.push_back(slot);
  return OG_OK;
}

// One launch of the barrier-free engine over all slots, bounded by budget_us.
int og_server_step(og_server* s, uint32_t budget_us, uint32_t* n_active) {
  if (!s) return OG_E_INVALID;
  og_graph* g = s->g;
  Workspace& ws = s->ws;
  cudaStream_t st = s->stream;
  const size_t smem = (size_t)kWarps * kLocalQueue * sizeof(uint2);
  TRY(occupancy_async(g, smem, s->cfg.layout == OG_LAYOUT_ELL && g->ell));
  bool astar = false;
  uint32_t running = 0;
  for (uint32_t i = 0; i < s->slots; ++i) {
    if (s->state[i] == 1 || s->state[i] == 2) {
      ++running;
      astar |= s->hq[i].kind == kASTAR;
    }
  }
  if (n_active) *n_active = running;
  if (!running) return OG_OK;
  TRY(clean_ring(ws, (uint64_t)s->slots * s->B * s->cap, st));
  AParams P = async_params(g, ws, ws.dist.as<uint32_t>(), s->slots, s->B, s->cap, s->ocap,
                           s->cfg, astar);
  P.budget_ns = (unsigned long long)budget_us * 1000ull;
  P.touched = ws.stouched.as<uint32_t>();
  P.tb_words = touch_words(g->n);
  const uint32_t np = (uint32_t)s->pending.size();
  if (np) {
    QDesc* hqd = ws.h_qd.as<QDesc>();
    memcpy(hqd, s->hq.data(), sizeof(QDesc) * s->slots);
    memcpy(ws.h_slots.p, s->pending.data(), sizeof(uint32_t) * np);
    CK(cudaMemcpyAsync(ws.qd.p, hqd, sizeof(QDesc) * s->slots, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws.slots.p, ws.h_slots.p, sizeof(uint32_t) * np,
                       cudaMemcpyHostToDevice, st));
    // Admitted slots: back to unreachable where the previous query reached (O(touched),
    // not O(n)), then started.
    CK(launch_touch_reset(P.dist, g->n, P.touched, P.tb_words, ws.slots.as<uint32_t>(), np,
                          g->sms, st));
    CK(launch_async_init(P, ws.slots.as<uint32_t>(), np, st));
    for (uint32_t slot : s->pending) s->state[slot] = 2;
    s->pending.clear();
  }
  CK(cudaMemsetAsync(&ws.sync.as<Sync>()->err, 0, sizeof(uint32_t), st));
  CK(cudaMemsetAsync(ws.stats.p, 0, sizeof(Stats), st));  // counters and wait diagnostics
  const int bps = s->cfg.blocks_per_sm ? std::min<int>((int)s->cfg.blocks_per_sm, g->occ_async)
                                       : g->occ_async;
  CK(launch_async(P, g->sms * bps, smem, st));
  CK(cudaMemcpyAsync(ws.h_sync.p, ws.sync.p, sizeof(Sync), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ws.h_aq.p, ws.aq.p, sizeof(AQState) * s->slots, cudaMemcpyDeviceToHost,
                     st));
  CK(cudaStreamSynchronize(st));
  const Sync* hy = ws.h_sync.as<Sync>();
  if (hy->err & kErrBounds) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "internal check %u failed (value %u, context %u)",
             hy->bad_code, hy->bad_val, hy->bad_aux);
    return OG_E_INTERNAL;
  }
  if (hy->err & kErrTimeout) {
    if (hy->timeout_at == 2u) {
      Stats hs;
      CK(cudaMemcpy(&hs, ws.stats.p, sizeof(Stats), cudaMemcpyDeviceToHost));
      const unsigned long long a = hs.v[kStTFrontier], b = hs.v[kStTFused],
                               w = hs.v[kStTBarrier], c = hs.v[kStTHub];
      snprintf(g_cuda_msg, sizeof(g_cuda_msg),
               "entry hand-off wait gave up: query %u position %u, bucket %u with %u "
               "appends, claim word epoch %u position %u, query cursor %u mode %u count %u",
               (uint32_t)(a >> 32), (uint32_t)a, (uint32_t)(b >> 32), (uint32_t)b,
               (uint32_t)(w >> 32), (uint32_t)w, (uint32_t)(c >> 32),
               (uint32_t)((c >> 28) & 0xFu), (uint32_t)(c & 0x0FFFFFFFu));
    } else {
      snprintf(g_cuda_msg, sizeof(g_cuda_msg), "idle wait gave up (no progress)");
    }
    return OG_E_TIMEOUT;
  }
  const AQState* ha = ws.h_aq.as<AQState>();
  const uint64_t per_q = (uint64_t)s->B * s->cap;
  running = 0;
  for (uint32_t i = 0; i < s->slots; ++i) {
    if (s->state[i] != 2) continue;
    if (ha[i].mode != kMDone) {
      ++running;
      continue;
    }
    if (ha[i].dirty) ws.dirty.emplace_back(i * per_q, (i + 1) * per_q);
    if (ha[i].aborted) {
      // Arena too small for this query: answer it alone with a growing arena.
      og_query q{s->hq[i].kind == kASTAR ? (uint32_t)OG_Q_ASTAR
                 : s->hq[i].kind == kPPSP ? (uint32_t)OG_Q_PPSP : (uint32_t)OG_Q_SSSP,
                 s->hq[i].src, s->hq[i].dst, s->hq[i].delta};
      uint32_t d = kInf;
      TRY(run_queries(g, &q, 1, &s->cfg, nullptr, &d, nullptr, st));
      s->results[i] = d;
    } else {
      s->results[i] = s->hq[i].kind == kSSSP ? 0u : ha[i].result;
    }
    s->state[i] = 3;
    s->done.push_back(i);
  }
  if (n_active) *n_active = running + (uint32_t)s->pending.size();
  if (hy->err & kErrSat) return OG_E_OVERFLOW;
  return OG_OK;
}

int og_server_poll(og_server* s, uint64_t* tags, uint32_t* d_out, uint32_t cap,
                   uint32_t* n_done) {
  if (!s || !n_done) return OG_E_INVALID;
  uint32_t k = 0;
  while (k < cap && !s->done.empty()) {
    const uint32_t slot = s->done.front();
    s->done.pop_front();
    if (tags) tags[k] = s->tags[slot];
    if (d_out) d_out[k] = s->results[slot];
    s->state[slot] = 0;
    s->free_list.push_back(slot);
    ++k;
  }
  *n_done = k;
  return OG_OK;
}

int og_server_slots(const og_server* s, uint32_t* max_slots, uint32_t* n_free) {
  if (!s) return OG_E_INVALID;
  if (max_slots) *max_slots = s->slots;
  if (n_free) *n_free = (uint32_t)s->free_list.size();
  return OG_OK;
}

void og_server_free(og_server* s) {
  if (!s) return;
  s->ws.release();
  if (s->g && s->g->servers) s->g->servers--;
  delete s;
}

// ---- autotuning ---------------------------------------------------------------------------

namespace {

// Coordinate search over the schedule, timing the queries qs in one launch per candidate.
int autotune_queries(og_graph* g, const std::vector<og_query>& qs, uint32_t delta_lo,
                     uint32_t delta_hi, og_config* out) {
  const uint32_t nsample = (uint32_t)qs.size();
  bool all_wbfs = true;
  for (const og_query& q : qs) all_wbfs &= q.kind == OG_Q_WBFS;
  og_config base = resolve(g, nullptr);
  base.engine = OG_ENGINE_ROUNDS;
  // One candidate: a warm-up run, then the best device time of two more runs (one run
  // alone is noisy enough to prefer a slower schedule).  A candidate that fails (e.g. a
  // wait limit reached by a pathological schedule) is skipped.
  auto measure = [&](const og_config& c, double* ns) -> bool {
    og_stats st;
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      if (run_queries(g, qs.data(), nsample, &c, nullptr, nullptr, &st, nullptr) != OG_OK)
        return false;
      if (rep > 0) best = std::min(best, (double)st.kernel_ns);
    }
    *ns = best;
    return true;
  };
  og_config best = base;
  double best_ns = 1e300;
  if (!measure(best, &best_ns)) return OG_E_CUDA;
  auto consider = [&](const og_config& c) {
    double ns;
    if (measure(c, &ns) && ns < best_ns) {
      best_ns = ns;
      best = c;
    }
  };
  // Delta (Section 6.2: the best coarsening factor depends on the graph), with fusion on.
  if (!all_wbfs) {
    if (!delta_lo) delta_lo = std::max(1u, default_delta(g) / 64);
    if (!delta_hi) delta_hi = std::max(delta_lo, default_delta(g) * 8);
    const og_config anchor = best;
    for (uint64_t d = pow2_ceil(delta_lo); d <= delta_hi; d *= 2) {
      // Delta and fusion interact (a narrow bucket leaves little to fuse), so each Delta
      // is timed with the default threshold and with fusion off.
      for (uint32_t f : {anchor.fusion_threshold, OG_FUSION_OFF}) {
        og_config c = anchor;
        c.delta = (uint32_t)d;
        c.fusion_threshold = f;
        consider(c);
      }
    }
  }
  // Fusion threshold (Section 5.2's scheduling function for it), frontier tile, CTAs/SM.
  for (uint32_t f : {OG_FUSION_OFF, 256u, 1024u, 2048u, 0xFFFFFFFFu}) {
    og_config c = best;
    c.fusion_threshold = f;
    consider(c);
  }
  for (uint32_t pc : {OG_PRECHECK_ON, OG_PRECHECK_OFF}) {
    og_config c = best;
    c.precheck = pc;
    consider(c);
  }
  if (g->ell) {
    for (uint32_t lay : {OG_LAYOUT_CSR, OG_LAYOUT_ELL}) {
      og_config c = best;
      c.layout = lay;
      consider(c);
    }
  }
  for (uint32_t pf : {OG_PREFETCH_ON, OG_PREFETCH_OFF}) {
    og_config c = best;
    c.prefetch = pf;
    consider(c);
  }
  auto sweep_tile = [&]() {
    for (uint32_t t : {32u, 64u, 128u, 256u, 512u}) {
      og_config c = best;
      c.expand_tile = t;
      consider(c);
    }
  };
  auto sweep_hub = [&]() {
    if (g->max_deg < 1024) return;  // skewed degrees: where hubs go to the grid-wide pass
    for (uint32_t h : {1024u, 4096u, 32768u, 0xFFFFFFFFu}) {
      og_config c = best;
      c.hub_degree = h;
      consider(c);
    }
  };
  // The frontier tile and the hub threshold interact (hubs leave the tiles' edge lists),
  // so they are swept twice: a tile picked under the default threshold can lose once the
  // threshold moves (R-MAT-24 SSSP: tile 128 then hub 1024, 125.7 ms; tile 256 with hub
  // 1024, 117.9 ms).
  sweep_tile();
  sweep_hub();
  sweep_tile();
  sweep_hub();
  for (uint32_t b = 1; b <= (uint32_t)std::max(1, g->occ); ++b) {
    og_config c = best;
    c.blocks_per_sm = b;
    consider(c);
  }
  // The barrier-free engine with warp-sized local buckets.
  for (uint32_t f : {48u, 64u, 128u}) {
    og_config c = best;
    c.engine = OG_ENGINE_ASYNC;
    c.fusion_threshold = f;
    c.blocks_per_sm = 0;
    consider(c);
  }
  // Return every launch field explicitly: a 0 would later mean "the graph's default",
  // which another tuning call may have changed (a batch then ran with the CTA count
  // tuned for a single query).
  if (!best.blocks_per_sm) {
    const bool ell = g->ell && (best.layout == OG_LAYOUT_ELL || best.layout == 0);
    const int occ = best.engine == OG_ENGINE_ASYNC ? g->occ_async_l[ell] : g->occ_l[ell];
    if (occ > 0) best.blocks_per_sm = (uint32_t)occ;
  }
  g->cfg = best;
  if (out) *out = best;
  return OG_OK;
}

}  // namespace

int og_autotune(og_graph* g, uint32_t kind, const uint32_t* srcs, const uint32_t* dsts,
                uint32_t nsample, uint32_t delta_lo, uint32_t delta_hi, og_config* out) {
  if (!g || !srcs || nsample == 0 || kind > OG_Q_WBFS) return OG_E_INVALID;
  if ((kind == OG_Q_PPSP || kind == OG_Q_ASTAR) && !dsts) return OG_E_INVALID;
  std::vector<og_query> qs(nsample);
  for (uint32_t i = 0; i < nsample; ++i)
    qs[i] = og_query{kind, srcs[i], dsts ? dsts[i] : 0u, 0u};
  return autotune_queries(g, qs, delta_lo, delta_hi, out);
}

int og_autotune_batch(og_graph* g, const og_query* queries, uint32_t nq, uint32_t delta_lo,
                      uint32_t delta_hi, og_config* out) {
  if (!g || !queries || nq == 0) return OG_E_INVALID;
  std::vector<og_query> qs(queries, queries + nq);
  for (const og_query& q : qs)
    if (q.kind > OG_Q_WBFS || q.src >= g->n ||
        ((q.kind == OG_Q_PPSP || q.kind == OG_Q_ASTAR) && q.dst >= g->n))
      return OG_E_INVALID;
  return autotune_queries(g, qs, delta_lo, delta_hi, out);
}

}  // extern "C"

// ---- allocation-free entry point ----------------------------------------------------------
// og_sssp_delta_noalloc runs the same round-synchronous kernel as og_sssp_delta, but its
// scratch (query cursor, barrier words, counters, bucket ring and overflow pile) lives in
// the fixed device array below instead of memory the library allocates.  It serves
// callers that cannot call cudaMalloc: code inside a host application whose allocator has
// already claimed the device memory, code on a path where cudaMalloc's implicit device
// synchronisation is not acceptable, and code that must not meet an out-of-memory error
// after start-up.  The array is reserved on every GPU that loads the library, for the
// life of the process.
namespace og {

constexpr size_t kNoAllocBytes = 64ull << 20;           // scratch array size (64 MiB)
constexpr uint32_t kNoAllocMaxN = 1u << 20;             // largest graph accepted
constexpr int kNoAllocMaxDevices = 64;
constexpr uint32_t kNoAllocRing = kMaxRing;             // materialised buckets
// Header of the array (byte offsets), then the bucket arena from kNoAllocHeader on.
constexpr size_t kNaSync = 0, kNaStats = 256, kNaQDesc = 512, kNaQState = 768;
constexpr size_t kNaPref = 1024, kNaCheck = 1536, kNaCounts = 2048, kNaHeader = 4096;
static_assert(sizeof(Sync) <= kNaStats - kNaSync, "Sync overlaps Stats in the header");
static_assert(sizeof(Stats) <= kNaQDesc - kNaStats, "Stats overlaps the query descriptor");
static_assert(sizeof(QDesc) <= kNaQState - kNaQDesc, "QDesc overlaps the query state");
static_assert(sizeof(QState) <= kNaPref - kNaQState, "QState overlaps the frontier prefix");
static_assert(2 * sizeof(uint32_t) <= kNaCheck - kNaPref, "prefix (nq + 1 words) overflows");
static_assert(sizeof(uint32_t) <= kNaCounts - kNaCheck, "check word overlaps the counters");
static_assert(kNoAllocRing * sizeof(uint32_t) <= kNaHeader - kNaCounts,
              "ring counters overflow the header");
static_assert(kNaHeader % 256 == 0 && kNoAllocBytes > kNaHeader, "arena alignment");

static __device__ __align__(256) unsigned char og_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
struct NoAllocDev {
  unsigned long long ctx_id = 0;  // context the address below belongs to (0 = none yet)
  void* ptr = nullptr;
  int occ = 0, sms = 0;
};
NoAllocDev g_noalloc[kNoAllocMaxDevices];

// Identifier of the calling thread's current CUDA context (unique for the life of the
// process), through the driver entry points the runtime exposes: a context re-created
// after cudaDeviceReset loads the module again, possibly at another address, and gets
// a new identifier.  0 when it cannot be read.
unsigned long long current_ctx_id() {
  using GetCur = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<GetCur>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  if (!get_cur || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}
}  // namespace

}  // namespace og

extern "C" int og_launch_status(uint32_t err, uint32_t bad_code, uint32_t bad_val,
                                uint32_t bad_aux, uint32_t arena_out) {
  return launch_status(err, bad_code, bad_val, bad_aux, arena_out != 0);
}

extern "C" int og_sssp_delta_noalloc(const uint32_t* offsets, const uint32_t* edges, uint32_t n,
                                     uint64_t m, uint32_t src, uint32_t delta,
                                     uint32_t* dist_out, void* stream) {
  using namespace og;
  if (!offsets || !dist_out || (m && !edges) || n == 0 || src >= n || delta == 0)
    return OG_E_INVALID;
  if (n > kNoAllocMaxN || m >= 0xFFFFFFFFull) return OG_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return OG_E_INVALID;
  const size_t smem = delta_smem_bytes(kBinCap);
  void* base = nullptr;
  int occ = 0, sms = 0;
  {
    // Set-up, once per device (and again if the device's context was re-created), with
    // that device current: the device address of the array -- in host code the array's
    // name is only a host-side stand-in -- and the launch shape.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDev& d = g_noalloc[dev];
    const unsigned long long ctx = current_ctx_id();
    if (!d.ptr || ctx == 0 || ctx != d.ctx_id) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, og_noalloc_scratch));
      if (!p) return OG_E_CUDA;
      if (!d.occ) {
        CK(delta_occupancy(&d.occ, smem, false));
        CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        if (d.occ < 1) {
          snprintf(g_cuda_msg, sizeof(g_cuda_msg), "persistent kernel does not fit on an SM");
          return OG_E_CUDA;
        }
      }
      d.ptr = p;
      d.ctx_id = ctx;
    }
    base = d.ptr;
    occ = d.occ;
    sms = d.sms;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  Sync* sync = reinterpret_cast<Sync*>(b + kNaSync);
  Stats* stats = reinterpret_cast<Stats*>(b + kNaStats);
  QDesc* qd = reinterpret_cast<QDesc*>(b + kNaQDesc);
  QState* qs = reinterpret_cast<QState*>(b + kNaQState);
  uint32_t* pref = reinterpret_cast<uint32_t*>(b + kNaPref);
  uint32_t* check = reinterpret_cast<uint32_t*>(b + kNaCheck);
  uint32_t* counts = reinterpret_cast<uint32_t*>(b + kNaCounts);
  // The weights are not scanned, so the widest ring is used (a relaxation may jump up
  // to kNoAllocRing - 1 buckets before it spills to the overflow pile).
  const uint32_t B = kNoAllocRing;
  const uint64_t arena = (kNoAllocBytes - kNaHeader) / sizeof(uint2);
  const uint32_t cap = (uint32_t)(arena / 2 / B);
  const uint32_t ocap = (uint32_t)(arena / 4);
  uint2* ring = reinterpret_cast<uint2*>(b + kNaHeader);
  uint2* ovf = ring + (size_t)B * cap;
  const uint2* adj = reinterpret_cast<const uint2*>(edges);

  // Calls share the array: its state words start from zero on every call (two calls
  // that overlap on the GPU would race on them).  The caller's graph is checked first
  // and the search only runs on a well-formed one.
  uint32_t hcheck = 0;
  CK(cudaMemsetAsync(b, 0, kNaHeader, st));
  CK(launch_check_csr(offsets, adj, n, (uint32_t)m, check, sms, st));
  CK(cudaMemcpyAsync(&hcheck, check, sizeof(hcheck), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hcheck) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "graph rejected:%s%s",
             (hcheck & 1u) ? " offsets not 0 .. m and non-decreasing" : "",
             (hcheck & 2u) ? " a neighbor id >= n" : "");
    return OG_E_INVALID;
  }

  QDesc hq;
  memset(&hq, 0, sizeof(hq));
  hq.src = src;
  hq.dst = kNone;
  hq.delta = delta;
  hq.kind = kSSSP;
  Params P{};
  P.off = offsets;
  P.adj = adj;
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
  P.hub_min = 0xFFFFFFFFu;  // no hub list (it would need more scratch)
  P.nq = 1;
  P.B = B;
  P.Bmask = B - 1;
  P.cap = cap;
  P.ocap = ocap;
  P.T = kDefaultFusion;
  P.tile = 128;
  P.bin_cap = kBinCap;
  P.max_rounds = 0xFFFFFFFFu;
  P.has_astar = 0;
  P.spin_ns = kDefaultSpinNs;
  CK(cudaMemcpyAsync(qd, &hq, sizeof(hq), cudaMemcpyHostToDevice, st));
  CK(launch_fill(dist_out, n, nullptr, 1, sms, st));
  CK(launch_init(P, nullptr, 1, st));
  CK(launch_delta(P, sms * occ, smem, st));
  Sync hs;
  QState hqs;
  CK(cudaMemcpyAsync(&hs, sync, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hqs, qs, sizeof(hqs), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return launch_status(hs.err, hs.bad_code, hs.bad_val, hs.bad_aux, hqs.aborted != 0);
}
