// Internal device structures of libog (not part of the ABI).
//
// Layout in HBM (one launch serves nq queries; query q is a "slot"):
//   off    uint32[n+1]      CSR offsets (read-only)
//   adj    uint2[m]         {neighbor, weight} pairs, one 8-byte load per edge
//   xy     float2[n]        coordinates (A* only)
//   dist   uint32[nq][n]    priority vector per query (Section 4.1: the dist vector)
//   ring   uint2[nq][B][cap]  materialised buckets: entries {vertex, dist at insert}
//   counts uint32[nq][B]    append counters of the ring slots
//   ovf    uint2[nq][2][ocap] overflow pile (double-buffered for redistribution)
//   qs     QState[nq]       bucket cursor of each query
//   sync   Sync             grid-barrier words, phase, error bits
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace og {

constexpr uint32_t kInf = 0xFFFFFFFFu;   // unreachable
constexpr uint32_t kSat = 0xFFFFFFFEu;   // saturated distance
constexpr uint32_t kNone = 0xFFFFFFFFu;  // no target
constexpr int kBlock = 256;              // threads per persistent CTA
constexpr int kWarps = kBlock / 32;
constexpr int kMaxQ = 512;               // queries per launch
constexpr int kMaxRing = 256;            // materialised buckets per query
constexpr uint32_t kOutbox = 512;        // staged entries of later buckets per CTA

// Dynamic shared memory of the round engine's persistent kernel: two CTA-local bins of
// bin_cap entries ({vertex, distance} + 16-bit query), then the outbox of kOutbox
// {vertex, distance, query, bucket} entries (16-byte aligned).
__host__ __device__ constexpr size_t bins_smem_bytes(uint32_t bin_cap) {
  return ((size_t)2 * bin_cap * (sizeof(uint2) + sizeof(uint16_t)) + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t delta_smem_bytes(uint32_t bin_cap) {
  return bins_smem_bytes(bin_cap) + (size_t)kOutbox * sizeof(uint4);
}

// kBF: unordered Bellman-Ford; its QDesc.delta is 0 and every insert goes to bucket
// cur + 1, so a bucket is one round's frontier.
enum Kind : uint32_t { kSSSP = 0, kPPSP = 1, kASTAR = 2, kBF = 3 };

enum Phase : uint32_t {
  kPhRelax = 0,      // process the current buckets (frontier pass + fused local loop)
  kPhRedistMin = 1,  // overflow pile: smallest live bucket
  kPhRedistMove = 2, // overflow pile: move entries of the new ring window into the ring
  kPhStop = 3,
  kPhPrologue = 4,   // kernel start: publish the frontier of the current state
  kPhBig = 5,        // edges of very-high-degree vertices, split over all CTAs
  kPhApply = 6,      // lazy bucket update: one insertion per vertex marked this round
  kPhPull = 7,       // direction optimisation: queries with a large frontier pull (every
                     // unsettled vertex scans its in-edges for current-bucket neighbours)
};

// A vertex whose out-degree is at least Params::hub_min (a hub of a skewed graph) is not
// expanded by the CTA that meets it: it is listed, and after the round every warp of the
// grid claims kBigSub-edge pieces of the listed hubs.  Each hub owns a contiguous range of
// kBigChunk-edge chunks; the chunk map names the hub of every chunk.
constexpr uint32_t kBigChunk = 1024;
constexpr uint32_t kBigSub = 256;                  // edges per warp claim
constexpr uint32_t kBigSubs = kBigChunk / kBigSub;  // claims per chunk
struct BigItem {
  uint32_t u, g, q, beg, end, cbase;  // cbase: first chunk of this hub
};

enum ErrBits : uint32_t { kErrTimeout = 1, kErrArena = 2, kErrSat = 4, kErrBounds = 8 };
// A timeout stops the launch; an exhausted arena only stops the query that hit it.
constexpr uint32_t kErrFatal = kErrTimeout | kErrBounds;

struct QDesc {
  uint32_t src, dst, delta, kind;
  float tx, ty;          // target coordinates (A*)
  uint32_t pad0, pad1;
};

struct QState {
  uint32_t cur;          // current bucket index
  uint32_t head, tail;   // frontier = ring slot(cur) positions [head, tail)
  uint32_t active;       // 1 while the query runs
  uint32_t ovf_n;        // entries appended to the active overflow pile
  uint32_t ovf_min;      // smallest bucket appended to it since the last redistribution
  uint32_t ovf_sel;      // active pile (0 / 1)
  uint32_t redist;       // redistribution in progress
  uint32_t ovf_n2, ovf_min2;  // the other pile during a redistribution
  uint32_t redist_min;   // smallest live bucket found by the redistribution
  uint32_t no_exit;      // A*: early exit disabled (a key fell below the cursor)
  uint32_t result;       // dist(src, dst) once finished
  uint32_t aborted;      // bucket arena exhausted: the query stopped early
  uint32_t pull;         // this round's frontier is processed by a pull phase
  uint32_t pad;
};

struct Sync {
  uint32_t arrive;       // barrier arrivals
  uint32_t gen;          // barriers released in this launch
  uint32_t err;          // ErrBits (sticky)
  uint32_t phase;        // phase to run after the barrier
  uint32_t work;         // frontier tiles claimed in this phase
  uint32_t total;        // frontier entries in this phase
  uint32_t rounds;       // rounds run in this launch
  uint32_t any_active;
  uint32_t active;       // barrier-free engine: queries not yet finished
  uint32_t big_claim;    // hub pieces claimed in the BIG phase (round engine)
  uint32_t bad_code;     // first failed internal bounds check (0 = none)
  uint32_t bad_val;      // the offending value
  uint32_t bad_aux;      // context (query or position)
  uint32_t progress;     // barrier-free engine: heartbeat of busy warps
  uint32_t timeout_at;   // which bounded wait gave up (1 idle, 2 entry hand-off)
  uint32_t lz_n;         // lazy bucket update: vertices marked this round
  unsigned long long big_word;  // (listed hubs << 32) | chunks reserved, this round
};

enum StatIdx {
  kStRounds, kStFused, kStItems, kStStale, kStRelax, kStImproved, kStLocal, kStGlobal,
  kStOvf, kStRedist, kStFlush,
  kStTFrontier, kStTFused, kStTBarrier, kStTHub,  // ns summed over CTAs (round engine)
  kStCount
};
struct Stats { unsigned long long v[16]; };

struct Params {
  const uint32_t* off;
  const uint2* adj;
  const uint4* ell;       // ELL-8 rows (64 B per vertex, unused slots have neighbor
                          // 0xFFFFFFFF) or null: then offsets + adj are used
  const float2* xy;
  uint32_t n;
  uint32_t xy_integral;   // coordinates integral and < 2^24 in magnitude
  uint32_t* dist;         // nq * n
  const QDesc* qd;
  QState* qs;
  uint2* ring;
  uint32_t* counts;
  uint2* ovf;
  uint32_t* fr_pref;      // nq + 1 prefix sums of the frontier sizes
  Sync* sync;
  Stats* stats;
  BigItem* big;           // hubs listed in the current round (or null: no hub list)
  uint32_t* big_map;      // chunk -> hub slot (kNone: chunk of a hub that did not fit)
  uint32_t big_cap;       // hub slots
  uint32_t map_cap;       // chunk map entries
  uint32_t hub_min;       // out-degree from which a vertex is listed as a hub
  uint32_t nq;
  uint32_t B, Bmask;
  uint32_t cap;           // entries per ring slot
  uint32_t ocap;          // entries per overflow pile
  uint32_t T;             // fusion threshold (0 = off)
  uint32_t tile;          // frontier entries per CTA grab
  uint32_t bin_cap;       // CTA-local bin capacity per buffer
  uint32_t max_rounds;    // stop (resumably) after this many rounds
  uint32_t has_astar;
  uint32_t precheck;      // load dist[v] first; atomicMin only if the new value is smaller
  uint32_t prefetch;      // prefetch an inserted vertex's adjacency into L2
  uint32_t lazy;          // lazy bucket update (Section 3.1) instead of eager inserts
  uint32_t lz_words;      // words per query of the marked-vertex bitmap
  uint32_t* lz_bits;      // nq x lz_words: vertex improved this round
  uint2* lz_list;         // {vertex, query} marked this round
  uint32_t lz_cap;
  unsigned long long spin_ns;
  // Direction optimisation (pull_div 0 = off): a query's round is a pull phase when its
  // frontier holds more than n / pull_div entries; tin / tadj = the in-edges (transpose).
  uint32_t pull_div;
  const uint32_t* toff;
  const uint2* tadj;      // {source, weight} per in-edge
};

// ---- barrier-free engine (og_async.cu) -----------------------------------------------
enum AMode : uint32_t { kMRelax = 0, kMRedistMin = 1, kMRedistMove = 2, kMDone = 3 };

struct AQState {
  unsigned long long word;  // (epoch << 32) | next unclaimed position of the current task
  uint32_t mode;            // AMode: relax the current bucket / redistribute the pile
  uint32_t cur;             // current bucket
  uint32_t work;            // outstanding entries of the current task
  uint32_t limit;           // size of a redistribution task
  uint32_t ovf_n, ovf_min, ovf_sel, ovf_n2;
  uint32_t ovf_min2, redist_min, no_exit, result;
  uint32_t aborted;         // arena exhausted: the query stopped early
  uint32_t dirty;           // ring positions may still hold entries (early exit / abort)
  uint32_t advances;        // bucket / task transitions
  uint32_t redists;         // overflow-pile redistributions
};

struct AParams {
  const uint32_t* off;
  const uint2* adj;
  const uint4* ell;
  const float2* xy;
  uint32_t n;
  uint32_t xy_integral;
  uint32_t* dist;
  const QDesc* qd;
  AQState* aq;
  uint2* ring;              // positions hold {v, d} packed in 64 bits, or all ones when free
  uint32_t* counts;
  uint2* ovf;
  Sync* sync;
  Stats* stats;
  uint32_t nq;
  uint32_t B, Bmask;
  uint32_t cap, ocap;
  uint32_t T;               // fusion threshold (0 = off)
  uint32_t lq_cap;          // per-warp FIFO capacity (entries)
  uint32_t has_astar;
  uint32_t precheck;
  uint32_t prefetch;
  unsigned long long spin_ns;
  unsigned long long budget_ns;  // stop (resumably) after this long; 0 = run to the end
  uint32_t* touched;        // nq x tb_words bitmap of kTouchBlock-vertex blocks holding a
                            // vertex this query reached (server: lets a slot's distance
                            // row be reset block by block); null = not tracked
  uint32_t tb_words;
};

// Granularity of the server's touched-vertex bitmap: one bit per 256 consecutive vertices.
constexpr uint32_t kTouchShift = 8;
constexpr uint32_t kTouchBlock = 1u << kTouchShift;
__host__ __device__ constexpr uint32_t touch_words(uint32_t n) {
  return (uint32_t)(((uint64_t)n + ((uint64_t)kTouchBlock << 5) - 1) / ((uint64_t)kTouchBlock << 5));
}

}  // namespace og
