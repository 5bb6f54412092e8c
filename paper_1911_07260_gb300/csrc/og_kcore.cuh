// Internal structures of the k-core kernel (og_kcore.cu), not part of the ABI.
#pragma once
#include "og_internal.cuh"

namespace og {

// ---- k-core peeling (og_kcore.cu) --------------------------------------------------------
// Section 6.1 "k-core" with the lazy bucketing of Section 5.1: priority = degree at start,
// the minimum non-empty bucket is the level k, extracting a vertex lowers each neighbour
// with a higher priority by one, floored at k.  A window of kKRing buckets [base,
// base + kKRing) is materialised; vertices above it are found by a scan when the window
// runs dry (the overflow bucket of the lazy queue), and a bucket that ran out of space is
// rebuilt by a scan at its level.
constexpr uint32_t kKRing = 256;
enum KPhase : uint32_t {
  kKMin = 0,    // smallest priority >= lo among all vertices (window refill, step 1)
  kKFill = 1,   // vertices with priority in [base, base + kKRing) -> their buckets
  kKScan = 2,   // vertices with priority == k -> frontier list (bucket that overflowed)
  kKPeel = 3,   // extract the frontier; lazy: count neighbour updates, eager: apply them
  kKApply = 4,  // lazy: apply each counted vertex's updates once (priority, bucket); the
                // vertices that drop to k are extracted in the same phase, their
                // neighbours counted into the other list
  kKStop = 5,
  kKPrologue = 6,
  kKHub = 7,    // edges of the round's hub vertices, split over every warp of the grid
};
struct KState {
  uint32_t k;          // current level (priority of the bucket being extracted)
  uint32_t base;       // first priority of the materialised window
  uint32_t cur;        // bucket index of level k in the window
  uint32_t fr_list;    // frontier: 0 = ring bucket cur, 1 = list[fsel]
  uint32_t fsel;       // list holding the frontier
  uint32_t fr_n;       // frontier entries
  uint32_t next_n[2];  // appends to list[0] / list[1] (vertices that dropped to k)
  uint32_t touched_n[2];  // lazy: vertices counted into touched[0] / touched[1]
  uint32_t tsel;          // lazy: list the counting phases append to (apply reads the other)
  uint32_t kmin;       // refill: smallest priority found
  uint32_t lo;         // refill: priorities below lo are settled
  uint32_t levels;     // levels extracted
  uint32_t scans;      // levels rebuilt by a scan
  uint32_t refills;    // window refills
  uint32_t asel;       // list receiving the vertices that drop to k this round
  uint32_t hub_claim;  // hub pieces claimed in the hub phase
  unsigned long long hub_word;  // (hubs listed << 32) | chunks reserved, this round
};
struct KParams {
  const uint32_t* off;
  const uint2* adj;
  uint32_t n;
  uint32_t* prio;       // priority; coreness when the kernel ends
  uint32_t* cnt;        // lazy: per-vertex count of extracted neighbours not yet applied
  uint32_t* touched[2]; // lazy: vertices whose count became non-zero, two lists
  uint32_t* list[2];    // frontier lists of the current level
  uint32_t* ring;       // kKRing buckets x cap vertex ids
  uint32_t* counts;     // appends per bucket
  uint32_t* lossy;      // bucket ran out of space: rebuild it by a scan at its level
  Sync* sync;
  KState* ks;
  Stats* stats;
  BigItem* hub;         // frontier vertices of out-degree >= hub_min this round
  uint32_t* hub_map;    // chunk -> hub slot
  uint32_t hub_cap, map_cap, hub_min;
  uint32_t cap;
  uint32_t eager;       // 1: eager bucket update (a CAS decrement and an insert per edge)
  uint32_t tile;
  unsigned long long spin_ns;
};

}  // namespace og
