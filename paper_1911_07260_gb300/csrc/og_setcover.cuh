// Internal structures of the approximate set cover kernel (og_setcover.cu), not part of
// the ABI.
#pragma once
#include "og_internal.cuh"

namespace og {

// ---- approximate set cover (og_setcover.cu) ----------------------------------------------
// Section 6.1 "Approximate Set Cover": the set of vertex v is its adjacency list, sets are
// bucketed by their number of uncovered elements on an integer (1 + eps) ladder, and the
// highest non-empty bucket is worked off in steps; a step recounts the bucket's sets
// (leave / move down / active), gives each uncovered element of an active set to the
// active set of smallest priority, and adds the active sets that received at least
// tau_j elements to the cover.
//
// Buckets live in band lists: band b holds every live set whose bucket is in
// [16 b, 16 b + 16), as (bucket << 32 | set) entries, in one of two buffers.  Gathering
// bucket j scans its band once: the members go to the step's member lists, the others
// are compacted into the band's other buffer.  A set enters each band at most once
// (buckets only fall), so band b needs room for the sets whose first bucket is in a band
// >= b: sum over sets of (first band + 1) <= n + m / 16 entries in all.
//
// A set's residual elements are packed (covered ones dropped) every time it is visited,
// alternating between two element buffers laid out like the adjacency array; the storage
// of a set is 0 (the graph's adjacency, never packed yet), 1 or 2.
constexpr uint32_t kScBand = 16;             // buckets per band
constexpr uint32_t kScChunk = 256;           // elements per warp claim of large sets
constexpr uint32_t kScLenBits = 30;          // residual size | storage << 30
constexpr uint32_t kScLenMask = (1u << kScLenBits) - 1u;
constexpr uint32_t kScMinHub = 16;           // a chunk then spans at most 17 large sets
constexpr uint32_t kScMaxHub = 1u << 26;     // a group of 32 small sets spans < 2^31 elements
constexpr uint32_t kScMaxBuckets = 1u << 22;
constexpr uint32_t kScCntShift = 36;         // large lists: (entries << 36) | elements
constexpr unsigned long long kScTotMask = (1ull << kScCntShift) - 1ull;

enum ScPhase : uint32_t {
  kScGather = 0,    // band entries of bucket j -> member lists; the rest compacted
  kScA = 1,         // pack every member (drop covered elements); small sets also classify
                    // themselves and claim the elements of the active ones
  kScA2 = 2,        // large sets: classify and claim
  kScB = 3,         // small sets: count received elements, join or stay, cover, move;
                    // large sets: count received elements
  kScC = 4,         // large sets: join or stay, cover, move
  kScStop = 5,
  kScPrologue = 6,
};

// Members of the current bucket (a step reads one pair of lists and appends the sets
// that stay to the other).
struct ScList {
  uint32_t* id;     // set
  uint32_t* lw;     // residual size | storage << 30, when listed
  uint32_t* dn;     // uncovered elements found by this step's pack
  uint32_t* wn;     // elements received this step
  uint32_t* st;     // large lists: first index of the set in the step's element space
};

struct ScState {
  uint32_t j;               // bucket being worked off
  uint32_t band;            // its band
  uint32_t step;            // steps run (the number of the current step)
  uint32_t csel;            // current member lists (0 / 1)
  uint32_t ns[2];           // small member lists: entries
  unsigned long long bw[2]; // large member lists: (entries << 36) | elements
  uint32_t gmax;            // gather: largest bucket among the band entries kept
  uint32_t gcnt;            // gather: band entries kept
  uint32_t gathers;         // buckets gathered
  uint32_t pad;
};

struct ScParams {
  const uint32_t* off;
  const uint2* adj;
  uint32_t n;
  const uint32_t* pri;          // priorities, a permutation of 0 .. n-1
  uint32_t* step_out;           // step in which each set joined (0 = never)
  uint32_t* len;                // residual size | storage << 30, of sets in band lists
  uint32_t* pk[2];              // packed element buffers (storage 1, 2), m entries each
  uint8_t* cov;                 // element covered
  unsigned long long* claim;    // ((~step) << 32) | priority of the element's claimant
  const uint32_t* t;            // ladder t[0 .. nb]
  const uint32_t* tau;          // received elements a set of bucket j needs to join
  uint32_t nb, nbands;
  unsigned long long* bl;       // band list entries
  const unsigned long long* bbase;  // band b: buffer 0 at bl + bbase[b], buffer 1 + bcap[b]
  const uint32_t* bcap;
  uint32_t* bcnt;               // entries in the band's current buffer
  uint32_t* bsel;               // the band's current buffer
  uint32_t* bmax;               // largest bucket among the band's entries
  uint32_t* hist;               // sets per first band (planning)
  unsigned long long bl_entries;  // room in bl
  uint32_t* seen;               // priority bitmap (validation)
  ScList sm[2], lg[2];          // small / large member lists
  uint32_t lg_cap;
  uint32_t hub;                 // residual size from which a set is large
  Sync* sync;
  ScState* ss;
  Stats* stats;
  unsigned long long spin_ns;
};

// Codes of report_bad from the set cover kernels.
constexpr uint32_t kScBadPriority = 60;  // priorities are not a permutation of 0 .. n-1

}  // namespace og
