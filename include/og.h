/*
 * og.h -- C ABI of the GB300 ordered shortest-path library (libog.so).
 *
 * The library computes single-source and point-to-point shortest paths with
 * Delta-stepping over a bucketed priority queue, using eager bucket updates and bucket
 * fusion (Section 3.2, the eager bucket update, and Section 3.3, bucket fusion, with
 * their figure of SSSP with eager updates and fusion).  Weighted BFS, PPSP and A* are
 * variants of the same loop (Section 6.1).  The lazy bucket update (Section 3.1), the
 * unordered Bellman-Ford baseline and k-core by peeling (Section 6.1, lazy with the
 * constant-sum reduction of Section 5.1, or eager) complete the comparisons of Section
 * 6.4; approximate set cover (Section 6.1) is the other bucketed ordered algorithm of
 * the paper's evaluation.  Every step runs in CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Vertices are uint32 ids in [0, n).  Weights are non-negative uint32.  Every id and
 *     per-vertex array crossing this interface is in the caller's numbering, whatever
 *     order the library keeps the graph in on the device (og_graph_set_order).
 *   - Distances are uint32; 0xFFFFFFFF means "unreachable" (the INT_MAX initialisation
 *     of the paper's priority vector, Section 4.1).  A path whose length reaches
 *     0xFFFFFFFE saturates there and the call returns OG_E_OVERFLOW.
 *   - "stream" is a cudaStream_t (NULL = legacy default stream).  Work is issued on it.
 *     Single-query calls and og_batch_run synchronise that stream before returning so
 *     they can report a status; device outputs are complete when they return OG_OK.
 *   - Ownership: the caller owns every buffer it passes; the library owns the og_graph
 *     and its device copies and scratch (bucket arenas, query state), and frees them in
 *     og_graph_free / og_server_free.
 *   - Errors: every int-returning call returns OG_OK (0) or one of the OG_E_* codes.  On
 *     error the outputs are unspecified.  No call aborts the process.
 *   - Thread safety: calls on one og_graph (or one og_server) must not overlap.
 */
#ifndef OG_H
#define OG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OG_OK 0
#define OG_E_INVALID 1   /* bad argument: n = 0, vertex out of range, offsets not
                            monotone, m >= 2^32, zero weight on wBFS, ...            */
#define OG_E_OOM 2       /* device or host allocation failed                         */
#define OG_E_CUDA 3      /* a CUDA runtime call failed (og_last_cuda_error tells which) */
#define OG_E_OVERFLOW 4  /* a distance reached the saturation value 0xFFFFFFFE       */
#define OG_E_TIMEOUT 5   /* a bounded device wait (grid barrier) gave up             */
#define OG_E_BUSY 6      /* no free serving slot                                      */
#define OG_E_ARENA 7     /* bucket arena exhausted even after regrowth                */
#define OG_E_INTERNAL 8  /* an internal consistency check failed inside a kernel (the
                            access was skipped; og_last_cuda_error has the details)   */

/* Query kinds (Section 6.1). */
#define OG_Q_SSSP 0      /* all distances from src                                    */
#define OG_Q_PPSP 1      /* dist(src, dst); stops on entering bucket i with
                            i * Delta >= best dist(src, dst) found so far             */
#define OG_Q_ASTAR 2     /* dist(src, dst) with priority g + h, h = floor(100 * Euclid) */
#define OG_Q_WBFS 3      /* SSSP with Delta = 1 (positive integer weights required)   */
#define OG_Q_BF 4        /* all distances from src by unordered, frontier-based
                            Bellman-Ford (the unordered baseline of Section 6's
                            comparison): round r relaxes the out-edges of every vertex
                            improved in round r - 1, with no priority order and no
                            fusion.  Round engine only (a batch holding one runs on it);
                            not accepted by the server or the autotuner.  The query's
                            delta field is ignored.                                   */

typedef struct og_graph og_graph;
typedef struct og_server og_server;

/* Schedule knobs: the scheduling language of Section 4.2 (its table of scheduling
 * functions for priority updates) as plain fields.  0 selects the graph's tuned or
 * default value for every field. */
typedef struct og_config {
  uint32_t delta;            /* priority coarsening factor (Section 2), >= 1          */
  uint32_t fusion_threshold; /* bucket fusion: a CTA keeps draining its local bin of the
                                current bucket while 0 < size < threshold (Section 3.3);
                                OG_FUSION_OFF disables fusion, 0xFFFFFFFF = unbounded   */
  uint32_t expand_tile;      /* frontier entries a CTA claims per grab (multiple of 32;
                                0 = 32 for average degree <= 8, else 256)              */
  uint32_t blocks_per_sm;    /* persistent CTAs per SM (capped by occupancy)           */
  uint32_t ring_buckets;     /* materialised buckets (power of two, <= 256); further
                                buckets go to one overflow pile (Section 5.1's lazy
                                queue idea of a few materialised buckets + overflow)   */
  uint32_t engine;           /* OG_ENGINE_ROUNDS or OG_ENGINE_ASYNC (0 = default: rounds) */
  uint32_t precheck;         /* read dist[v] before the atomicMin and skip relaxations that
                                cannot improve: OG_PRECHECK_ON / _OFF (0 = on when the
                                average degree exceeds 8)                              */
  uint32_t layout;           /* adjacency read by the kernels: OG_LAYOUT_CSR, or
                                OG_LAYOUT_ELL (one 64-byte row of up to 8 edges per
                                vertex, built at upload when every degree is <= 8;
                                0 = ELL where the rows exist, else CSR; the server
                                defaults to CSR)                                       */
  uint32_t prefetch;         /* OG_PREFETCH_ON / _OFF: prefetch an inserted vertex's
                                adjacency into L2 (0 = off)                           */
  uint32_t hub_degree;       /* out-degree from which a frontier vertex is a hub: instead
                                of being expanded by the CTA that meets it, its edges
                                are split over every warp of the grid in a pass after
                                the round (round engine, CSR layout; 0 = default 4096,
                                0xFFFFFFFF = no hubs)                                  */
  uint32_t bucket_update;    /* OG_UPDATE_EAGER (Section 3.2; 0 = default) or
                                OG_UPDATE_LAZY (Section 3.1): a round only relaxes and
                                marks each improved vertex once; after the round every
                                marked vertex makes one insertion, into the bucket of
                                its final distance (the buffer reduction).  Lazy turns
                                fusion off and runs on the round engine.                */
  uint32_t pull_divisor;     /* direction optimisation (the pull direction of Section 4.2's
                                scheduling language; round engine, SSSP / wBFS queries):
                                a query's round pulls -- every vertex not yet settled
                                scans its in-edges for neighbours in the current bucket
                                -- when its frontier holds more than n / pull_divisor
                                entries, and pushes otherwise.  0 = always push (the
                                default).  The in-edges are built on the device the first
                                time a pull is asked for and kept with the graph.      */
  uint64_t spin_limit_ns;    /* cap on each grid-barrier wait (default 2 s)            */
  uint64_t arena_entries;    /* bucket-entry capacity per query (ring + overflow)      */
} og_config;

#define OG_FUSION_OFF 0xFFFFFFFEu
#define OG_UPDATE_EAGER 1u
#define OG_UPDATE_LAZY 2u

/* Engines.  Both run the same eager Delta-stepping with bucket fusion and give the same
 * distances.  ROUNDS (the default) follows the paper's round structure: every CTA fuses
 * rounds of its local bucket with block-level synchronisation, and rounds are separated
 * by a grid-wide barrier (rounds counts those barriers).  ASYNC replaces the grid barrier
 * by a per-query completion count: each warp fuses its own local bucket, idle warps take
 * over copied buckets, and a query moves to its next bucket the moment its current one
 * has no outstanding entry (rounds counts those bucket transitions). */
#define OG_PRECHECK_ON 1u
#define OG_PRECHECK_OFF 2u
#define OG_LAYOUT_CSR 1u
#define OG_LAYOUT_ELL 2u
#define OG_PREFETCH_ON 1u
#define OG_PREFETCH_OFF 2u

#define OG_ENGINE_DEFAULT 0u
#define OG_ENGINE_ROUNDS 1u
#define OG_ENGINE_ASYNC 2u

/* Counters of one call (summed over its queries). */
typedef struct og_stats {
  uint64_t rounds;           /* global rounds (grid-wide barriers between phases)      */
  uint64_t fused_iters;      /* CTA-local fused iterations (summed over CTAs)          */
  uint64_t items;            /* bucket entries dequeued                                */
  uint64_t stale;            /* dequeued entries skipped as out of date                */
  uint64_t relax;            /* edges relaxed                                          */
  uint64_t improved;         /* relaxations that lowered a distance                    */
  uint64_t local_inserts;    /* inserts kept in a CTA-local bin (fusion)               */
  uint64_t global_inserts;   /* inserts into materialised global buckets               */
  uint64_t overflow_inserts; /* inserts into the overflow pile                         */
  uint64_t redistributions;  /* overflow-pile redistributions                          */
  uint64_t restarts;         /* arena regrowth restarts                                */
  uint64_t kernel_ns;        /* device time of the persistent kernel(s), CUDA events   */
  uint64_t flushes;          /* local buckets copied to a global bucket (fusion limit) */
  uint64_t t_frontier_ns;    /* round engine, summed over CTAs: frontier passes,       */
  uint64_t t_fused_ns;       /*   fused-round loops,                                   */
  uint64_t t_barrier_ns;     /*   grid-barrier waits,                                  */
  uint64_t t_hub_ns;         /*   and hub passes (BIG phase)                           */
} og_stats;

typedef struct og_query {
  uint32_t kind;             /* OG_Q_*                                                 */
  uint32_t src;
  uint32_t dst;              /* PPSP / A*: target; ignored otherwise                   */
  uint32_t delta;            /* 0 = config / graph default                             */
} og_query;

/* ---- graph -------------------------------------------------------------------------
 * og_graph_upload: copies a CSR graph to the device (Section 4.1: an edgeset with
 * integer weights).  offsets: host uint64[n+1], non-decreasing, offsets[0] = 0,
 * offsets[n] = m < 2^32.  neighbors, weights: host uint32[m]; the out-edges of u are
 * neighbors[offsets[u] .. offsets[u+1]) with the matching weights.  The library keeps
 * its own copy (uint32 offsets, interleaved {neighbor, weight} pairs).  A graph of at
 * least 2^20 vertices whose n/8 highest-degree vertices hold half of the edges or more
 * (a power-law graph) is stored hot-first (og_graph_set_order), if the device has the
 * memory for the rebuild.  Returns OG_E_INVALID for n = 0, bad offsets or a neighbor >= n. */
int og_graph_upload(const uint64_t* offsets, const uint32_t* neighbors,
                    const uint32_t* weights, uint32_t n, uint64_t m, void* stream,
                    og_graph** out);

/* Vertex coordinates for A*: float32[2n] as (x, y) pairs, host or device pointer (the
 * library detects which).  Copied.  The A* heuristic is floor(100 * Euclidean distance)
 * to the target; with integral coordinates below 2^24 it is computed exactly in
 * integers, otherwise as max(0, floor(100 * d) - 1) in double. */
int og_graph_set_coords(og_graph* g, const float* xy, void* stream);

/* Vertex order on the device (a layout choice; every result is the same).  Every search
 * reads the distance of each relaxed edge's target at random, and on a power-law graph
 * most of those reads hit a few high-degree vertices.  OG_ORDER_HOT_FIRST stores the n/8
 * vertices of largest degree (ties: smaller id) at device ids 0 .. n/8 - 1 in that order,
 * and the vertices they displace at the ids they left, so the hot distance words share
 * cache lines that stay in L2; OG_ORDER_USER keeps the caller's ids; OG_ORDER_AUTO is the
 * upload's rule above.  Ids and per-vertex arrays keep the caller's numbering at every
 * call (sources, targets, coordinates, priorities, distances, coreness, join steps): the
 * library maps them, touching only the moved vertices.  The adjacency is rebuilt on the
 * device (needs a second copy of it for the duration; OG_E_OOM leaves the graph as it
 * was).  OG_E_BUSY while a server created on the graph exists; OG_E_INVALID for another
 * order.  Synchronises stream. */
#define OG_ORDER_AUTO 0u
#define OG_ORDER_HOT_FIRST 1u
#define OG_ORDER_USER 2u
int og_graph_set_order(og_graph* g, uint32_t order, void* stream);
/* The order in effect (OG_ORDER_HOT_FIRST or OG_ORDER_USER) and how many vertices have
 * a device id other than their own id (either pointer may be NULL). */
int og_graph_get_order(const og_graph* g, uint32_t* order, uint32_t* moved);
/* The hot-first order for out-degrees degrees[0 .. n) (host arrays; no device call):
 * device_to_user[x] receives the caller's vertex stored at device id x, and *hot_edges
 * (may be NULL) the edges the n/8 hottest vertices hold -- what og_graph_set_order
 * applies and what the upload's rule weighs.  OG_E_INVALID for NULL arrays or n = 0. */
int og_hot_first_order(const uint32_t* degrees, uint32_t n, uint32_t* device_to_user,
                       uint64_t* hot_edges);

/* n, m, minimum and maximum edge weight (any pointer may be NULL). */
int og_graph_info(const og_graph* g, uint32_t* n, uint64_t* m, uint32_t* min_w,
                  uint32_t* max_w);

/* Graph-level default schedule (og_autotune writes one).  0 fields keep defaults. */
int og_graph_set_config(og_graph* g, const og_config* cfg);
int og_graph_get_config(const og_graph* g, og_config* cfg);

void og_graph_free(og_graph* g);

/* Library defaults (Delta 0 = derived from the weights, fusion 1024, ...). */
void og_config_default(og_config* cfg);

/* ---- single queries -----------------------------------------------------------------
 * og_sssp_delta: Delta-stepping SSSP from src with eager bucket update and bucket
 * fusion (Section 3.3).  delta 0 = graph default.  dist_out: uint32[n], host or device
 * pointer; on OG_OK it holds every distance from src. */
int og_sssp_delta(og_graph* g, uint32_t src, uint32_t delta, uint32_t* dist_out,
                  void* stream);

/* og_wbfs: weighted BFS = SSSP with Delta = 1 (Section 6.1, "SSSP and wBFS"); every
 * weight must be >= 1 (OG_E_INVALID otherwise). */
int og_wbfs(og_graph* g, uint32_t src, uint32_t* dist_out, void* stream);

/* og_sssp_bellman_ford: the same distances as og_sssp_delta, computed by the unordered
 * Bellman-Ford baseline (OG_Q_BF); stats (may be NULL) receives its round count and
 * work counters for the ordered-vs-unordered comparison (Section 6, "unordered
 * GraphIt" rows). */
int og_sssp_bellman_ford(og_graph* g, uint32_t src, uint32_t* dist_out, og_stats* stats,
                         void* stream);

/* og_kcore: coreness of every vertex (Section 6.1, "k-core"): the largest k such that the
 * vertex belongs to a subgraph whose vertices all have degree >= k, computed by peeling
 * with buckets of vertex priorities (priority = degree at the start; the minimum
 * non-empty bucket is the level k; extracting a vertex lowers every neighbour whose
 * priority is above k by one, floored at k).  The graph must be symmetric (each
 * undirected edge stored in both directions); degrees and decrements count CSR entries,
 * so on a simple symmetric graph this is the usual coreness.  Weights are ignored.
 *   mode: OG_KCORE_LAZY -- lazy bucket update with the constant-sum (histogram)
 *         reduction of Section 5.1: one priority update and one bucket insertion per
 *         vertex and round; OG_KCORE_EAGER -- eager update (Section 3.2): one
 *         compare-and-swap decrement and one bucket insertion per edge.
 *   cfg: NULL or a config; used fields: expand_tile (frontier entries per claim, rounded
 *        up to 256; a small frontier gets smaller tiles), hub_degree (frontier vertices
 *        of at least this out-degree have their edges split over every warp of the grid;
 *        0 = 256 here, whatever the graph's stored schedule), blocks_per_sm (0 = 2 here),
 *        spin_limit_ns,
 *        arena_entries (vertex ids held by the
 *        256 materialised buckets; default 4n; a bucket that runs out of space is rebuilt
 *        by a scan at its level, so any size gives the same result).
 *   core_out: uint32[n], host or device.  stats (may be NULL): rounds = peeling rounds,
 *        fused_iters = levels extracted, items / stale = frontier entries / entries
 *        already extracted, relax = edges scanned, improved = priority updates,
 *        global_inserts = bucket insertions, redistributions = window refills,
 *        flushes = levels rebuilt by a scan, kernel_ns, and summed over CTAs:
 *        t_frontier_ns (peel phases), t_fused_ns (lazy apply phases), t_hub_ns (hub
 *        phases), t_barrier_ns.
 * Returns OG_E_INVALID for a bad mode or NULL output. */
#define OG_KCORE_LAZY 0u
#define OG_KCORE_EAGER 1u
int og_kcore(og_graph* g, uint32_t mode, const og_config* cfg, uint32_t* core_out,
             og_stats* stats, void* stream);

/* og_setcover: approximate unweighted set cover (Section 6.1, "Approximate Set Cover") of
 * the graph's set system: the set of vertex v is its out-adjacency list S_v (entries
 * counted with multiplicity), the universe is the union of all S_v, every set costs 1.
 * Sets are bucketed by their number D of uncovered elements on the integer ladder
 * t_0 = 1, t_(j+1) = t_j + max(1, floor(t_j * eps_ppm / 10^6)) (bucket j: t_j <= D <
 * t_(j+1)), and the highest non-empty bucket j is worked off in steps.  One step
 * (1) recounts D for every set of bucket j: D = 0 leaves, D < t_j moves to the bucket of
 * D, the others are active; (2) gives every uncovered element of an active set to the
 * active set of smallest priority that contains it; (3) adds to the cover every active
 * set that received at least ceil(t_j * 10^6 / (10^6 + eps_ppm)) elements -- a nearly
 * independent subset of the bucket -- and marks all of its elements covered; the others
 * stay in bucket j.  The result depends only on the graph, eps_ppm and the priorities.
 * Each chosen set covers at least (largest residual) / (1 + eps)^2 new elements, so the
 * cover is within (1 + eps)^2 H(largest set) of the optimum.
 *   eps_ppm: eps in millionths, 0 .. 1000000 (10000 = 0.01).
 *   priority: uint32[n], host or device, a permutation of 0 .. n-1 (random priorities
 *        give the method's expected number of steps per bucket); NULL = the identity.
 *   cfg: NULL or a config; used fields: hub_degree (a set with at least this many
 *        uncovered elements has them split over every warp of the grid; 0 = 32; clamped
 *        to [16, 2^26]), blocks_per_sm (0 = 4), spin_limit_ns.  The graph's stored
 *        schedule (tuned for Delta-stepping) is not used.
 *   step_out: uint32[n], host or device: the 1-based step in which set v joined the
 *        cover, 0 if it did not.
 *   stats (may be NULL): rounds = steps, fused_iters = buckets worked off, items = set
 *        visits, relax = elements scanned, improved = sets chosen, global_inserts = sets
 *        moved to a lower bucket, kernel_ns (including the set-up kernels), and summed
 *        over CTAs: t_frontier_ns (pack and claim phases), t_fused_ns (count, join and
 *        cover phases), t_hub_ns (bucket gathers), t_barrier_ns.
 * Requirements: every out-degree below 2^30, m below 2^32, at most 2^22 buckets.
 * Returns OG_E_INVALID for eps_ppm > 10^6, priorities that are not a permutation, a
 * graph beyond the requirements or a NULL output. */
int og_setcover(og_graph* g, uint32_t eps_ppm, const uint32_t* priority, const og_config* cfg,
                uint32_t* step_out, og_stats* stats, void* stream);

/* og_ppsp: point-to-point distance (Section 6.1, "PPSP"): Delta-stepping from src that
 * stops on entering bucket i with i * Delta >= the best dist(src, dst) found.
 * d_out: host uint32, receives dist(src, dst) (0xFFFFFFFF if unreachable). */
int og_ppsp(og_graph* g, uint32_t src, uint32_t dst, uint32_t delta, uint32_t* d_out,
            void* stream);

/* og_astar: A* (Section 6.1, "A* Search"): the bucket of a vertex is
 * floor((g + h) / Delta) with h = floor(100 * Euclidean distance to dst) from the
 * coordinates.  coords: float32[2n] (host or device) or NULL to use
 * og_graph_set_coords.  Same stop rule and output as og_ppsp.  If the heuristic proves
 * inconsistent on some edge the query keeps running until its buckets are empty, so the
 * result stays exact. */
int og_astar(og_graph* g, uint32_t src, uint32_t dst, const float* coords,
             uint32_t delta, uint32_t* d_out, void* stream);

/* Any query kind with an explicit schedule and counters (cfg and stats may be NULL).
 * dist_out (SSSP / wBFS: uint32[n], host or device; PPSP / A*: may be NULL) and d_out
 * (host uint32; PPSP / A*: dist(src, dst); may be NULL). */
int og_query_run(og_graph* g, const og_query* q, const og_config* cfg,
                 uint32_t* dist_out, uint32_t* d_out, og_stats* stats, void* stream);

/* ---- batches (many queries, one persistent launch) ------------------------------------
 * Runs nq queries concurrently: each has its own distance array and bucket ring, all
 * share one persistent kernel and its rounds.  q: host array of nq queries.
 * dist_out: uint32[nq * n] (host or device; query i at dist_out + i*n) or NULL when
 * only d_out is wanted.  d_out: host uint32[nq] (dist(src, dst) for PPSP / A*, 0 for
 * the others) or NULL. */
int og_batch_run(og_graph* g, const og_query* q, uint32_t nq, const og_config* cfg,
                 uint32_t* dist_out, uint32_t* d_out, og_stats* stats, void* stream);

/* ---- serving (continuous batching) -----------------------------------------------------
 * A server keeps the graph and up to max_slots queries resident.  og_server_submit
 * admits a PPSP / A* / SSSP query into a free slot (OG_E_BUSY if none).  og_server_step
 * runs one persistent launch of the barrier-free engine over every admitted query for at
 * most budget_us microseconds (0 = until all admitted queries finish); a query that is
 * not done keeps its state and continues in the next step, and queries admitted between
 * steps join the next launch.  og_server_poll returns finished queries (tag and
 * dist(src, dst)) and frees their slots.  Results do not depend on what else is in
 * flight.  max_slots = 0 sizes the slot count from free device memory. */
int og_server_create(og_graph* g, uint32_t max_slots, const og_config* cfg, void* stream,
                     og_server** out);
int og_server_submit(og_server* s, const og_query* q, uint64_t tag);
int og_server_step(og_server* s, uint32_t budget_us, uint32_t* n_active);
int og_server_poll(og_server* s, uint64_t* tags, uint32_t* d_out, uint32_t cap,
                   uint32_t* n_done);
int og_server_slots(const og_server* s, uint32_t* max_slots, uint32_t* n_free);
void og_server_free(og_server* s);

/* ---- autotuning (Section 5.3) ------------------------------------------------------------
 * Times the given sample queries under candidate schedules (Delta over powers of two in
 * [delta_lo, delta_hi], then the fusion threshold, then the expansion tile) and returns
 * the fastest in *out (also stored as the graph default).  kind: OG_Q_*.  srcs / dsts:
 * host arrays of nsample sources (and targets for PPSP / A*; NULL otherwise). */
int og_autotune(og_graph* g, uint32_t kind, const uint32_t* srcs, const uint32_t* dsts,
                uint32_t nsample, uint32_t delta_lo, uint32_t delta_hi, og_config* out);

/* The same search timed on a whole batch: queries (host array of nq, mixed kinds allowed;
 * a query's delta field should be 0 so that each candidate's Delta applies) run together
 * in the launches of og_batch_run under each candidate.  A batch needs its own schedule:
 * its CTA-local bins hold entries of many queries at once, so the best fusion threshold
 * and tile differ from those of one query.  Stores the winner as the graph default and
 * in *out.  OG_E_INVALID for an empty batch, a bad kind or a vertex id >= n. */
int og_autotune_batch(og_graph* g, const og_query* queries, uint32_t nq, uint32_t delta_lo,
                      uint32_t delta_hi, og_config* out);

/* ---- allocation-free variant -----------------------------------------------------------
 * og_sssp_delta_noalloc: the same Delta-stepping SSSP as og_sssp_delta for callers that
 * cannot allocate device memory -- code inside a host application whose allocator has
 * already claimed the GPU's memory, code on a path where cudaMalloc's implicit device
 * synchronisation is not acceptable, code that must not meet an out-of-memory error
 * after start-up.  It calls no cudaMalloc, cudaFree or other allocating routine.  The
 * paper has no counterpart; this is a deployment variant.
 *   offsets: device uint32[n+1]; edges: device uint32[2m] holding (neighbor, weight)
 *   pairs, the out-edges of u at pairs offsets[u] .. offsets[u+1]-1; dist_out: device
 *   uint32[n], receives every distance from src (0xFFFFFFFF = unreachable).  All three
 *   stay owned by the caller.
 *   The graph is checked on the device before the search: offsets[0] = 0,
 *   offsets[n] = m, offsets non-decreasing and every neighbor < n, else OG_E_INVALID
 *   (the search never runs on a malformed graph; the check reads offsets[0 .. n] and the
 *   m pairs only).  OG_E_INTERNAL reports a failed internal bounds check of the kernel
 *   (og_last_cuda_error has the details), OG_E_TIMEOUT a grid-barrier wait that gave up.
 *   Scratch: a 64 MiB static device array inside libog.so, reserved on every GPU that
 *   loads the library until the process exits.  n above 2^20 (1,048,576) vertices is
 *   rejected with OG_E_INVALID; a run whose buckets outgrow the array returns OG_E_ARENA
 *   (it never grows).
 *   The first call on a device, and the first after the device's context was re-created
 *   (cudaDeviceReset), does the set-up: it looks up the array's device address.  Make
 *   that first call before any stream capture.  Every call shares the array and clears
 *   its state words first, so calls that overlap on the GPU (other streams, other host
 *   threads) race: serialise them.  The call synchronises stream twice (after the graph
 *   check and at the end) before returning its status. */
int og_sssp_delta_noalloc(const uint32_t* offsets, const uint32_t* edges, uint32_t n,
                          uint64_t m, uint32_t src, uint32_t delta, uint32_t* dist_out,
                          void* stream);

/* ---- diagnostics ----------------------------------------------------------------------- */
/* The status every round-engine entry point derives from the error word its persistent
 * launch leaves behind (exposed so that the mapping can be checked without a GPU):
 * err = the launch's error bits (1 a bounded wait gave up, 2 a query's arena ran out, 4 a
 * distance saturated, 8 an internal bounds check failed); bad_code / bad_val / bad_aux =
 * the first failed check's code, value and context; arena_out = a query ran out of
 * bucket space where the arena cannot grow.  Precedence: OG_E_INTERNAL (the check's
 * details go to og_last_cuda_error), OG_E_TIMEOUT, OG_E_ARENA, OG_E_OVERFLOW, OG_OK. */
int og_launch_status(uint32_t err, uint32_t bad_code, uint32_t bad_val, uint32_t bad_aux,
                     uint32_t arena_out);
/* Memory round-trip probe (a measurement aid; the paper has no counterpart): ctas x
 * threads threads each follow a chain of hops dependent accesses through a fresh
 * device array of bytes bytes (a power of two, 4 KiB .. 16 GiB).  The chains visit
 * footprint / 128 lines of 128 bytes spread evenly over the array (footprint a power of
 * two, 4 KiB .. bytes; every hop lands far from the previous one): footprint = bytes
 * touches the whole array, a small footprint spread over a large array stays in L2 but
 * spans many pages.  *ns_per_hop receives the kernel time / hops, i.e. the round-trip
 * time of one access with that many chains in flight.  Each thread follows chains (1, 2,
 * 4, 8 or 16) independent chains, so ctas x threads x chains / *ns_per_hop is the rate
 * of independent random accesses.  mode 0: relaxed loads served by L2; 1: atomicMin
 * whose result is used (the array is left unchanged); 2: non-coherent loads through L1.
 * Allocates and frees its array; synchronises the device.  OG_E_INVALID for bad sizes
 * (threads a multiple of 32, at most 1024) or another chain count. */
int og_probe_chain(uint32_t mode, uint64_t bytes, uint64_t footprint, uint32_t ctas,
                   uint32_t threads, uint32_t chains, uint32_t hops, double* ns_per_hop);
const char* og_strerror(int code);
const char* og_last_cuda_error(void);
int og_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OG_H */
