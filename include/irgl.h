/*
 * irgl.h -- C-ABI of libirgl.so: the worklist-driven ForAll over a CSR graph
 * that IrGL's Pipe / Iterate / ForAll constructs lower to (Pai & Pingali,
 * "Lowering IrGL to CUDA", arXiv 1607.05707), instantiated for data-driven
 * BFS, SSSP and connected components on one GB300 (sm_103a).
 *
 * Conventions for every call:
 *  - Plain pointers and sizes only. "device" pointers are CUDA global-memory
 *    addresses on the context's device; "host" pointers are ordinary (pinned
 *    or pageable) host memory.
 *  - Every call returns an irgl_status: 0 on success, a negative code on
 *    failure. No exception, abort or device trap crosses this boundary.
 *    irgl_last_error() returns a thread-local message for the last failure.
 *  - Calls are ordered on the context's CUDA stream (the caller's stream).
 *    Calls that must report a device-side outcome (iterate, invoke, size,
 *    batch_run, ...) synchronise on that stream before returning.
 *  - Objects created by the library (contexts, graphs, worklists, batches,
 *    servers) are owned by the library and freed by the matching *_destroy.
 *    State/result buffers passed in by the caller remain the caller's.
 *  - Values: uint32 levels, distances and labels; INF = 0xFFFFFFFF marks an
 *    unreachable vertex.
 */
#ifndef IRGL_H
#define IRGL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int irgl_status;

#define IRGL_OK 0
#define IRGL_ERR_INVALID_ARG (-1)     /* bad pointer, size, CSR structure or flag */
#define IRGL_ERR_OOM (-2)             /* device or host allocation failed */
#define IRGL_ERR_WL_OVERFLOW (-3)     /* a push found the out-worklist full */
#define IRGL_ERR_BARRIER_TIMEOUT (-4) /* a grid barrier wait hit its time limit */
#define IRGL_ERR_CUDA (-5)            /* a CUDA runtime call failed */
#define IRGL_ERR_NOT_SYMMETRIC (-6)   /* CC needs a graph loaded with IRGL_SYMMETRIC */
#define IRGL_ERR_ADMISSION (-7)       /* a query can never fit the server's memory budget */
#define IRGL_ERR_MAX_ROUNDS (-8)      /* Iterate stopped at max_rounds with work left */
#define IRGL_ERR_NOT_READY (-9)       /* polled result not finished yet */
#define IRGL_ERR_UNSUPPORTED (-10)    /* option not available for this kernel/mode */
#define IRGL_ERR_LOCK_TIMEOUT (-11)   /* an Atomic section's lock wait hit its time limit */
#define IRGL_ERR_TIME_LIMIT (-12)     /* a persistent launch ran past its wall-time limit (60 s by default;
                                         test hook key 7 sets it in ms): the work did not converge in time */

#define IRGL_INF 0xFFFFFFFFu

/* The three operators of the worklist ForAll. */
typedef enum {
  IRGL_BFS = 0,  /* level assignment, Sec. 4.1 level-by-level BFS listing */
  IRGL_SSSP = 1, /* data-driven edge relaxation with atomicMin */
  IRGL_CC = 2,   /* min-label propagation over a symmetric graph */
  IRGL_CC_JUMP = 3 /* same labels by min-hooking and pointer jumping (persistent Iterate only) */
} irgl_kernel;

/* How Iterate drives the kernel (Sec. 4.4 kernel invocations). */
typedef enum {
  IRGL_PER_LAUNCH = 0, /* host loop: one launch per invocation, host reads the out-worklist size */
  IRGL_PERSISTENT = 1  /* iteration outlining: one cooperative launch, grid barrier between rounds */
} irgl_mode;

/* ReduceAndReturn reductions (Sec. 3.5). */
typedef enum { IRGL_REDUCE_ANY = 0, IRGL_REDUCE_ALL = 1 } irgl_reduce;

/* irgl_csr_load flags */
#define IRGL_HOST_PTRS 0x0   /* row_ptr/col/w are host arrays: the library copies them */
#define IRGL_DEVICE_PTRS 0x1 /* device arrays: borrowed, must outlive the graph, 16-byte aligned */
#define IRGL_SYMMETRIC 0x2   /* every edge (u,v) has its reverse (v,u); required by CC */
#define IRGL_VALIDATE 0x4    /* full host validation (always done for host pointers) */
#define IRGL_IN_EDGES 0x8    /* host pointers only: also build and upload the in-edge CSR (transpose),
                                which direction-optimising BFS needs on a non-symmetric graph */

typedef struct irgl_ctx irgl_ctx;
typedef struct irgl_graph irgl_graph;
typedef struct irgl_worklist irgl_worklist;
typedef struct irgl_batch irgl_batch;
typedef struct irgl_server irgl_server;

/* Block-level launch choices (Sec. 4.4; chosen by irgl_autotune or defaults).
 * A zero field means "use the default". */
typedef struct {
  uint32_t cta_size;      /* threads per CTA: 128, 256, 512 or 1024 (FixedBlock kernels) */
  uint32_t warp_thresh;   /* out-degree >= warp_thresh: the list goes to one warp */
  uint32_t cta_thresh;    /* out-degree >= cta_thresh: the list goes to the whole CTA */
  uint32_t chunk;         /* worklist tiles (cta_size items each) taken per dynamic grab */
  uint32_t blocks_per_sm; /* persistent grid = min(this, occupancy) x SMs; 0 = occupancy */
  uint32_t max_blocks;    /* upper bound on the grid; 0 = none */
  uint32_t flags;         /* IRGL_TUNE_NO_SPLIT: persistent kernels keep long lists in the CTA bin
                             instead of splitting their edges over the whole grid */
  uint32_t delta;         /* persistent SSSP and CC only: near-far bucket width. Improvements to a
                             value (distance, label) >= the current limit wait on a far list until
                             the rounds below the limit drain; 0 = plain rounds (every improvement
                             is pushed). CC with delta = 1 floods the smallest label first, so
                             each vertex mostly takes its final label once. Batches and servers:
                             per-query near-far for their SSSP queries (below) */
  uint32_t defer_deg;     /* persistent SSSP with plain rounds (delta = 0, no sub-rounds): a popped
                             vertex with at least defer_deg out-edges whose distance is above the
                             smallest distance pushed for the round + defer_delta is pushed again
                             instead of expanded, so long lists are mostly scanned once, near their
                             final distance (0 = default 128; IRGL_TUNE_NO_DEFER turns it off) */
  uint32_t defer_delta;   /* that margin (0 = default 2) */
} irgl_tuning;

#define IRGL_TUNE_NO_SPLIT 0x1u
#define IRGL_TUNE_DIROPT 0x2u /* persistent BFS: rounds with a large frontier run bottom-up (every
                                 unvisited vertex looks for a parent among its in-edges); needs a
                                 symmetric graph or one loaded with IRGL_IN_EDGES, else ignored */
#define IRGL_TUNE_BITMAP 0x4u /* persistent BFS: a 1-bit-per-vertex copy of "level != INF", read
                                 through L1, filters edges to visited vertices before the level is
                                 read from L2 (off by default: slower on R-MAT scale 20, where the
                                 bit updates cost more than the L2 reads they save) */
#define IRGL_TUNE_LOCAL(k) (((uint32_t)(k) & 15u) << 8) /* persistent BFS and SSSP: after its tiles,
                                    each CTA expands the vertices it just discovered k more times (CTA-local
                                    sub-rounds, CTA barriers only) before flushing the rest to the
                                    out-worklist, so high-diameter graphs need fewer grid barriers; BFS
                                    then runs as unit-weight label-correcting relaxation (same levels).
                                    Pays on high-diameter graphs (meshes, grids), costs extra work on
                                    low-diameter ones (R-MAT); irgl_autotune tries k = 0, 4, 15.
                                    max_rounds is capped at 2^32 / (k + 1) - 1 global rounds.
                                    Ignored with IRGL_TUNE_DIROPT or IRGL_TUNE_NO_PACKED. */
#define IRGL_TUNE_NO_PACKED 0x8u /* persistent SSSP: keep distances and the dedup stamps in two
                                    arrays (by default one 64-bit word per vertex holds both,
                                    lowered by one atomicMin, and the distances are copied to the
                                    output at the end) */
#define IRGL_TUNE_NO_BCAST 0x10u /* persistent BFS, SSSP and CC: run small-frontier rounds like the
                                    others. By default, on a graph with an adjacency list at least as
                                    long as the smaller degree threshold (known when the CSR was loaded
                                    from host arrays or validated; else assumed), a round whose frontier
                                    has at most 768 items (and at most 2^20 / grid) skips the degree bins
                                    and the grid-wide list of long adjacency lists: every CTA reads the
                                    whole frontier, scans its degrees in shared memory and relaxes an
                                    equal share of its edges (one grid barrier per round instead of two) */
#define IRGL_TUNE_NO_SMEM 0x40u /* persistent BFS, SSSP and CC: use the grid-wide kernels even when
                                    the graph fits in one CTA's shared memory. By default a graph whose
                                    CSR, values and two worklists fit the device's opt-in shared memory
                                    per block (about 227 KB: some 4,000 vertices and 16,000 edges for
                                    SSSP) runs the whole Iterate in one CTA of 1024 threads with every
                                    access in shared memory and __syncthreads between the rounds; the
                                    schedule flags (sub-rounds, near-far, bottom-up rounds, bins) do
                                    not apply to it, and the stats report grid 1, CTA 1024 */
#define IRGL_TUNE_DENSE 0x80u /* persistent BFS, and SSSP on packed words (no near-far, no
                                    sub-rounds): a round whose frontier holds more than n / 8 items
                                    looks at every vertex in id order and pops those the previous
                                    round pushed (the round id in their packed word; for BFS, level
                                    = the round), so row offsets are read in order and the adjacency
                                    lists of neighbouring frontier vertices are neighbours in memory */
#define IRGL_TUNE_NO_DEFER 0x1000u /* persistent SSSP: expand every popped vertex (no deferred long lists) */
#define IRGL_TUNE_THREAD_BIN 0x20u /* all kernels: the lane that popped an adjacency list of 1..4 edges
                                    walks it itself (no per-edge search or shuffle) instead of the warp's
                                    scan bin dealing it out with the other short lists. Off by default:
                                    on R-MAT scale 20 the scan bin's denser strips win (SSSP 627 vs
                                    643 us per query, 256-instance batch 14.1 vs 13.5 GTEPS) */

/* Per-call counters. */
typedef struct {
  uint32_t rounds;        /* kernel invocations (Iterate rounds) executed */
  uint32_t grid;          /* CTAs per launch */
  uint32_t cta_size;      /* threads per CTA */
  uint32_t launches;      /* CUDA kernel launches issued by the call */
  uint64_t edges_scanned; /* adjacency entries read, re-relaxations included */
  uint32_t last_out;      /* size of the final out-worklist (0 when Iterate drained it) */
  float device_ms;        /* CUDA-event time of the call's launches, when the call measures it (else 0) */
} irgl_stats;

/* ---------------------------------------------------------------- errors */

const char* irgl_last_error(void);
const char* irgl_status_string(irgl_status s);

/* ---------------------------------------------------------------- context
 * A context binds a device and a CUDA stream (cudaStream_t passed as void*;
 * NULL = the legacy default stream). It owns the device status block and the
 * scratch worklists/stamps that Iterate uses. One context must not be used
 * from two host threads at once. Graphs, worklists, batches and servers made
 * on a context keep a pointer to it: destroy them before the context (their
 * destroy functions read it). */
irgl_status irgl_ctx_create(int device, void* cuda_stream, irgl_ctx** out);
irgl_status irgl_ctx_destroy(irgl_ctx* ctx);
irgl_status irgl_ctx_set_stream(irgl_ctx* ctx, void* cuda_stream);
/* Number of SMs and the default tuning for a kernel on this device. */
irgl_status irgl_ctx_info(irgl_ctx* ctx, uint32_t* sm_count, irgl_tuning* defaults);

/* ---------------------------------------------------------------- graphs
 * CSR graph: row_ptr[0..n] (uint32, row_ptr[0] = 0, non-decreasing,
 * row_ptr[n] = m), col[0..m) (uint32, < n), optional w[0..m) (int32 >= 0,
 * required by SSSP). Out-edges of u are col[row_ptr[u] .. row_ptr[u+1]),
 * i.e. graph.edges(n) of the BFS listing in Sec. 4.1.
 * Host pointers are validated and copied. Device pointers are borrowed
 * (validated only with IRGL_VALIDATE) and must be 16-byte aligned.
 * m must be < 2^32. SSSP additionally needs max(w) * (n - 1) < 2^32 - 1 so
 * that uint32 distance sums cannot wrap; otherwise SSSP returns INVALID_ARG. */
irgl_status irgl_csr_validate(uint32_t n, uint64_t m, const uint32_t* row_ptr, const uint32_t* col,
                              const int32_t* w, int flags);
irgl_status irgl_csr_load(irgl_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* row_ptr,
                          const uint32_t* col, const int32_t* w, int flags, irgl_graph** out);
irgl_status irgl_graph_destroy(irgl_graph* g);
irgl_status irgl_graph_info(const irgl_graph* g, uint32_t* n, uint64_t* m, int* flags);

/* ---------------------------------------------------------------- worklists
 * Device worklist of uint32 items (vertex ids) with a device tail counter
 * (Sec. 4.1 worklist mechanics; Sec. 4.2 WorklistInitializer /
 * WorklistInitializerFromArray). Pushes made by a kernel invocation land in
 * the out-worklist and are never popped by the same invocation
 * (bulk-synchronous worklists). */
irgl_status irgl_worklist_create(irgl_ctx* ctx, uint32_t capacity, irgl_worklist** out);
irgl_status irgl_worklist_destroy(irgl_worklist* wl);
/* Append k items from a host array (stream-ordered copy). */
irgl_status irgl_worklist_push(irgl_worklist* wl, const uint32_t* items_host, uint32_t k);
/* Append the items 0..k-1 (e.g. "all vertices" for CC). */
irgl_status irgl_worklist_push_range(irgl_worklist* wl, uint32_t k);
irgl_status irgl_worklist_clear(irgl_worklist* wl);
/* Current size (synchronises). */
irgl_status irgl_worklist_size(irgl_worklist* wl, uint32_t* out);
/* Copy up to cap items to a host array; *n receives the size (synchronises). */
irgl_status irgl_worklist_read(irgl_worklist* wl, uint32_t* items_host, uint32_t cap, uint32_t* n);

/* ---------------------------------------------------------------- kernels
 * irgl_init_state writes the initial values of an Iterate into a caller-owned
 * device array state[0..n): BFS/SSSP: INF everywhere, 0 at every item of
 * `initial` (Initial[src] in the BFS listing); CC: state[v] = v.
 * `initial` may be NULL for CC. */
irgl_status irgl_init_state(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial,
                            uint32_t* state_dev);

/* Invoke (Table 1, Sec. 4.4): one kernel invocation. Every item of `in` is
 * popped (ForAll over in, Sec. 3.1); each out-edge is relaxed; every vertex
 * whose value changed is pushed to `out` (cooperative conversion). `in` is
 * empty afterwards. `level` is the BFS LEVEL (a vertex first reached gets
 * level + 1); it is ignored by SSSP/CC. *result receives the ReduceAndReturn
 * value over the popped items of "this item pushed at least one vertex":
 * Any = some item did, All = every item did (All over no items = 1,
 * Any over no items = 0). result may be NULL. */
irgl_status irgl_invoke(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* in, irgl_worklist* out,
                        uint32_t* state_dev, uint32_t level, irgl_reduce r, const irgl_tuning* t, int* result);

/* Iterate ... Initial[...] until the worklist is empty (Table 1; Sec. 4.2-4.4).
 * Writes the initial values into state_dev (as irgl_init_state), then runs
 * rounds: pop the in-worklist, push to the out-worklist, swap, LEVEL++, until
 * a round pushes nothing. `initial` holds the start items (it is read, not
 * modified); NULL means all vertices (CC). max_rounds is the Or-ed
 * extra_cond: 0 = none; reaching it with work left returns
 * IRGL_ERR_MAX_ROUNDS (state then holds a partial result).
 * Mode IRGL_PERSISTENT runs every round inside one cooperative launch with a
 * bounded grid barrier between rounds (iteration outlining,
 * SyncRunningThreads, Sec. 3.4); IRGL_PER_LAUNCH launches once per round and
 * reads the out-worklist size on the host. t may be NULL (defaults).
 * stats may be NULL. Synchronises on the stream before returning. */
irgl_status irgl_iterate(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial,
                         uint32_t* state_dev, irgl_mode mode, const irgl_tuning* t, uint32_t max_rounds,
                         irgl_stats* stats);

/* Asynchronous persistent Iterate: enqueues the same single cooperative launch
 * as irgl_iterate(..., IRGL_PERSISTENT, ...) on the context's stream and
 * returns without waiting. The caller must not reuse the context's scratch
 * state from another stream meanwhile; the outcome (device error code,
 * rounds, edges) is collected by irgl_ctx_sync. Several asynchronous calls on
 * one context run back to back in stream order; irgl_ctx_sync then reports
 * the first device error, the rounds of the last launch and the summed edges. */
irgl_status irgl_iterate_async(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial,
                               uint32_t* state_dev, const irgl_tuning* t, uint32_t max_rounds);
/* Wait for the context's stream and report the device status accumulated since
 * the last synchronising call. stats may be NULL. */
irgl_status irgl_ctx_sync(irgl_ctx* ctx, irgl_stats* stats);

/* Convenience form of Iterate for one query: sources from a host array
 * (nsrc may be 0 for CC); the result goes to `state`, which is a device array
 * (state_on_host = 0) or a host array of n entries (state_on_host = 1, the
 * library copies the result back before returning). */
irgl_status irgl_run(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, const uint32_t* srcs_host, uint32_t nsrc,
                     uint32_t* state, int state_on_host, irgl_mode mode, const irgl_tuning* t,
                     uint32_t max_rounds, irgl_stats* stats);

/* ---------------------------------------------------------------- tracing
 * Per-round trace of persistent launches on this context (Iterate and batch):
 * after each round's grid barrier one thread records the globaltimer time
 * (ns), the round's in-worklist size and its out-worklist size. Record 0 is
 * the end of the prologue (state initialisation); for single-query Iterates
 * its out field holds the prologue's duration in ns (from the kernel's start).
 * Record rounds + 1, when the capacity has room for it, is the end of the
 * epilogue (results written), marked with in = out = 0xFFFFFFFF.
 * irgl_trace_enable(ctx, 0) switches tracing off; enabling allocates 16 bytes
 * per round of capacity, plus 64 for the phase records below. irgl_trace_read
 * copies min(cap, capacity, rounds of the last launch + 2) records. */
irgl_status irgl_trace_enable(irgl_ctx* ctx, uint32_t max_rounds);
irgl_status irgl_trace_read(irgl_ctx* ctx, uint64_t* t_ns, uint32_t* in_n, uint32_t* out_n, uint32_t cap,
                            uint32_t* nrec);
/* Phase records of the last single-query persistent Iterate (grid-wide kernel),
 * one per round, 8 words each (globaltimer ns): [0] ~(earliest end of the
 * round's first phase over all CTAs), [1] its latest end, [2] the time CTA 0
 * left the first grid barrier, [3] the big list published there ((entries << 40)
 * | edges; 0 = none), [4] ~(earliest end of the big phase), [5] its latest end,
 * [6] the time CTA 0 left the second barrier, [7] 0. Copies min(cap, capacity,
 * rounds) records into `words` (cap * 8 entries). */
irgl_status irgl_trace_phases(irgl_ctx* ctx, uint64_t* words, uint32_t cap, uint32_t* nrec);

/* ---------------------------------------------------------------- block sizes
 * Sec. 4.4 rule for an outlined Pipe: the control kernel's block size must be
 * in T_control = intersection over the Pipe's kernels of the block sizes each
 * accepts. masks[i] is kernel i's set as a bitmask (bit b = CTA size 128 << b,
 * b = 0..3). An empty intersection returns IRGL_ERR_UNSUPPORTED (no
 * outlining); otherwise *out = preferred if it is in the set, else the
 * highest size in the set (preferred = 0: always the highest). */
irgl_status irgl_control_cta(const uint32_t* masks, uint32_t count, uint32_t preferred, uint32_t* out);

/* ---------------------------------------------------------------- autotuning
 * Coordinate descent over the irgl_tuning fields (CTA size, CTA and warp
 * degree thresholds, chunk, CTAs per SM, total grid max_blocks in {full, 1, 2,
 * 8, 32, SMs}; for BFS and SSSP also the CTA-local sub-rounds, flags =
 * IRGL_TUNE_LOCAL(0, 4 or 15), and for BFS on a graph with in-edges (or a
 * symmetric one) IRGL_TUNE_DIROPT; for SSSP also the near-far delta), each
 * candidate timed as the median
 * CUDA-event time of `reps` persistent Iterate runs of kernel k from the given
 * sources on graph g (after one warm-up run). *best receives the fastest
 * tuning and *best_ms its time. Results do not depend on the tuning (the
 * fixed point is unique); only the time does. */
irgl_status irgl_autotune(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, const uint32_t* srcs_host, uint32_t nsrc,
                          uint32_t reps, irgl_tuning* best, float* best_ms);

/* ---------------------------------------------------------------- batching
 * A batch runs many independent queries ("instances": a graph, a kernel and
 * its sources) in one persistent cooperative launch per wave (below). Each instance owns a
 * range of a device state arena (its result), its worklist items travel on the
 * shared double-buffered worklist as arena offsets that a sorted offset table
 * maps back to the instance, and its termination flag is the round of its
 * last push. Instances may differ in graph, size and kernel; the CTA size is
 * chosen by the T_control rule above, with the tuning's CTA size (default 128)
 * as the preference. irgl_batch_prepare allocates the arena (20 bytes per
 * instance vertex: a 64-bit word holding the value and the id of the round
 * that last lowered it, the u32 result and two worklist entries; 16 bytes with
 * IRGL_TUNE_NO_PACKED, which keeps values and stamps in two arrays; 32 bytes
 * with near-far), uploads
 * the descriptors and, with use_cuda_graph = 1, captures the whole launch
 * sequence (admission kernels + persistent kernel + result extraction) in a
 * CUDA graph that irgl_batch_launch replays (if the
 * capture fails the sequence is launched directly; irgl_batch_info tells).
 * Every launch recomputes all instances from their sources.
 * Queries are added before prepare; query ids are 0, 1, ... in add order.
 * Near-far (tuning delta != 0, packed words): each SSSP query has its own
 * limit, delta at admission. A popped item whose distance is at or above its
 * query's limit is not expanded; it waits on a far list, which every round
 * looks at once: items its query's limit has passed go back onto the
 * out-worklist, the rest stay. A query's limit rises by delta after every
 * round in which it pushed nothing onto the out-worklist. Results are the
 * same; only the edges scanned and the rounds change (64 SSSP queries on a
 * 1024^2 weighted mesh scan about 40 times its edges each with plain rounds). */
irgl_status irgl_batch_create(irgl_ctx* ctx, uint32_t max_queries /* <= 1024 */, irgl_batch** out);
irgl_status irgl_batch_destroy(irgl_batch* b);
irgl_status irgl_batch_add(irgl_batch* b, irgl_graph* g, irgl_kernel k, const uint32_t* srcs_host, uint32_t nsrc,
                           uint32_t* query_id);
irgl_status irgl_batch_prepare(irgl_batch* b, const irgl_tuning* t, int use_cuda_graph);
/* Waves: prepare splits the queries, in add order, into consecutive groups
 * whose packed state (8 bytes per vertex) fits in `bytes`; a run admits and
 * iterates one group after another (one persistent launch each, all in the
 * same CUDA graph), so the random state accesses of the active group hit L2
 * instead of DRAM. This pays for low-diameter queries whose rounds are
 * bandwidth-bound (256 R-MAT instances: 8.5 -> 6.6 ms with L2 / 2) and costs
 * for high-diameter ones, whose rounds are latency-bound and which then run
 * their rounds wave after wave (64 BFS on a 1024^2 grid: 10 waves, 10x the
 * rounds); irgl_batch_autotune measures the choice. 0 (the default) or
 * UINT64_MAX = one wave (every query active at once). A query larger than
 * `bytes` is a wave of its own. Takes effect at the next irgl_batch_prepare.
 * The per-query rounds count the rounds of the query's own wave;
 * stats->rounds sums the waves. */
irgl_status irgl_batch_set_wave_bytes(irgl_batch* b, uint64_t bytes);
irgl_status irgl_batch_waves(irgl_batch* b, uint32_t* waves);
/* Enqueue one run (events bracket it); irgl_batch_sync waits, checks the device
 * status and fills stats (device_ms = event time of the run). */
irgl_status irgl_batch_launch(irgl_batch* b);
irgl_status irgl_batch_sync(irgl_batch* b, irgl_stats* stats);
irgl_status irgl_batch_run(irgl_batch* b, irgl_stats* stats); /* launch + sync */
irgl_status irgl_batch_info(irgl_batch* b, uint32_t* nqueries, uint32_t* grid, uint32_t* cta_size, int* graph_captured,
                            uint64_t* arena_entries);
/* Device pointer to query q's result (n entries, valid until the next launch or
 * destroy) and the rounds that query was active (from its termination flag). */
irgl_status irgl_batch_result(irgl_batch* b, uint32_t query_id, uint32_t** state_dev, uint32_t* n, uint32_t* rounds);
irgl_status irgl_batch_copy_result(irgl_batch* b, uint32_t query_id, uint32_t* host_out);
/* Every query's result in one transfer: host_out (arena_entries values, see
 * irgl_batch_info) receives the queries' results back to back in add order
 * (query q at the sum of n over the queries added before it). Pinned host
 * memory makes the copy asynchronous to the CPU; it completes before return. */
irgl_status irgl_batch_copy_results(irgl_batch* b, uint32_t* host_out);
/* Autotune a prepared batch: the same coordinate descent, each candidate timed
 * as the median event time of `reps` whole-batch runs (the batch is re-prepared
 * per candidate, with the CUDA-graph choice it was prepared with; the
 * near-far delta too when the batch holds SSSP queries), then the wave budget (a quarter, half or all of the L2, or one wave; see
 * irgl_batch_set_wave_bytes). The batch is left prepared with the best tuning
 * and budget (irgl_batch_waves tells the wave count). */
irgl_status irgl_batch_autotune(irgl_batch* b, uint32_t reps, irgl_tuning* best, float* best_ms);

/* ---------------------------------------------------------------- serving
 * Continuous batching server for BFS/SSSP queries against device-resident
 * graphs. A worker thread admits queued queries in arrival order while a
 * slot is free and the query's state fits the device arena (20 bytes per
 * vertex of its graph, 16 with IRGL_TUNE_NO_PACKED, 32 with near-far as in
 * batches (tuning delta); first-fit), launches
 * epochs of the batched persistent
 * kernel (at most epoch_rounds rounds over every active query), and retires
 * the queries that finished: their result is copied to the caller's host
 * buffer (if one was given) on a second stream while later epochs run, and the
 * query is reported done (irgl_server_poll) once its copy has landed; then its
 * memory and slot are reused. The worker keeps two epochs in flight (it reads
 * one back while the next runs). Queries
 * that arrive while others run join the next epoch; their work overlaps on
 * the device. Submission is thread-safe. */
typedef struct {
  uint64_t arena_bytes;   /* device budget for query state; 0 = 40% of the free HBM at creation */
  uint32_t max_slots;     /* concurrently active queries, 1..1024 */
  uint32_t epoch_rounds;  /* rounds per persistent launch */
  uint32_t count_edges;   /* 1: count out-edges of reached vertices per query (for GTEPS) */
  uint32_t solo_min_n;    /* queries on graphs of at least this many vertices run alone, one
                             persistent launch each between epochs, instead of sharing the batch
                             arena (their state would evict the other queries' from L2); 0 = graphs
                             whose state and stamps exceed half the L2, 0xFFFFFFFF = never */
  irgl_tuning tuning;     /* launch choices of the batched kernel (zeros = defaults) */
} irgl_server_config;

typedef struct {
  int32_t status;     /* IRGL_OK or the error that ended the query */
  uint32_t rounds;    /* rounds the query was active */
  double latency_s;   /* submission -> result in the host buffer */
  double t_submit_s;  /* host steady-clock times */
  double t_done_s;
  uint64_t edges;     /* out-edges of reached vertices (count_edges = 1) */
} irgl_query_info;

typedef struct {
  uint64_t submitted, completed, rejected, epochs, rounds, edges;
  double busy_s;      /* worker time spent in epochs */
  double kernel_s;    /* CUDA-event time of the epoch kernels */
  uint32_t active, queued;
  uint64_t arena_entries;
  uint32_t grid, cta_size;
  uint64_t solo;      /* completed queries that ran alone (solo_min_n) */
} irgl_server_counters;

irgl_status irgl_server_create(irgl_ctx* ctx, const irgl_server_config* cfg, irgl_server** out);
/* host_out: NULL or a host array of the graph's n entries that receives the
 * result (it must stay valid until the query completes). Returns
 * IRGL_ERR_ADMISSION if the query can never fit the arena. */
irgl_status irgl_server_submit(irgl_server* s, irgl_graph* g, irgl_kernel k, uint32_t src, uint32_t* host_out,
                               uint64_t* ticket);
/* IRGL_OK and *info when finished, IRGL_ERR_NOT_READY otherwise. */
irgl_status irgl_server_poll(irgl_server* s, uint64_t ticket, irgl_query_info* info);
/* Wait until every submitted query finished (IRGL_ERR_NOT_READY on timeout). */
irgl_status irgl_server_drain(irgl_server* s, uint32_t timeout_ms);
irgl_status irgl_server_stats(irgl_server* s, irgl_server_counters* out);
irgl_status irgl_server_destroy(irgl_server* s);

/* ---------------------------------------------------------------- no-allocation entry point
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory at all: for instance a plugin whose host
 * application's allocator reserves the whole device at start-up, or a
 * latency-critical loop that cannot take the implicit device synchronisation
 * a cudaMalloc may bring. It runs the persistent BFS Iterate from one source
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *   device, cuda_stream: the GPU and the stream (cudaStream_t as void*) to run on;
 *                        a non-null stream of another device is IRGL_ERR_INVALID_ARG
 *   n, m, row_ptr, col:  the caller's device CSR (as irgl_csr_load; col 16-byte aligned)
 *   src:                 source vertex, < n
 *   level:               caller's device array of n uint32 levels (INF = unreachable)
 *   rounds:              optional host out: Iterate rounds executed
 * Scratch (status block, two worklists, big list) lives in one file-scope
 * device array of about 9.6 MiB that every GPU loading the library keeps until
 * the process exits; n is limited to 1,048,576 vertices (IRGL_ERR_INVALID_ARG
 * beyond, before any GPU work). Every call shares that array and it keeps the
 * last call's contents (each call clears its counters), so calls whose GPU work
 * overlaps race and give wrong results. The first call on a device looks up
 * the array's address with that device current. Every call copies its source
 * from host memory, reads its status back and synchronises cuda_stream before
 * returning, so it cannot be captured into a CUDA graph. */
irgl_status irgl_bfs_noalloc(int device, void* cuda_stream, uint32_t n, uint64_t m, const uint32_t* row_ptr,
                             const uint32_t* col, uint32_t src, uint32_t* level, uint32_t* rounds);

/* ---------------------------------------------------------------- minimum spanning forest
 * Boruvka's algorithm (Sec. 3.3, Listing "Find-Minimum-Cross-Component-Edge")
 * as a Pipe of three kernels (Sec. 4.3): find_min (each vertex's lightest
 * cross-component edge, merged into its component's record inside an Atomic
 * section on the component's lock), link (record each component's edge, hook
 * the component to the other one), and jump (pointer jumping until no vertex
 * changes, Iterate Until !Any). The Pipe repeats until no component has a
 * cross edge. Edges are ordered by the key (w, min(u,v), max(u,v)), so the
 * forest is unique; parallel copies of an edge (same key) are interchangeable.
 *
 * Lock forms of the Atomic section (Sec. 3.3):
 *   IRGL_LOCK_BLOCKING: atomicCAS retry loop, divergence-safe (the attempt and
 *     the critical section share one branch);
 *   IRGL_LOCK_TICKET:   ticket lock;
 *   IRGL_LOCK_RETRY:    one attempt (Atomic ... Else): a vertex that misses the
 *     lock goes to the retry worklist, and find_min is invoked again on that
 *     list (in and retry swapped, out kept; Sec. 4.3) with contiguous blocks of
 *     items per thread (Retry Backoff) until the list is empty.
 * Lock waits (and one find_min's retries) are bounded by half the context's
 * barrier time limit (1 s by default; test hook key 1) and end the call with
 * IRGL_ERR_LOCK_TIMEOUT. Test hook key 6 makes one component's lock start
 * held (never released).
 *
 * mode: IRGL_PERSISTENT outlines the whole Pipe into one cooperative launch
 *   whose CTA size is chosen by the T_control rule (irgl_control_cta) over the
 *   three kernels; IRGL_PER_LAUNCH launches each kernel invocation from a host
 *   loop that reads the counters in between.
 * g: loaded with IRGL_SYMMETRIC and weights (IRGL_ERR_NOT_SYMMETRIC,
 *   IRGL_ERR_INVALID_ARG otherwise).
 * out_edges: cap >= n - 1 uint32 CSR edge indices (device memory, or host
 *   memory when out_on_host != 0), written in no particular order: one
 *   direction (u -> v, either) of each forest edge. t: cta_size preference,
 *   blocks_per_sm and max_blocks are used; NULL = defaults. stats: optional.
 * Synchronises on the context's stream before returning. */
typedef enum { IRGL_LOCK_BLOCKING = 0, IRGL_LOCK_TICKET = 1, IRGL_LOCK_RETRY = 2 } irgl_lock;

typedef struct {
  uint32_t edges;        /* forest edges written to out_edges */
  uint32_t iterations;   /* Boruvka iterations (Pipe repetitions) */
  uint64_t weight;       /* sum of the forest edges' weights */
  uint32_t invocations;  /* kernel invocations inside the Pipe (find_min, retries, link, jump passes) */
  uint32_t retries;      /* vertices pushed to the retry worklist (IRGL_LOCK_RETRY) */
  uint32_t locks;        /* lock acquisitions (the rest passed the pre-lock weight test) */
  uint32_t launches;     /* kernel launches */
  uint32_t grid;
  uint32_t cta_size;
  float device_ms;       /* event time of the whole call on its stream */
  uint32_t reserved;
} irgl_msf_stats;

irgl_status irgl_msf(irgl_ctx* ctx, irgl_graph* g, irgl_mode mode, irgl_lock lock, uint32_t* out_edges, uint32_t cap,
                     int out_on_host, const irgl_tuning* t, irgl_msf_stats* stats);

/* ---------------------------------------------------------------- test hooks
 * Fault injection on the host side only (no device fault is ever raised):
 *   key 1: barrier time limit in microseconds (0 = default 2 s)
 *   key 2: index of a CTA that skips its first grid-barrier arrival
 *          (-1 = none) -- the other CTAs then time out and report
 *          IRGL_ERR_BARRIER_TIMEOUT.
 *   key 3: override the capacity of the Iterate scratch worklists (0 = n).
 *   key 4: cap the big list of persistent Iterate launches (0 = default), so
 *          long lists beyond the cap take the warp-bin path.
 *   key 5: 1 = direction-optimising BFS runs every round bottom-up.
 *   key 6: minimum spanning forest: the lock of this component (vertex id;
 *          -1 = none) starts held and is never released, so its waits run
 *          out and the call returns IRGL_ERR_LOCK_TIMEOUT.
 *   key 7: wall-time limit of persistent Iterate, batch and server launches in
 *          milliseconds (0 = default 60 s); a launch past it stops at its next
 *          round with IRGL_ERR_TIME_LIMIT (batches and servers read it when they
 *          are prepared or created).
 *   key 8: 1 = persistent Iterate, batch and server rounds whose frontier is
 *          smaller than one tile per CTA keep it in static per-CTA spans
 *          instead of spreading it over every CTA (batches and servers read it
 *          when they are prepared or run an epoch). */
irgl_status irgl_debug_set(irgl_ctx* ctx, int key, int64_t value);

#ifdef __cplusplus
}
#endif
#endif /* IRGL_H */
