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

#define IRGL_INF 0xFFFFFFFFu

/* The three operators of the worklist ForAll. */
typedef enum {
  IRGL_BFS = 0,  /* level assignment, Sec. 4.1 level-by-level BFS listing */
  IRGL_SSSP = 1, /* data-driven edge relaxation with atomicMin */
  IRGL_CC = 2    /* min-label propagation over a symmetric graph */
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
} irgl_tuning;

/* Per-call counters. */
typedef struct {
  uint32_t rounds;        /* kernel invocations (Iterate rounds) executed */
  uint32_t grid;          /* CTAs per launch */
  uint32_t cta_size;      /* threads per CTA */
  uint32_t launches;      /* CUDA kernel launches issued by the call */
  uint64_t edges_scanned; /* adjacency entries read, re-relaxations included */
  uint32_t last_out;      /* size of the final out-worklist (0 when Iterate drained it) */
  uint32_t reserved;
} irgl_stats;

/* ---------------------------------------------------------------- errors */

const char* irgl_last_error(void);
const char* irgl_status_string(irgl_status s);

/* ---------------------------------------------------------------- context
 * A context binds a device and a CUDA stream (cudaStream_t passed as void*;
 * NULL = the legacy default stream). It owns the device status block and the
 * scratch worklists/stamps that Iterate uses. One context must not be used
 * from two host threads at once. */
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

/* ---------------------------------------------------------------- test hooks
 * Fault injection on the host side only (no device fault is ever raised):
 *   key 1: barrier time limit in microseconds (0 = default 2 s)
 *   key 2: index of a CTA that skips its first grid-barrier arrival
 *          (-1 = none) -- the other CTAs then time out and report
 *          IRGL_ERR_BARRIER_TIMEOUT.
 *   key 3: override the capacity of the Iterate scratch worklists (0 = n). */
irgl_status irgl_debug_set(irgl_ctx* ctx, int key, int64_t value);

#ifdef __cplusplus
}
#endif
#endif /* IRGL_H */
