// Device side of the worklist ForAll (sm_103a).
//
// One round ("kernel invocation") pops every item of the in-worklist
// (ForAll(wlidx In wl), Sec. 3.1), walks the out-edges of the popped vertex
// (the nested ForAll(e In graph.edges(n)) of the Sec. 4.1 BFS listing),
// applies the operator and pushes every vertex whose value changed onto the
// out-worklist (pushes go to `out`, pops come from `in`: Sec. 4.2).
//
//  * Nested edge parallelism by degree: a popped vertex's adjacency list is
//    handled by the whole CTA (degree >= cta_thresh), by one warp
//    (>= warp_thresh) or, for short lists, by a CTA-wide scan that deals the
//    edges of all short lists of the tile out to the threads one edge each.
//    CTA and warp lists are read with 16-byte vector loads after an alignment
//    peel.
//  * Cooperative conversion of pushes: each warp aggregates its pushes with
//    ballot/popc (or a shuffle scan for multi-item pushes), reserves space in a
//    shared-memory stage with one shared atomic, and the CTA flushes the stage
//    with one global atomicAdd on the out-worklist tail and coalesced stores.
//  * Iteration outlining: the persistent kernel runs all rounds in one
//    cooperative launch, separated by a grid barrier (SyncRunningThreads,
//    Sec. 3.4) whose spin is bounded in time; a timeout sets an error code
//    and every CTA returns.
//  * ReduceAndReturn Any/All (Sec. 3.5): per-thread values are aggregated per
//    CTA with __syncthreads_or and folded in with one atomic per CTA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace irgl {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Operator ids (OP_RUNTIME: taken per query from the batch descriptor).
// OP_BFSR: BFS levels by label-correcting relaxation (SSSP with unit weights:
// a popped vertex's current level + 1), the form the CTA-local sub-rounds need,
// since a vertex can be reached there before its level is final.
enum : uint32_t { OP_BFS = 0, OP_SSSP = 1, OP_CC = 2, OP_RUNTIME = 3, OP_CCJ = 4, OP_BFSR = 5 };

// Operators whose values can be scheduled near-far (smallest first): SSSP
// distances and min-label CC labels.
template <uint32_t OP>
constexpr bool kNearFarOp = OP == OP_SSSP || OP == OP_CC;

// Operators that can keep (value, round id) in one 64-bit word per vertex:
// single-graph SSSP, and every query of the batched kernel.
template <uint32_t OP>
constexpr bool kPackedOp = OP == OP_SSSP || OP == OP_RUNTIME || OP == OP_BFSR;
enum : int { RED_NONE = 0, RED_ANY = 1, RED_ALL = 2 };
// Device error codes (first one wins).
enum : uint32_t {
  DERR_NONE = 0,
  DERR_WL_OVERFLOW = 1,
  DERR_BARRIER_TIMEOUT = 2,
  DERR_MAX_ROUNDS = 3,
  DERR_BAD_ITEM = 4,
  DERR_LOCK_TIMEOUT = 5,   // an Atomic section's lock wait hit the time limit
  DERR_MSF_ITERS = 6,      // more Boruvka iterations than a forest can need
  DERR_TIME_LIMIT = 7,     // a persistent launch ran past its wall-time limit
};

// Device status block. Each contended family sits on its own 128-byte line.
// Invariant between launches: arrive, exit_count, tail[], grab[], rel, qmask, qnear, bfar_tail,
// big_ctr, any_true and any_false are 0 (every kernel restores them on a
// clean exit; the host clears the block after an error).
constexpr uint32_t kMaxGrid = 2048;  // CTAs of a persistent launch (16-bit arrival count)

struct alignas(128) DevStatus {
  // grid-barrier arrivals of the current barrier: (pushes << 32) | (CTAs that
  // appended to the big list << 16) | arrivals; reset by each barrier's releaser
  unsigned long long arrive;
  uint32_t exit_count;
  uint32_t pad0[29];
  uint32_t tail[4];
  uint32_t pad1[28];
  uint32_t grab[4];
  uint32_t pad2[28];
  uint32_t err;
  uint32_t err_info;
  uint32_t epoch;     // dedup stamp base; advanced past every stamp a launch used
  uint32_t rounds;    // rounds executed by the last Iterate launch
  uint32_t any_true;  // ReduceAndReturn accumulators
  uint32_t any_false;
  uint32_t result;    // last ReduceAndReturn value
  uint32_t last_out;  // out-worklist size when a persistent launch stopped
  unsigned long long edges;  // adjacency entries scanned (accumulates until the host clears it)
  uint32_t pad3[22];
  // grid-barrier release word: (generation << 40) | (flags << 32) | published out-worklist size,
  // flags = device error code (bits 0..6) | big-list-pending (bit 7)
  unsigned long long rel;
  uint32_t pad4[30];
  // big list of the current round: (entries << 40) | edges, appended with one atomic per tile
  unsigned long long big_ctr;
  unsigned long long big_pub;  // copy published by the barrier's releaser
  uint32_t pad5[28];
  // per-round bitmaps of the batched queries that pushed (folded into qlast)
  uint32_t qmask[2][32];
  // near-far (SSSP, CC): sizes of the two far lists and the smallest value pushed to each
  uint32_t far_tail[2];
  uint32_t far_min[2];
  uint32_t pad6[4];
  // direction-optimising BFS: out-edges of the vertices each round pushed (triple-buffered)
  unsigned long long mf[3];
  // SSSP deferred expansion: ~(smallest distance pushed) per round (triple-buffered; 0 = none)
  uint32_t pmin[3];
  uint32_t pad7[15];
  // batched near-far: per-round bitmaps of the queries (by slot) that pushed to
  // the out-worklist, and the sizes of the far lists (both triple-buffered)
  uint32_t qnear[3][32];
  uint32_t bfar_tail[3];
  // direction-optimising BFS: sizes of the lists of vertices the bottom-up
  // rounds left open (triple-buffered by bottom-up round)
  uint32_t bu_n[3];
  uint32_t pad8[26];
};
static_assert(sizeof(DevStatus) == 1664, "status layout");

// Long adjacency lists of a round (degree >= cta_thresh) are not walked by the
// CTA that popped them: they go to a grid-wide list and, after a barrier, every
// CTA walks an equal share of their concatenated edges.
struct BigList {
  uint4* e;                  // {beg, end, val, q}
  unsigned long long* off;   // first edge of each entry in the concatenation (increasing)
  uint32_t cap;              // entries; 0 = disabled (lists stay in the CTA bin)
};
constexpr unsigned long long kBigEdgeMask = (1ull << 40) - 1;
constexpr uint32_t kRelBigFlag = 0x80u;

// __launch_bounds__ minimum CTAs per SM: 1024 resident threads per SM, so the
// register allocator may use up to 64 registers per thread.
template <int CTA>
struct MinBlocks {
  static constexpr int value = CTA >= 1024 ? 1 : 1024 / CTA;
};

// Launch tuning visible to the device.
struct Tune {
  uint32_t warp_thresh;
  uint32_t cta_thresh;
  uint32_t chunk;
  uint32_t thread_max;  // lists of 1..thread_max edges are walked by the lane that popped them (0 = none)
};
constexpr uint32_t kThreadBin = 4;

// Single-graph kernel parameters.
struct KParams {
  const uint32_t* __restrict__ row_ptr;
  const uint32_t* __restrict__ col;
  const int32_t* __restrict__ w;
  uint32_t n;
  uint32_t* state;
  uint32_t* stamp;
  const uint32_t* init_items;  // round-0 input; nullptr = items 0..n-1
  const uint32_t* init_count;  // device size of init_items; nullptr = n
  uint32_t init_cap;           // capacity of init_items (its size is clamped to it)
  uint32_t* items[2];          // scratch worklists (persistent mode)
  uint32_t cap;                // capacity of each scratch worklist
  DevStatus* st;
  Tune tn;
  uint32_t max_rounds;         // 0xFFFFFFFF = none
  unsigned long long timeout_ns;
  unsigned long long time_limit_ns;  // wall time after which the launch stops with DERR_TIME_LIMIT (0 = none)
  int skip_cta;                // test hook: this CTA never reaches the first barrier
  int init_state;              // write the Iterate initial values in the prologue
  unsigned long long* trace;   // optional per-round trace: {end time ns, (in_n << 32) | out_n}
  // optional per-round phase records (trace_cap records of kPhaseWords words; see trace_phase)
  unsigned long long* trace_ph;
  uint32_t trace_cap;          // rounds the trace can hold
  BigList big;
  // near-far schedule, SSSP and CC (delta = 0: off)
  uint32_t* far[2];
  uint32_t far_cap;
  uint32_t* far_stamp;
  uint32_t delta;
  // direction-optimising BFS (diropt = 0: top-down rounds only)
  const uint32_t* in_row_ptr;
  const uint32_t* in_col;
  uint32_t diropt;
  unsigned long long m_total;
  // BFS visited bitmap (bit v set => level[v] != INF), ceil(n / 32) words,
  // cleared in the prologue; nullptr = off
  uint32_t* vis;
  // SSSP: per vertex (dist << 32) | id of the round that last lowered it, n
  // words, filled in the prologue and copied out to `state` at the end;
  // nullptr = dist in `state` and dedup stamps in `stamp`
  unsigned long long* ds;
  // CTA-local sub-rounds per round (packed relaxations only; 0 = off): after
  // its tiles a CTA expands what it pushed to its shared-memory stage, up to
  // this many more times, before flushing the rest to the out-worklist
  uint32_t local_rounds;
  // direction-optimising BFS: two lists (n entries each) of the vertices a
  // bottom-up round left unvisited although they have in-edges; the next
  // bottom-up round looks at those only (nullptr: every vertex, every time)
  uint32_t* bu_list[2];
  // rounds over small frontiers run without the big list (broadcast_round); 0 = off
  uint32_t bcast;
  // a round whose frontier has more than n / dense_div items runs dense (every
  // vertex in id order, popped if the previous round pushed it); 0 = never
  uint32_t dense_div;
  // rounds whose frontier is below one tile per CTA spread it over the grid; 0 = off
  uint32_t spread;
  // SSSP on packed words, plain rounds: a popped vertex of degree >= defer_deg
  // whose distance exceeds the round's smallest pushed distance + defer_delta
  // is pushed again instead of expanded (defer_deg 0: off)
  uint32_t defer_deg;
  uint32_t defer_delta;
};

// Per-launch (one round) arguments.
struct RoundArgs {
  const uint32_t* in_items;  // nullptr = items 0..n-1
  const uint32_t* in_count;  // nullptr = n
  uint32_t in_cap;           // the size read from in_count is clamped to this
  uint32_t* in_consume;      // if set, zeroed after the round (the in-worklist was popped)
  uint32_t* out_items;
  uint32_t* out_tail;
  uint32_t out_cap;
  uint32_t level;            // BFS LEVEL
};

// Batched mode: one descriptor per query (instance), kept sorted by arena base.
// A worklist item is an arena index base + v; its query is found by binary
// search over the sorted bases (the per-instance offset table).
constexpr int kMaxBatchQueries = 1024;

struct QDesc {
  const uint32_t* row_ptr;
  const uint32_t* col;
  const int32_t* w;
  uint32_t n;     // vertices of the query's graph
  uint32_t op;    // OP_BFS / OP_SSSP / OP_CC
  uint32_t base;  // arena offset of the query's state (and stamps)
  uint32_t slot;  // query id (index into qlast)
};

struct BParams {
  const QDesc* desc;        // nq descriptors, sorted by base
  const uint32_t* sbases;   // nq sorted bases
  uint32_t nq;
  uint32_t* state;          // arena: result of every query (filled from ds after the run)
  uint32_t* stamp;          // arena: push dedup stamps (unused when ds is set)
  unsigned long long* ds;   // arena: (value << 32) | id of the round that last lowered it
  uint32_t* qlast;          // per query id: stamp (round id) of its last push
  uint32_t* items[2];       // shared worklists of arena indices
  uint32_t cap;
  uint32_t* cont;           // cont[0]: buffer holding pending items, cont[1]: their count
  DevStatus* st;
  Tune tn;
  uint32_t max_rounds;      // rounds per launch (an epoch); 0xFFFFFFFF = run to empty
  int rounds_cap_is_error;  // 1: hitting max_rounds is DERR_MAX_ROUNDS; 0: epoch end
  unsigned long long timeout_ns;
  unsigned long long time_limit_ns;  // wall time after which the launch stops with DERR_TIME_LIMIT (0 = none)
  unsigned long long* trace;
  uint32_t trace_cap;
  BigList big;
  // near-far for SSSP queries (delta != 0): a popped item at or above its
  // query's limit waits on the far list; cont[2], cont[3] carry the far list
  // (buffer, size) between launches like cont[0], cont[1] the out-worklist
  uint32_t delta;
  uint32_t* blim;           // per slot: the query's limit at the end of the last launch
  uint32_t* far_items[2];   // far lists of arena indices
  uint32_t far_cap;
  uint32_t* far_stamp;      // arena: round id of the far list a vertex was last put on
  // CTA-local sub-rounds per round (0 = off). Round r then owns the ids
  // ep0 + r (k + 1) .. ep0 + r (k + 1) + k: its base id marks pushes (qlast)
  // and the far lists, sub-round j stamps packed words with base + j
  uint32_t local_rounds;
  // rounds whose frontier is below one tile per CTA spread it over the grid; 0 = off
  uint32_t spread;
  // deferred expansion of long lists for SSSP queries (plain rounds): three
  // buffers of kMaxBatchQueries words, ~(smallest distance a query pushed in a
  // round) by slot; nullptr = off
  uint32_t* dmin;
  uint32_t defer_deg;
  uint32_t defer_delta;
};

// ----------------------------------------------------------------------------- small helpers

// Wall-time bound of a persistent launch: CTA 0 checks it at the start of a
// round and sets the sticky error, which the next grid barrier publishes, so
// every CTA leaves the round loop together; a run that would never converge
// ends with a status instead of holding the GPU.
__device__ __forceinline__ unsigned long long globaltimer_ns();
__device__ __forceinline__ void check_time_limit(uint32_t* err, unsigned long long t0, unsigned long long limit) {
  if (limit != 0 && blockIdx.x == 0 && threadIdx.x == 0 && globaltimer_ns() - t0 > limit)
    atomicCAS(err, 0u, static_cast<uint32_t>(DERR_TIME_LIMIT));
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Adjacency (col, w) loads: read once per round, so (unless IRGL_NO_L2_HINTS) they
// carry an L2 evict-first policy and skip L1, keeping the randomly accessed
// state and stamp arrays resident in L2.
#ifndef IRGL_NO_L2_HINTS
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
template <class T>
__device__ __forceinline__ T ld_adj(const T* p) {
  static_assert(sizeof(T) == 4, "scalar adjacency load");
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(l2_evict_first()));
  return static_cast<T>(v);
}
__device__ __forceinline__ uint4 ld_adj4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
__device__ __forceinline__ int4 ld_adj4(const int4* p) {
  const uint4 v = ld_adj4(reinterpret_cast<const uint4*>(p));
  return make_int4(static_cast<int>(v.x), static_cast<int>(v.y), static_cast<int>(v.z), static_cast<int>(v.w));
}
#else
template <class T>
__device__ __forceinline__ T ld_adj(const T* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ld_adj4(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ int4 ld_adj4(const int4* p) { return __ldg(p); }
#endif

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, x, o);
    if (lane >= static_cast<uint32_t>(o)) x += t;
  }
  return x;
}

struct Out {
  uint32_t* items;
  uint32_t* tail;
  uint32_t cap;
  uint32_t* err;
};

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t code) { atomicCAS(err, DERR_NONE, code); }

// ----------------------------------------------------------------------------- shared memory

template <int CTA>
struct Smem {
  // push stage capacity (items): flushed at tile and phase ends; pushes that
  // do not fit go straight to the out-worklist (warp-aggregated)
  static constexpr int kStage = 16 * CTA < 8192 ? 16 * CTA : 8192;
  static constexpr int kWarps = CTA / 32;
  uint32_t stage[kStage];
  uint32_t stage_n;
  uint32_t gbase;
  uint32_t grab_base;
  uint32_t flag;
  uint32_t own_tid, own_beg, own_end, own_val, own_q;  // CTA bin owner broadcast
  uint32_t pub_out;                         // out-worklist size published by the grid barrier
  uint32_t pub_err;                         // device error code published by the grid barrier
  uint32_t round_pushes;                    // out-worklist slots this CTA reserved in the current round
  uint32_t far_min_cta;                     // smallest distance this CTA pushed to the far list
  uint32_t big_appended;                    // this CTA appended to the big list in the current round
  uint32_t pub_flags;                       // kRelBigFlag when the big list is pending
  unsigned long long pub_big;               // published big-list counter
  unsigned long long mf_cta;                // out-edges of the vertices this CTA pushed this round
  uint32_t pmin_cta;                        // smallest distance this CTA pushed since its last report (SSSP)
  unsigned long long edges;
  uint8_t pushed[CTA];                      // ReduceAndReturn All: item pushed something
};

template <int CTA>
struct BatchSmem {
  Smem<CTA> core;
  uint32_t sbases[kMaxBatchQueries];
  uint32_t qbits[kMaxBatchQueries / 32];  // queries (by slot) this CTA pushed for in the current round
  uint32_t qfar[kMaxBatchQueries / 32];   // queries (by slot) this CTA kept on the far list
  uint32_t lim[kMaxBatchQueries];         // near-far: this round's limit of each query (by id)
};

// ----------------------------------------------------------------------------- cooperative-conversion push

// Flush the stage to the out-worklist: one global atomicAdd, coalesced stores.
// Called by every thread of the CTA at a CTA-uniform point, after a barrier.
template <int CTA>
__device__ __forceinline__ void flush_stage(Smem<CTA>& sm, const Out& out, uint32_t from = 0) {
  const uint32_t end = min(sm.stage_n, static_cast<uint32_t>(Smem<CTA>::kStage));
  const uint32_t n = end > from ? end - from : 0u;
  if (n == 0) {
    if (from != 0) {  // the stage held only expanded items: empty it
      __syncthreads();
      if (threadIdx.x == 0) sm.stage_n = 0;
      __syncthreads();
    }
    return;
  }
  if (threadIdx.x == 0) {
    sm.gbase = atomicAdd(out.tail, n);
    sm.round_pushes += n;
  }
  __syncthreads();
  const uint32_t gb = sm.gbase;
  for (uint32_t i = threadIdx.x; i < n; i += CTA) {
    const uint32_t idx = gb + i;
    if (idx < out.cap) __stcg(out.items + idx, sm.stage[from + i]);
    else set_err(out.err, DERR_WL_OVERFLOW);
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.stage_n = 0;
  __syncthreads();
}

// Items that did not fit the stage go straight to global memory, aggregated per warp.
__device__ __forceinline__ void push_global_warp(const Out& out, uint32_t* round_pushes, uint32_t cnt_lane,
                                                 uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t incl = warp_incl_scan(cnt_lane);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  uint32_t gb = 0;
  if (lane == 31) {
    gb = atomicAdd(out.tail, total);
    atomicAdd(round_pushes, total);
  }
  gb = __shfl_sync(kFull, gb, 31);
  uint32_t pos = gb + incl - cnt_lane;
  const uint32_t vs[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (static_cast<uint32_t>(i) < cnt_lane) {
      if (pos < out.cap) __stcg(out.items + pos, vs[i]);
      else set_err(out.err, DERR_WL_OVERFLOW);
      ++pos;
    }
  }
}

// One candidate item per lane: ballot/popc aggregation into the stage.
template <int CTA>
__device__ __forceinline__ void push1(Smem<CTA>& sm, const Out& out, bool p, uint32_t v) {
  const unsigned m = __ballot_sync(kFull, p);
  if (m == 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const int ld = __ffs(m) - 1;
  const uint32_t cnt = __popc(m);
  uint32_t base = 0;
  if (lane == static_cast<uint32_t>(ld)) base = atomicAdd(&sm.stage_n, cnt);
  base = __shfl_sync(kFull, base, ld);
  const uint32_t pos = base + __popc(m & lanemask_lt());
  const bool fits = pos < static_cast<uint32_t>(Smem<CTA>::kStage);
  if (p && fits) sm.stage[pos] = v;
  if (base + cnt > static_cast<uint32_t>(Smem<CTA>::kStage)) {
    const bool ov = p && !fits;
    push_global_warp(out, &sm.round_pushes, ov ? 1u : 0u, v, 0u, 0u, 0u);
  }
}

// Up to four candidate items per lane (flags f bits 0..3): warp scan aggregation.
template <int CTA>
__device__ __forceinline__ void push4(Smem<CTA>& sm, const Out& out, uint32_t f, uint32_t v0, uint32_t v1,
                                      uint32_t v2, uint32_t v3) {
  if (!__any_sync(kFull, f != 0u)) return;  // most strips push nothing: one vote, no scan
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t k = __popc(f);
  const uint32_t incl = warp_incl_scan(k);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&sm.stage_n, total);
  base = __shfl_sync(kFull, base, 31);
  constexpr uint32_t S = Smem<CTA>::kStage;
  uint32_t pos = base + incl - k;
  uint32_t ov = 0;
  // compact the flagged values of this lane: o0..o3 in order
  uint32_t o[4] = {0u, 0u, 0u, 0u};
  uint32_t j = 0;
  if (f & 1u) { o[0] = v0; j = 1; }
  if (f & 2u) { if (j == 0) o[0] = v1; else o[1] = v1; ++j; }
  if (f & 4u) { if (j == 0) o[0] = v2; else if (j == 1) o[1] = v2; else o[2] = v2; ++j; }
  if (f & 8u) { if (j == 0) o[0] = v3; else if (j == 1) o[1] = v3; else if (j == 2) o[2] = v3; else o[3] = v3; ++j; }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (static_cast<uint32_t>(i) < k) {
      if (pos < S) sm.stage[pos] = o[i];
      else ++ov;
      ++pos;
    }
  }
  if (base + total > S) {
    // overflowed items of this lane are its last `ov` compacted values
    const uint32_t skip = k - ov;
    uint32_t g0 = 0, g1 = 0, g2 = 0, g3 = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t src = skip + static_cast<uint32_t>(i);
      const uint32_t val = src == 0 ? o[0] : src == 1 ? o[1] : src == 2 ? o[2] : o[3];
      if (i == 0) g0 = val; else if (i == 1) g1 = val; else if (i == 2) g2 = val; else g3 = val;
    }
    push_global_warp(out, &sm.round_pushes, ov, g0, g1, g2, g3);
  }
}

// ----------------------------------------------------------------------------- warp helpers

// Largest lane j < n whose `key` (held by lane j; non-decreasing over lanes,
// lane 0's key <= e) is <= e. Five shuffle steps, all lanes together.
template <class K>
__device__ __forceinline__ uint32_t warp_find(K key, K e, uint32_t n) {
  uint32_t lo = 0, hi = n - 1;
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const uint32_t md = (lo + hi + 1) >> 1;
    const K km = __shfl_sync(kFull, key, md);
    if (lo < hi) {
      if (km <= e) lo = md;
      else hi = md - 1;
    }
  }
  return lo;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long x) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFull, x, o);
    if (lane >= static_cast<uint32_t>(o)) x += t;
  }
  return x;
}

// ----------------------------------------------------------------------------- graph views

// One graph, vertex ids are state indices. OP fixed at compile time.
template <uint32_t OP>
struct SingleView {
  const uint32_t* __restrict__ row_ptr;
  const uint32_t* __restrict__ col;
  const int32_t* __restrict__ w;
  uint32_t* state;
  uint32_t* stamp;
  uint32_t n;
  static constexpr bool kBatched = false;
  static constexpr const uint32_t* lim = nullptr;
  __device__ __forceinline__ uint32_t nverts(uint32_t) const { return n; }
  __device__ __forceinline__ uint32_t op(uint32_t) const { return OP; }
  __device__ __forceinline__ const uint32_t* rowp(uint32_t) const { return row_ptr; }
  __device__ __forceinline__ const uint32_t* colp(uint32_t) const { return col; }
  __device__ __forceinline__ const int32_t* wp(uint32_t) const { return w; }
  __device__ __forceinline__ uint32_t sbase(uint32_t) const { return 0u; }
  __device__ __forceinline__ void decode(uint32_t item, uint32_t& q, uint32_t& u) const { q = 0; u = item; }
  __device__ __forceinline__ void mark(uint32_t, uint32_t) const {}
  __device__ __forceinline__ uint32_t slot(uint32_t) const { return 0u; }
};

// Many queries over many graphs; op taken per query at run time.
struct BatchView {
  const QDesc* __restrict__ desc;
  const uint32_t* sbases;  // shared-memory copy
  uint32_t nq;
  uint32_t* state;
  uint32_t* stamp;
  uint32_t* qbits;  // shared-memory bitmap of queries that pushed this round
  uint32_t* qfar;   // shared-memory bitmap of queries that kept far items this round
  const uint32_t* lim;  // near-far: per-query limits (shared memory), or nullptr
  uint32_t* far_stamp;
  static constexpr bool kBatched = true;
  __device__ __forceinline__ uint32_t op(uint32_t q) const { return __ldg(&desc[q].op); }
  __device__ __forceinline__ const uint32_t* rowp(uint32_t q) const {
    return reinterpret_cast<const uint32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&desc[q].row_ptr)));
  }
  __device__ __forceinline__ const uint32_t* colp(uint32_t q) const {
    return reinterpret_cast<const uint32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&desc[q].col)));
  }
  __device__ __forceinline__ const int32_t* wp(uint32_t q) const {
    return reinterpret_cast<const int32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&desc[q].w)));
  }
  __device__ __forceinline__ uint32_t sbase(uint32_t q) const { return sbases[q]; }
  __device__ __forceinline__ uint32_t nverts(uint32_t q) const { return __ldg(&desc[q].n); }
  __device__ __forceinline__ uint32_t slot(uint32_t q) const { return __ldg(&desc[q].slot); }
  __device__ __forceinline__ void decode(uint32_t item, uint32_t& q, uint32_t& u) const {
    uint32_t lo = 0, hi = nq - 1;
    while (lo < hi) {
      const uint32_t md = (lo + hi + 1) >> 1;
      if (sbases[md] <= item) lo = md;
      else hi = md - 1;
    }
    q = lo;
    u = item - sbases[lo];
  }
  // per-instance termination flag: a shared-memory bit per query; the CTA
  // folds its bits into the round's global bitmap once, before the barrier
  __device__ __forceinline__ void mark(uint32_t q, uint32_t) const {
    const uint32_t slot = __ldg(&desc[q].slot);
    atomicOr(&qbits[slot >> 5], 1u << (slot & 31u));
  }
  // near-far: the query holds far items (still active, but no out-worklist push)
  __device__ __forceinline__ void mark_far(uint32_t q) const {
    const uint32_t slot = __ldg(&desc[q].slot);
    atomicOr(&qfar[slot >> 5], 1u << (slot & 31u));
  }
};

// ----------------------------------------------------------------------------- operator

// Relax edge (u -> v): `val` is the popped vertex's operator value
// (BFS: the level to assign; SSSP: dist[u]; CC: label[u]). Returns true when v
// must be pushed (its value changed and, for SSSP/CC, it is not yet on the
// out-worklist of this round: the stamp dedup keeps each round <= n items).
template <uint32_t OP>
__device__ __forceinline__ bool relax(uint32_t op_rt, uint32_t* state, uint32_t* stamp, uint32_t v, uint32_t val,
                                      int32_t wt, uint32_t ep) {
  const uint32_t op = OP == OP_RUNTIME ? op_rt : OP;
  if (op == OP_BFS) {
    if (__ldcg(state + v) != kInf) return false;
    return atomicCAS(state + v, kInf, val) == kInf;
  }
  const uint32_t nd = op == OP_SSSP ? val + static_cast<uint32_t>(wt) : val;
  if (nd >= __ldcg(state + v)) return false;
  const uint32_t old = atomicMin(state + v, nd);
  if (nd >= old) return false;
  return atomicExch(stamp + v, ep) != ep;
}

// Same operator with the destination's current value `cur` already loaded, so
// callers can issue all their state loads before the first atomic.
template <uint32_t OP>
__device__ __forceinline__ bool decide(uint32_t op_rt, uint32_t* state, uint32_t* stamp, uint32_t v, uint32_t val,
                                       int32_t wt, uint32_t cur, uint32_t ep) {
  const uint32_t op = OP == OP_RUNTIME ? op_rt : OP;
  if (op == OP_BFS) {
    if (cur != kInf) return false;
    return atomicCAS(state + v, kInf, val) == kInf;
  }
  const uint32_t nd = op == OP_SSSP ? val + static_cast<uint32_t>(wt) : val;
  if (nd >= cur) return false;
  const uint32_t old = atomicMin(state + v, nd);
  if (nd >= old) return false;
  return atomicExch(stamp + v, ep) != ep;
}

template <uint32_t OP>
__device__ __forceinline__ bool needs_w(uint32_t op_rt) {
  return (OP == OP_RUNTIME ? op_rt : OP) == OP_SSSP;
}

// ----------------------------------------------------------------------------- one tile of items

struct RoundCtx {
  const uint32_t* in_items;
  uint32_t in_n;
  Out out;
  uint32_t bfs_val;  // level assigned by BFS in this round (single-graph mode)
  uint32_t ep;       // dedup stamp of this round
  uint32_t* grab;
  Tune tn;
  BigList big;                    // cap 0: long lists stay in the CTA bin
  unsigned long long* big_ctr;
  // near-far (SSSP, CC): improvements to a value >= limit go to the far list
  uint32_t limit;                 // kInf: every improvement goes to `out`
  Out far_out;
  uint32_t* far_stamp;
  uint32_t phase;                 // far-list dedup id of the current phase
  uint32_t* changes;              // pointer-jumping CC: hooks that lowered a parent (shared memory)
  unsigned long long* mf;         // direction-optimising BFS: out-degrees of pushed vertices (shared memory)
  const uint32_t* row_ptr;        //   and the row offsets to take them from
  uint32_t* vis;                  // BFS visited bitmap, or nullptr
  unsigned long long* ds;         // SSSP packed (dist, round id) words, or nullptr
  uint32_t dsr;                   //   and this round's id in them (1, 2, ...)
  uint32_t local_rounds;          // CTA-local sub-rounds after the tiles (0 = none)
  const uint32_t* local_items;    // a sub-round's items: a range of the CTA's stage (shared memory)
  const uint32_t* far_in;         // batched near-far: the far items waiting from earlier rounds
  uint32_t far_in_n;
  // dense round (single query): the items are every vertex in id order and a
  // vertex is popped only if the previous round pushed it (its packed word
  // carries dense_id; BFS: its level is this round's); else 0
  uint32_t dense = 0;
  uint32_t dense_id = 0;
  uint32_t spread = 0;  // persistent launches: a frontier below one tile per CTA is spread over the grid
  // single-query SSSP deferred expansion: lists of >= defer_deg edges whose
  // vertex is above defer_lim wait a round (kInf: none); pmin gathers the
  // smallest distance pushed (shared memory), or nullptr
  uint32_t defer_lim = kInf;
  uint32_t defer_deg = 0;
  uint32_t* pmin = nullptr;
  // batched form: per-slot smallest pushed distances of the last round (limits
  // of this one; nullptr: no deferral) and of this round (nullptr: not noted)
  const uint32_t* bdmin_cur = nullptr;
  uint32_t* bdmin_next = nullptr;
  uint32_t defer_delta = 0;
};

// Batched deferred expansion: lanes that pushed SSSP distances for the same
// query slot combine their smallest into one atomic on that slot's word of
// the round's buffer (stored complemented, so 0 means nothing pushed). Every
// lane of the warp calls it; mn = kInf: nothing to note.
__device__ __forceinline__ void note_pushes(uint32_t* next, uint32_t slot, uint32_t mn) {
  const uint32_t key = mn != kInf ? slot : 0xFFFFFFFFu;
  const unsigned grp = __match_any_sync(kFull, key);
  const uint32_t gm = __reduce_min_sync(grp, mn);
  if (key != 0xFFFFFFFFu && (threadIdx.x & 31u) == static_cast<uint32_t>(__ffs(grp) - 1)) atomicMax(next + slot, ~gm);
}

// The destination's current value as the operator reads it. BFS with the
// visited bitmap: the bit is read through L1 (a 128 KB bitmap of 2^20 vertices
// stays there, where the 4 MB level array would be read from L2 per edge). A
// bit is set only after the level is written, so a set bit is always right; a
// stale clear bit (set later in this round, or cached before) falls through
// to the L2 read of the level, which decides.
template <uint32_t OP>
__device__ __forceinline__ uint32_t load_cur(const RoundCtx& rc, const uint32_t* state, uint32_t sb, uint32_t v) {
  if (OP == OP_BFS && rc.vis != nullptr && ((rc.vis[v >> 5] >> (v & 31u)) & 1u)) return 0u;
  if (kPackedOp<OP> && rc.ds != nullptr) return static_cast<uint32_t>(__ldcg(rc.ds + sb + v) >> 32);
  return __ldcg(state + v);
}

// decide() with the near-far routing (SSSP, CC): 0 = no push, 1 = push to this
// round's out-worklist, 2 = push to the far list. Near pushes dedup on the
// round stamp, far pushes on the phase stamp, so a vertex improved first above
// and then below the limit within one round still reaches the out-worklist.
template <uint32_t OP>
__device__ __forceinline__ uint32_t decide_route(uint32_t op_rt, uint32_t* state, uint32_t* stamp, uint32_t v,
                                                 uint32_t val, int32_t wt, uint32_t cur, const RoundCtx& rc,
                                                 uint32_t sb, uint32_t& nd_out) {
  if (OP == OP_CCJ) {
    // hook: the larger of the two endpoints' parents is pointed at the smaller one
    if (val == cur) return 0u;
    const uint32_t lo = min(val, cur), hi = max(val, cur);
    if (atomicMin(state + hi, lo) > lo) atomicAdd(rc.changes, 1u);
    return 0u;
  }
  if (OP == OP_BFS) {
    const bool p = decide<OP>(op_rt, state, stamp, v, val, wt, cur, rc.ep);
    if (p && rc.vis) atomicOr(rc.vis + (v >> 5), 1u << (v & 31u));
    if (p && rc.mf) atomicAdd(rc.mf, static_cast<unsigned long long>(__ldg(rc.row_ptr + v + 1) - __ldg(rc.row_ptr + v)));
    return p ? 1u : 0u;
  }
  if (kPackedOp<OP> && rc.ds != nullptr) {
    // one 64-bit atomicMin lowers the value and stamps the round: v is
    // pushed by the thread that lowers it first in this round (a far
    // improvement stamps 0: see decide_n). BFS levels are lowered from INF.
    const uint32_t o = OP == OP_RUNTIME ? op_rt : OP;
    const uint32_t nd = o == OP_SSSP ? val + static_cast<uint32_t>(wt) : (o == OP_BFSR ? val + 1u : val);
    // batched BFS under CTA-local sub-rounds is label-correcting (as in decide_n)
    const bool first_only = o == OP_BFS && !(OP == OP_RUNTIME && rc.local_rounds != 0);
    if (first_only ? cur != kInf : nd >= cur) return 0u;
    const bool far = OP == OP_SSSP && rc.limit != kInf && nd >= rc.limit;
    const unsigned long long old =
        atomicMin(rc.ds + sb + v, (static_cast<unsigned long long>(nd) << 32) | (far ? 0u : rc.dsr));
    if (nd >= static_cast<uint32_t>(old >> 32)) return 0u;
    if (!far) {
      const bool push = static_cast<uint32_t>(old) != rc.dsr;
      if (OP == OP_SSSP && push && rc.pmin != nullptr) atomicMin(rc.pmin, nd);
      return push ? 1u : 0u;
    }
    nd_out = nd;
    return atomicExch(rc.far_stamp + v, rc.phase) != rc.phase ? 2u : 0u;
  }
  if (!kNearFarOp<OP> || rc.limit == kInf) return decide<OP>(op_rt, state, stamp, v, val, wt, cur, rc.ep) ? 1u : 0u;
  const uint32_t nd = OP == OP_SSSP ? val + static_cast<uint32_t>(wt) : val;
  if (nd >= cur) return 0u;
  const uint32_t old = atomicMin(state + v, nd);
  if (nd >= old) return 0u;
  if (nd < rc.limit) return atomicExch(stamp + v, rc.ep) != rc.ep ? 1u : 0u;
  nd_out = nd;
  return atomicExch(rc.far_stamp + sb + v, rc.phase) != rc.phase ? 2u : 0u;
}

// The operator on N edges of one lane at once. Every atomic whose result
// decides a push is issued before any of those results is read, so the N L2
// round trips overlap instead of following one another. Same outcome as
// decide_route edge by edge (which pointer-jumping CC keeps using), near-far
// routing included. `state`/`stamp` are array bases, edge k's vertex is
// sb[k] + v[k].
template <uint32_t OP, int N>
__device__ __forceinline__ void decide_n(const RoundCtx& rc, uint32_t* state, uint32_t* stamp,
                                         const uint32_t (&op)[N], const uint32_t (&sb)[N], const uint32_t (&v)[N],
                                         const uint32_t (&val)[N], const int32_t (&wt)[N], const uint32_t (&cur)[N],
                                         uint32_t valid, uint32_t (&r)[N], uint32_t (&nd)[N]) {
  if (OP == OP_CCJ) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      nd[k] = 0;
      r[k] = ((valid >> k) & 1u) ? decide_route<OP>(op[k], state + sb[k], stamp + sb[k], v[k], val[k], wt[k], cur[k],
                                                      rc, sb[k], nd[k])
                                 : 0u;
    }
    return;
  }
  bool t[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t o = OP == OP_RUNTIME ? op[k] : OP;
    nd[k] = o == OP_SSSP ? val[k] + static_cast<uint32_t>(wt[k]) : (o == OP_BFSR ? val[k] + 1u : val[k]);
    // BFS takes unvisited vertices only, except batched BFS under CTA-local
    // sub-rounds, where a vertex can be reached before its level is final
    // and later lowered (unit-weight relaxation: same fixed point)
    const bool first_only = o == OP_BFS && !(OP == OP_RUNTIME && rc.local_rounds != 0);
    t[k] = ((valid >> k) & 1u) != 0 && (first_only ? cur[k] == kInf : nd[k] < cur[k]);
  }
  // near-far: an improvement to a value >= the limit goes to the far list,
  // deduplicated per phase by far_stamp (route 2)
  const bool nf = kNearFarOp<OP> && rc.limit != kInf;
  bool far[N];
#pragma unroll
  for (int k = 0; k < N; ++k) far[k] = nf && nd[k] >= rc.limit;
  if (kPackedOp<OP> && rc.ds != nullptr && !nf) {
    unsigned long long old[N];
#pragma unroll
    for (int k = 0; k < N; ++k)
      old[k] = t[k] ? atomicMin(rc.ds + sb[k] + v[k], (static_cast<unsigned long long>(nd[k]) << 32) | rc.dsr) : 0ull;
#pragma unroll
    for (int k = 0; k < N; ++k)
      r[k] = (t[k] && nd[k] < static_cast<uint32_t>(old[k] >> 32) && static_cast<uint32_t>(old[k]) != rc.dsr) ? 1u : 0u;
    if (OP == OP_SSSP && rc.pmin != nullptr) {
      uint32_t mn = kInf;
#pragma unroll
      for (int k = 0; k < N; ++k) mn = r[k] ? min(mn, nd[k]) : mn;
      if (mn != kInf) atomicMin(rc.pmin, mn);
    }
    return;
  }
  if (OP == OP_SSSP && rc.ds != nullptr) {
    // A far improvement writes round id 0: the vertex is not on this round's
    // out-worklist (its value was >= the limit, so no near push happened this
    // round), and a later near improvement in the round must still push it.
    unsigned long long old[N];
#pragma unroll
    for (int k = 0; k < N; ++k)
      old[k] = t[k] ? atomicMin(rc.ds + v[k], (static_cast<unsigned long long>(nd[k]) << 32) | (far[k] ? 0u : rc.dsr))
                    : 0ull;
    bool imp[N];
    uint32_t fx[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      imp[k] = t[k] && nd[k] < static_cast<uint32_t>(old[k] >> 32);
      fx[k] = ~rc.phase;
      if (imp[k] && far[k]) fx[k] = atomicExch(rc.far_stamp + v[k], rc.phase);
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
      r[k] = !imp[k] ? 0u
                     : far[k] ? (fx[k] != rc.phase ? 2u : 0u) : (static_cast<uint32_t>(old[k]) != rc.dsr ? 1u : 0u);
    return;
  }
  uint32_t old[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t o = OP == OP_RUNTIME ? op[k] : OP;
    uint32_t* const s = state + sb[k] + v[k];
    old[k] = 0u;
    if (t[k]) old[k] = o == OP_BFS ? atomicCAS(s, kInf, nd[k]) : atomicMin(s, nd[k]);
  }
  bool imp[N];
  uint32_t ex[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t o = OP == OP_RUNTIME ? op[k] : OP;
    imp[k] = t[k] && (o == OP_BFS ? old[k] == kInf : nd[k] < old[k]);
    ex[k] = far[k] ? ~rc.phase : ~rc.ep;
    if (imp[k] && o != OP_BFS)
      ex[k] = far[k] ? atomicExch(rc.far_stamp + sb[k] + v[k], rc.phase) : atomicExch(stamp + sb[k] + v[k], rc.ep);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t o = OP == OP_RUNTIME ? op[k] : OP;
    r[k] = (imp[k] && (o == OP_BFS || ex[k] != (far[k] ? rc.phase : rc.ep))) ? (far[k] ? 2u : 1u) : 0u;
    if (OP == OP_BFS && r[k] != 0u) {
      if (rc.vis) atomicOr(rc.vis + (v[k] >> 5), 1u << (v[k] & 31u));
      if (rc.mf)
        atomicAdd(rc.mf, static_cast<unsigned long long>(__ldg(rc.row_ptr + v[k] + 1) - __ldg(rc.row_ptr + v[k])));
    }
  }
}

// Far-list pushes: warp-aggregated straight to global memory (rare next to
// out-worklist pushes), plus the CTA's smallest far distance.
template <int CTA>
__device__ __forceinline__ void push_far4(Smem<CTA>& sm, const Out& fo, uint32_t f, uint32_t v0, uint32_t v1,
                                          uint32_t v2, uint32_t v3, uint32_t dmin) {
  if (!__any_sync(kFull, f != 0)) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t k = __popc(f);
  const uint32_t incl = warp_incl_scan(k);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  uint32_t gb = 0;
  if (lane == 31) gb = atomicAdd(fo.tail, total);
  gb = __shfl_sync(kFull, gb, 31);
  uint32_t pos = gb + incl - k;
  const uint32_t vs[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (f >> i & 1u) {
      if (pos < fo.cap) __stcg(fo.items + pos, vs[i]);
      else set_err(fo.err, DERR_WL_OVERFLOW);
      ++pos;
    }
  }
  if (f) atomicMin(&sm.far_min_cta, dmin);
}

// Edges [beg, end) of one owner, GROUP threads cooperating (GROUP = 32: a warp,
// GROUP = CTA: the whole CTA); `rank` in [0, GROUP). 16-byte vector loads of
// col (and w) after an alignment peel; the loop trip count is uniform across
// the group so the warp-level pushes see converged warps.
template <uint32_t OP, int CTA, int GROUP, class V>
__device__ __forceinline__ bool group_edges(const V& g, Smem<CTA>& sm, const RoundCtx& rc, uint32_t q, uint32_t beg,
                                            uint32_t end, uint32_t val, uint32_t rank) {
  const uint32_t op = g.op(q);
  const uint32_t* __restrict__ col = g.colp(q);
  const int32_t* __restrict__ w = g.wp(q);
  const uint32_t sb = g.sbase(q);
  uint32_t* state = g.state + sb;
  uint32_t* stamp = g.stamp + sb;
  const bool nw = needs_w<OP>(op);
  bool any = false;
  const uint32_t a = min(end, (beg + 3u) & ~3u);
  const uint32_t b = a + ((end - a) & ~3u);
  // head (edges before the 16-byte boundary) and tail (after the last full vector): scalar
  auto scalar = [&](uint32_t e, uint32_t lim) {
    uint32_t r = 0, v = 0, nd = 0;
    if (e < lim) {
      v = ld_adj(col + e);
      const int32_t wt = nw ? ld_adj(w + e) : 0;
      r = decide_route<OP>(op, state, stamp, v, val, wt, load_cur<OP>(rc, state, sb, v), rc, sb, nd);
    }
    push1<CTA>(sm, rc.out, r == 1u, sb + v);
    if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, r == 2u ? 1u : 0u, sb + v, 0u, 0u, 0u, nd);
    any |= r != 0;
  };
  scalar(beg + rank, a);
  for (uint32_t base = a; base < b; base += 4u * GROUP) {
    const uint32_t e = base + 4u * rank;
    uint32_t fn = 0, ff = 0, dmin = kInf, pmn = kInf;
    uint4 c = make_uint4(0, 0, 0, 0);
    if (e < b) {
      c = ld_adj4(reinterpret_cast<const uint4*>(col + e));
      int4 ww = make_int4(0, 0, 0, 0);
      if (nw) ww = ld_adj4(reinterpret_cast<const int4*>(w + e));
      // all four destination loads in flight before any atomic, then all four atomics
      const uint32_t vv[4] = {c.x, c.y, c.z, c.w};
      const int32_t wv[4] = {ww.x, ww.y, ww.z, ww.w};
      const uint32_t ops[4] = {op, op, op, op};
      const uint32_t sbs[4] = {sb, sb, sb, sb};  // arena base of every edge's destination
      const uint32_t vals[4] = {val, val, val, val};
      uint32_t cc[4], rr[4], ndv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cc[k] = load_cur<OP>(rc, state, sb, vv[k]);
      // array bases plus per-edge arena offsets, as in every other bin (the
      // packed words are indexed ds + sb + v)
      decide_n<OP, 4>(rc, g.state, g.stamp, ops, sbs, vv, vals, wv, cc, 0xFu, rr, ndv);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (rr[k] == 1u) {
          fn |= 1u << k;
          pmn = min(pmn, ndv[k]);
        }
        if (kNearFarOp<OP> && rr[k] == 2u) {
          ff |= 1u << k;
          dmin = min(dmin, ndv[k]);
        }
      }
    }
    push4<CTA>(sm, rc.out, fn, sb + c.x, sb + c.y, sb + c.z, sb + c.w);
    if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, ff, sb + c.x, sb + c.y, sb + c.z, sb + c.w, dmin);
    if constexpr (V::kBatched) {
      if (rc.bdmin_next != nullptr) note_pushes(rc.bdmin_next, g.slot(q), op == OP_SSSP ? pmn : kInf);
    }
    any |= (fn | ff) != 0;
    if (GROUP == CTA) {
      // the predicate is taken at the barrier, when every warp's pushes are in
      if (__syncthreads_or(sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2))) flush_stage<CTA>(sm, rc.out);
    }
  }
  scalar(b + rank, end);
  if (V::kBatched && any) g.mark(q, rc.ep);  // per-instance termination flag
  return any;
}


// Batched near-far: put `item` of query q on this round's far list (want; at
// most once per round by the far stamp) and mark the query as still active.
// Called by every lane of a converged warp.
template <int CTA, class V>
__device__ __forceinline__ void push_far_item(const V& g, Smem<CTA>& sm, const RoundCtx& rc, bool want, uint32_t item,
                                              uint32_t q) {
  bool f = false;
  if (want) {
    f = atomicExch(g.far_stamp + item, rc.ep) != rc.ep;
    g.mark_far(q);
  }
  push_far4<CTA>(sm, rc.far_out, f ? 1u : 0u, item, 0u, 0u, 0u, kInf);
}

// Put the round id `dsr` into a packed (value, round id) word whose value it
// keeps: true when this call did it (the caller pushes the vertex), false when
// the word already holds dsr (the vertex is already on this round's
// out-worklist). A bounded CAS loop; a word lowered under it is re-read.
__device__ __forceinline__ bool stamp_pending(unsigned long long* p, unsigned long long w, uint32_t dsr) {
  for (int k = 0; k < 64; ++k) {
    if (static_cast<uint32_t>(w) == dsr) return false;
    const unsigned long long o = atomicCAS(p, w, (w & 0xFFFFFFFF00000000ull) | dsr);
    if (o == w) return true;
    w = o;
  }
  return true;  // contended: push anyway (a duplicate only repeats an expansion)
}

// Batched near-far: every far item of the last round is looked at once. Its
// query's limit has passed it: it goes onto this round's out-worklist (a near
// push, so the limit stays); else it stays on the far list. Static share per
// CTA; the trip count is CTA-uniform, so the warp-aggregated pushes converge.
template <int CTA, class V>
__device__ __forceinline__ void far_sweep(const V& g, Smem<CTA>& sm, const RoundCtx& rc) {
  for (uint32_t base = blockIdx.x * CTA; base < rc.far_in_n; base += gridDim.x * CTA) {
    const uint32_t i = base + threadIdx.x;
    bool near = false, keep = false;
    uint32_t item = 0, q = 0;
    if (i < rc.far_in_n) {
      item = __ldcg(rc.far_in + i);
      uint32_t u;
      g.decode(item, q, u);
      const unsigned long long w = __ldcg(rc.ds + item);
      if (static_cast<uint32_t>(w >> 32) < g.lim[q]) {
        near = stamp_pending(rc.ds + item, w, rc.dsr);
        if (near) g.mark(q, rc.ep);
      } else {
        keep = true;
      }
    }
    push1<CTA>(sm, rc.out, near, item);
    push_far_item<CTA>(g, sm, rc, keep, item, q);
  }
}

template <uint32_t OP, int CTA, int RED, class V>
__device__ __forceinline__ void process_tile(const V& g, Smem<CTA>& sm, const RoundCtx& rc, uint32_t idx,
                                             uint32_t& edges, uint32_t& any_true, uint32_t& any_false) {
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31;
  const uint32_t wbase = tid & ~31u;
  bool valid = idx < rc.in_n;
  uint32_t q = 0, beg = 0, end = 0, val = 0, item = 0;
  unsigned long long pw = 0;  // the popped packed word (single-query SSSP)
  if (valid) {
    item = rc.local_items ? rc.local_items[idx] : (rc.in_items ? __ldcg(rc.in_items + idx) : idx);
    uint32_t u;
    g.decode(item, q, u);
    uint32_t dval = 0;
    if (!V::kBatched && rc.dense) {
      // dense round: vertex `item` is popped only if the previous round pushed it
      if (kPackedOp<OP> && rc.ds != nullptr) {
        const unsigned long long wd = __ldcg(rc.ds + item);
        dval = static_cast<uint32_t>(wd >> 32);
        valid = static_cast<uint32_t>(wd) == rc.dense_id && dval != kInf;
      } else {
        dval = __ldcg(g.state + item);
        valid = OP == OP_BFS && dval + 1u == rc.bfs_val;
      }
    }
    if (!valid) {
    } else if (u >= g.nverts(q)) {  // a caller-pushed item outside the graph: report and skip it
      set_err(rc.out.err, DERR_BAD_ITEM);
      valid = false;
    } else if (!V::kBatched && rc.dense) {
      beg = __ldg(g.rowp(q) + u);
      end = __ldg(g.rowp(q) + u + 1);
      val = OP == OP_BFS ? rc.bfs_val : dval;
    } else {
      const uint32_t* rp = g.rowp(q);
      beg = __ldg(rp + u);
      end = __ldg(rp + u + 1);
      const uint32_t op = g.op(q);
      if (kPackedOp<OP> && rc.ds != nullptr && rc.local_items != nullptr)
        // a CTA-local pop: take the value and clear the round stamp in one
        // atomic, so an improvement that lands after this read (from any CTA,
        // in any sub-round) pushes the vertex again instead of counting on a
        // pending expansion that has just happened (a batched BFS item carries
        // the level its out-edges assign, its own + 1)
        val = static_cast<uint32_t>(atomicAnd(rc.ds + item, 0xFFFFFFFF00000000ull) >> 32) +
              (OP == OP_RUNTIME && op == OP_BFS ? 1u : 0u);
      else if (kPackedOp<OP> && rc.ds != nullptr && (OP != OP_RUNTIME || op != OP_BFS)) {
        pw = __ldcg(rc.ds + item);
        val = static_cast<uint32_t>(pw >> 32);
      } else if (op == OP_BFS)
        val = !V::kBatched ? rc.bfs_val
                           : (rc.ds != nullptr ? static_cast<uint32_t>(__ldcg(rc.ds + item) >> 32) : __ldcg(g.state + item)) + 1u;
      else val = __ldcg(g.state + item);
    }
  }
  if constexpr (!V::kBatched && OP == OP_SSSP) {
    // Deferred expansion of long lists: a vertex of degree >= defer_deg whose
    // distance is above defer_lim (the smallest distance pushed for this round
    // plus a margin) is likely to be lowered again before it is final, and each
    // expansion of it rescans all its edges. It stays on the worklist instead:
    // pushed again for the next round (once: the round id in its packed word),
    // its distance counted in the round's smallest, so the smallest item of a
    // round is never deferred and every vertex is expanded in the end.
    bool again = false;
    if (valid && rc.defer_lim != kInf && !rc.dense && rc.local_items == nullptr && end - beg >= rc.defer_deg &&
        val > rc.defer_lim) {
      again = stamp_pending(rc.ds + item, pw, rc.dsr);
      if (again) atomicMin(rc.pmin, val);
      valid = false;
      beg = end = 0;
    }
    if (rc.defer_lim != kInf) push1<CTA>(sm, rc.out, again, item);
  }
  if constexpr (V::kBatched) {
    // the same for SSSP queries of a batch, each against its own smallest
    // pushed distance of the last round (its slot's word; 0: none noted)
    bool again = false;
    if (rc.bdmin_cur != nullptr && valid && rc.local_items == nullptr && end - beg >= rc.defer_deg &&
        g.op(q) == OP_SSSP) {
      const uint32_t sl = g.slot(q);
      const uint32_t pm = __ldcg(rc.bdmin_cur + sl);
      if (pm != 0u && static_cast<unsigned long long>(val) > static_cast<unsigned long long>(~pm) + rc.defer_delta) {
        again = stamp_pending(rc.ds + item, pw, rc.dsr);
        if (again) {
          atomicMax(rc.bdmin_next + sl, ~val);
          g.mark(q, rc.ep);
        }
        valid = false;
        beg = end = 0;
      }
    }
    if (rc.bdmin_cur != nullptr) push1<CTA>(sm, rc.out, again, item);
  }
  if constexpr (V::kBatched) {
    if (g.lim != nullptr) {
      // near-far: an SSSP item at or above its query's limit is not expanded
      // now; it waits on the far list (once per round) until the limit passes it
      const bool defer = valid && g.op(q) == OP_SSSP && val >= g.lim[q];
      if (defer) {
        valid = false;
        beg = end = 0;
      }
      push_far_item<CTA>(g, sm, rc, defer, item, q);
    }
  }
  const uint32_t deg = end - beg;
  edges += deg;
  bool pushed = false;

  // Long lists. With the big list on, each warp appends its long lists (one
  // 64-bit atomic reserves slots and edge offsets together); the whole grid
  // walks them after the round's first barrier. A frontier smaller than one
  // tile per CTA sends every list of warp size or more there: even spread over
  // every CTA, a warp walking a list of a few hundred edges alone is slower
  // than the big phase's equal shares. Lists that do not fit the big list fall
  // back to the warp bin. With the big list off (one-launch rounds), the CTA
  // bin walks lists >= cta_thresh one at a time.
  const uint32_t split = (rc.big.cap != 0 && rc.in_n < gridDim.x * CTA) ? min(rc.tn.warp_thresh, rc.tn.cta_thresh)
                                                                         : rc.tn.cta_thresh;
  bool big = valid && deg >= split;
  if (rc.big.cap != 0) {
    if (__any_sync(kFull, big)) {
      const unsigned long long mine = big ? ((1ull << 40) | deg) : 0ull;
      const unsigned long long incl = warp_incl_scan64(mine);
      const unsigned long long total = __shfl_sync(kFull, incl, 31);
      unsigned long long base = 0;
      if (lane == 31) {
        base = atomicAdd(rc.big_ctr, total);
        sm.big_appended = 1;
      }
      base = __shfl_sync(kFull, base, 31);
      if (big) {
        const unsigned long long at = base + incl - mine;
        const uint32_t slot = static_cast<uint32_t>(at >> 40);
        if (slot < rc.big.cap) {
          rc.big.e[slot] = make_uint4(beg, end, val, q);
          rc.big.off[slot] = at & kBigEdgeMask;
          big = false;
        }
      }
    }
  } else {
    // CTA bin: the whole CTA walks one long list at a time.
    while (__syncthreads_or(big)) {
      if (big) sm.own_tid = tid;
      __syncthreads();
      if (tid == sm.own_tid) {
        sm.own_beg = beg;
        sm.own_end = end;
        sm.own_val = val;
        sm.own_q = q;
        big = false;
      }
      __syncthreads();
      const bool p = group_edges<OP, CTA, CTA>(g, sm, rc, sm.own_q, sm.own_beg, sm.own_end, sm.own_val, tid);
      if (RED == RED_ALL && p) sm.pushed[sm.own_tid] = 1;
      pushed |= p;
    }
  }

  // Warp bin: each warp walks its members' medium lists one at a time.
  bool mid = valid && ((deg >= rc.tn.warp_thresh && deg < split) || big);
  for (;;) {
    const unsigned m = __ballot_sync(kFull, mid);
    if (m == 0) break;
    const int ld = __ffs(m) - 1;
    const uint32_t wb = __shfl_sync(kFull, beg, ld);
    const uint32_t we = __shfl_sync(kFull, end, ld);
    const uint32_t wv = __shfl_sync(kFull, val, ld);
    const uint32_t wq = __shfl_sync(kFull, q, ld);
    if (lane == static_cast<uint32_t>(ld)) mid = false;
    const bool p = group_edges<OP, CTA, 32>(g, sm, rc, wq, wb, we, wv, lane);
    if (RED == RED_ALL && p) sm.pushed[wbase + ld] = 1;
    pushed |= p;
  }

  // Thread bin (opt-in): a list of at most thread_max (<= 4) edges is walked by
  // the lane that popped it, all its loads and atomics in flight together; no
  // search or shuffle per edge (meshes and grids have nothing else).
  const bool tiny = valid && deg > 0 && deg <= rc.tn.thread_max && deg < rc.tn.warp_thresh && deg < split;
  if (__any_sync(kFull, tiny)) {
    uint32_t v[kThreadBin], cur[kThreadBin], sbv[kThreadBin], opv[kThreadBin], ovv[kThreadBin], rr[kThreadBin],
        ndv[kThreadBin];
    int32_t wt[kThreadBin];
    uint32_t vmask = 0;
    const uint32_t oq = tiny ? g.op(q) : static_cast<uint32_t>(OP_BFS);
    const uint32_t sq = tiny ? g.sbase(q) : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kThreadBin; ++k) {
      v[k] = 0;
      wt[k] = 0;
      sbv[k] = sq;
      opv[k] = oq;
      ovv[k] = val;
      if (tiny && k < deg) {
        v[k] = ld_adj(g.colp(q) + beg + k);
        if (needs_w<OP>(oq)) wt[k] = ld_adj(g.wp(q) + beg + k);
        vmask |= 1u << k;
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < kThreadBin; ++k)
      cur[k] = ((vmask >> k) & 1u) ? load_cur<OP>(rc, g.state + sq, sq, v[k]) : 0u;
    decide_n<OP, kThreadBin>(rc, g.state, g.stamp, opv, sbv, v, ovv, wt, cur, vmask, rr, ndv);
    uint32_t f = 0, ff = 0, dmin = kInf;
#pragma unroll
    for (uint32_t k = 0; k < kThreadBin; ++k) {
      if (rr[k] == 1u) f |= 1u << k;
      if (rr[k] == 2u) {
        ff |= 1u << k;
        dmin = min(dmin, ndv[k]);
      }
    }
    if ((f | ff) != 0u) {
      if (RED == RED_ALL) sm.pushed[tid] = 1;
      if (V::kBatched) g.mark(q, rc.ep);
    }
    push4<CTA>(sm, rc.out, f, sq + v[0], sq + v[1], sq + v[2], sq + v[3]);
    if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, ff, sq + v[0], sq + v[1], sq + v[2], sq + v[3], dmin);
    pushed |= (f | ff) != 0;
  }

  // Scan bin, per warp: the short lists of the warp's 32 items are dealt out
  // four edges per lane per strip (strided by 32, so loads coalesce within a
  // list); each edge finds its list by a shuffle binary search over the
  // warp's exclusive degree prefix. No CTA barrier is involved.
  const bool small = valid && deg > 0 && deg < rc.tn.warp_thresh && deg < split && !tiny;
  const uint32_t sdeg = small ? deg : 0u;
  const uint32_t sincl = warp_incl_scan(sdeg);
  const uint32_t sexcl = sincl - sdeg;
  const uint32_t total = __shfl_sync(kFull, sincl, 31);
  constexpr uint32_t E = 4;
  for (uint32_t base = 0; base < total; base += E * 32) {
    uint32_t v[E], cur[E], sb[E], op[E], ov[E], own[E], oqs[E];
    int32_t wt[E];
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) {
      const uint32_t e = base + k * 32 + lane;
      own[k] = warp_find<uint32_t>(sexcl, e < total ? e : total - 1, 32);
    }
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) {
      const uint32_t e = base + k * 32 + lane;
      const uint32_t ob = __shfl_sync(kFull, beg, own[k]);
      const uint32_t oe = __shfl_sync(kFull, sexcl, own[k]);
      const uint32_t oq = __shfl_sync(kFull, q, own[k]);
      oqs[k] = oq;
      ov[k] = __shfl_sync(kFull, val, own[k]);
      v[k] = 0;
      wt[k] = 0;
      sb[k] = 0;
      op[k] = OP_BFS;
      if (e < total) {
        const uint32_t edge = ob + (e - oe);
        op[k] = g.op(oq);
        sb[k] = g.sbase(oq);
        v[k] = ld_adj(g.colp(oq) + edge);
        if (needs_w<OP>(op[k])) wt[k] = ld_adj(g.wp(oq) + edge);
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < E; ++k)
      cur[k] = (base + k * 32 + lane < total) ? load_cur<OP>(rc, g.state + sb[k], sb[k], v[k]) : 0u;
    uint32_t f = 0, ff = 0, dmin = kInf, vmask = 0, rr[E], ndv[E];
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) vmask |= (base + k * 32 + lane < total ? 1u : 0u) << k;
    decide_n<OP, 4>(rc, g.state, g.stamp, op, sb, v, ov, wt, cur, vmask, rr, ndv);
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) {
      const uint32_t r = rr[k];
      if (r == 1u) f |= 1u << k;
      if (r == 2u) {
        ff |= 1u << k;
        dmin = min(dmin, ndv[k]);
      }
      if (r != 0u) {
        if (RED == RED_ALL) sm.pushed[wbase + own[k]] = 1;
        if (V::kBatched) g.mark(oqs[k], rc.ep);
      }
    }
    if constexpr (V::kBatched) {
      if (rc.bdmin_next != nullptr) {
#pragma unroll
        for (uint32_t k = 0; k < E; ++k)
          note_pushes(rc.bdmin_next, g.slot(oqs[k]), (rr[k] == 1u && op[k] == OP_SSSP) ? ndv[k] : kInf);
      }
    }
    push4<CTA>(sm, rc.out, f, sb[0] + v[0], sb[1] + v[1], sb[2] + v[2], sb[3] + v[3]);
    if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, ff, sb[0] + v[0], sb[1] + v[1], sb[2] + v[2], sb[3] + v[3], dmin);
    pushed |= (f | ff) != 0;
  }

  if (RED == RED_ANY) any_true |= pushed ? 1u : 0u;
  // a sub-round reads its items from the stage: no flush may move them under it
  const bool full = __syncthreads_or(rc.local_items == nullptr &&
                                     sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2));
  if (RED == RED_ALL) {
    if (valid && !sm.pushed[tid]) any_false = 1u;
    sm.pushed[tid] = 0;
  }
  if (full) flush_stage<CTA>(sm, rc.out);
}

// ForAll over the in-worklist (Sec. 3.1): the first `chunk` tiles of CTA items
// of each CTA are static (blockIdx-th span); the rest is grabbed dynamically
// with one atomic per span, so small frontiers cost no contended atomic. A
// frontier below one tile per CTA is spread over every CTA instead (below).
template <uint32_t OP, int CTA, int RED, class V>
__device__ __forceinline__ void round_body(const V& g, Smem<CTA>& sm, const RoundCtx& rc, uint32_t& edges,
                                           uint32_t& any_true, uint32_t& any_false) {
  const uint32_t span = CTA * rc.tn.chunk;
  const uint32_t static_end = gridDim.x * span;
  uint32_t gb = blockIdx.x * span;
  if (rc.spread != 0 && rc.in_n <= gridDim.x * CTA) {
    // A frontier smaller than one tile per CTA is spread over the whole grid:
    // CTA b takes items b, b + grid, ..., dealt across its warps (slot s goes
    // to warp s % warps, lane s / warps), so a few thousand items keep every
    // warp's chain of loads and atomics to one or two strips instead of
    // loading 128 items onto each of a few CTAs.
    const uint32_t slot = (threadIdx.x & 31u) * (CTA / 32) + (threadIdx.x >> 5);
    if (blockIdx.x < rc.in_n) process_tile<OP, CTA, RED>(g, sm, rc, blockIdx.x + slot * gridDim.x, edges, any_true, any_false);
    gb = rc.in_n;  // every item is taken
  }
  for (;;) {
    if (gb >= rc.in_n) break;
    for (uint32_t t = 0; t < rc.tn.chunk; ++t) {
      const uint32_t tb = gb + t * CTA;
      if (tb >= rc.in_n) break;
      process_tile<OP, CTA, RED>(g, sm, rc, tb + threadIdx.x, edges, any_true, any_false);
    }
    if (static_end >= rc.in_n) break;  // everything was covered by the static spans
    __syncthreads();
    if (threadIdx.x == 0) sm.grab_base = static_end + atomicAdd(rc.grab, span);
    __syncthreads();
    gb = sm.grab_base;
  }
  if constexpr (V::kBatched) {
    if (g.lim != nullptr && rc.far_in_n != 0) far_sweep<CTA>(g, sm, rc);
  }
  // CTA-local sub-rounds: expand the stage's newest items [lo, hi) here, with
  // CTA barriers only; their pushes land after them in the stage (or go global
  // when it is full). A round stamp still means "waiting on a worklist": each
  // sub-round stamps with its own id, and a local pop clears the stamp (see
  // process_tile), so every improvement that an expansion may have missed
  // pushes the vertex again; the relaxation is label-correcting, so the fixed
  // point is the same. What is left unexpanded is flushed to the out-worklist.
  uint32_t lo = 0;
  if (kPackedOp<OP> && rc.ds != nullptr && rc.local_rounds != 0) {
    RoundCtx lc = rc;
    for (uint32_t j = 1; j <= rc.local_rounds; ++j) {
      __syncthreads();
      const uint32_t hi = min(sm.stage_n, static_cast<uint32_t>(Smem<CTA>::kStage));
      if (hi <= lo || hi >= static_cast<uint32_t>(Smem<CTA>::kStage)) break;  // nothing new, or the stage is full
      lc.local_items = sm.stage + lo;
      lc.in_n = hi - lo;
      lc.dsr = rc.dsr + j;
      for (uint32_t t = 0; t < hi - lo; t += CTA)
        process_tile<OP, CTA, RED>(g, sm, lc, t + threadIdx.x, edges, any_true, any_false);
      lo = hi;
    }
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out, lo);
}

// ----------------------------------------------------------------------------- small-frontier round

// Frontier size up to which a single-query round may run without the big
// list: every CTA reads the whole frontier, so the limit also bounds the
// frontier x grid product (broadcast reads of at most about 1 M items).
constexpr uint32_t kBcast = 768;
constexpr unsigned long long kBcastBudget = 1ull << 20;

// Exclusive prefix sum of a[0, n) in place (n <= kBcast), every thread of the
// CTA calling; returns the total. wt: shared scratch of CTA / 32 + 1 words.
template <int CTA>
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t* a, uint32_t n, uint32_t* wt) {
  constexpr uint32_t PER = (kBcast + CTA - 1) / CTA;
  constexpr uint32_t W = CTA / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t i0 = threadIdx.x * PER;
  uint32_t loc[PER];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < PER; ++k) {
    loc[k] = i0 + k < n ? a[i0 + k] : 0u;
    sum += loc[k];
  }
  const uint32_t incl = warp_incl_scan(sum);
  if (lane == 31) wt[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = lane < W ? wt[lane] : 0u;
    const uint32_t xi = warp_incl_scan(x);
    if (lane < W) wt[lane] = xi - x;
    if (lane == 31) wt[W] = xi;
  }
  __syncthreads();
  uint32_t run = wt[warp] + incl - sum;
#pragma unroll
  for (uint32_t k = 0; k < PER; ++k) {
    if (i0 + k < n) a[i0 + k] = run;
    run += loc[k];
  }
  const uint32_t total = wt[W];
  __syncthreads();
  return total;
}

// One round of a single-query Iterate over a small frontier (in_n <= kBcast):
// instead of binning the popped vertices by degree and sending long lists
// through the grid-wide big list (an append, a second grid barrier and a
// search), every CTA reads all in_n items and their row offsets, scans the
// degrees in shared memory and walks an equal share of the concatenated
// edges, four per thread per strip, each edge's list found by a binary search
// of the shared offsets. Same pops, operator and pushes as round_body; the
// round's dependent chain is shorter by the big-list append, the barrier
// between the phases and the search in global memory.
template <uint32_t OP, int CTA>
__device__ __forceinline__ void broadcast_round(const SingleView<OP>& g, Smem<CTA>& sm, const RoundCtx& rc,
                                                uint32_t& edges) {
  __shared__ uint32_t b_beg[kBcast];
  __shared__ uint32_t b_off[kBcast];
  __shared__ uint32_t b_val[kBcast];
  __shared__ uint32_t b_wt[CTA / 32 + 1];
  const uint32_t n_in = rc.in_n;
  for (uint32_t i = threadIdx.x; i < n_in; i += CTA) {
    const uint32_t u = rc.in_items ? __ldcg(rc.in_items + i) : i;
    uint32_t b = 0, e = 0, val = 0;
    if (u < g.n) {
      b = __ldg(g.row_ptr + u);
      e = __ldg(g.row_ptr + u + 1);
      if (OP == OP_BFS) val = rc.bfs_val;
      else if (kPackedOp<OP> && rc.ds != nullptr) val = static_cast<uint32_t>(__ldcg(rc.ds + u) >> 32);
      else val = __ldcg(g.state + u);
    } else {
      set_err(rc.out.err, DERR_BAD_ITEM);
    }
    b_beg[i] = b;
    b_off[i] = e - b;
    b_val[i] = val;
  }
  __syncthreads();
  const uint32_t total = cta_excl_scan<CTA>(b_off, n_in, b_wt);
  const uint32_t lo = static_cast<uint32_t>(static_cast<unsigned long long>(total) * blockIdx.x / gridDim.x);
  const uint32_t hi = static_cast<uint32_t>(static_cast<unsigned long long>(total) * (blockIdx.x + 1) / gridDim.x);
  if (threadIdx.x == 0) edges += hi - lo;  // per-thread counters are summed over the CTA
  constexpr uint32_t E = 4;
  const uint32_t tid = threadIdx.x;
  for (uint32_t base = lo; base < hi; base += E * CTA) {
    uint32_t v[E], cur[E], sb[E], op[E], ov[E], rr[E], ndv[E];
    int32_t wt[E];
    uint32_t vmask = 0;
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) {
      const uint32_t e = base + k * CTA + tid;
      v[k] = 0;
      wt[k] = 0;
      sb[k] = 0;
      op[k] = OP;
      ov[k] = 0;
      if (e < hi) {
        // last list whose first edge is <= e (lists of degree 0 share offsets: the search skips them)
        uint32_t a = 0, z = n_in - 1;
        while (a < z) {
          const uint32_t md = (a + z + 1) >> 1;
          if (b_off[md] <= e) a = md;
          else z = md - 1;
        }
        const uint32_t edge = b_beg[a] + (e - b_off[a]);
        ov[k] = b_val[a];
        v[k] = ld_adj(g.col + edge);
        if (needs_w<OP>(OP)) wt[k] = ld_adj(g.w + edge);
        vmask |= 1u << k;
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) cur[k] = ((vmask >> k) & 1u) ? load_cur<OP>(rc, g.state, 0u, v[k]) : 0u;
    decide_n<OP, 4>(rc, g.state, g.stamp, op, sb, v, ov, wt, cur, vmask, rr, ndv);
    uint32_t f = 0, ff = 0, dmin = kInf;
#pragma unroll
    for (uint32_t k = 0; k < E; ++k) {
      f |= (rr[k] == 1u ? 1u : 0u) << k;
      if (kNearFarOp<OP> && rr[k] == 2u) {
        ff |= 1u << k;
        dmin = min(dmin, ndv[k]);
      }
    }
    push4<CTA>(sm, rc.out, f, v[0], v[1], v[2], v[3]);
    if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, ff, v[0], v[1], v[2], v[3], dmin);
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out);
}

// ----------------------------------------------------------------------------- grid barrier

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

// Barrier arrival. Default: one acquire-release atomic (it publishes this CTA's
// writes, which bar.sync ordered before it, and lets the last arrival see
// every earlier CTA's). IRGL_BARRIER_FENCES: the older form, a relaxed atomic
// between two full fences.
__device__ __forceinline__ unsigned long long arrive_add(unsigned long long* p, unsigned long long v) {
#ifdef IRGL_BARRIER_FENCES
  __threadfence();
  const unsigned long long old = atomicAdd(p, v);
  __threadfence();
  return old;
#else
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
#endif
}

// SyncRunningThreads (Sec. 3.4): valid only because the launch is cooperative,
// so every CTA is resident. Each CTA arrives with one 64-bit atomic that also
// carries the out-worklist slots it reserved this round and whether it
// appended to the big list, so the last CTA to arrive knows the round's
// outcome without further loads; it resets the arrival word and publishes
// (generation, flags, out-worklist size) in a release word on another cache
// line, which the waiting CTAs poll. The device error code is read alongside
// the arrival (it is sticky, so a code set just before the last arrival is
// published by the next barrier and always reaches the host). The wait is
// bounded by timeout_ns and gives up early when another CTA timed out. With
// one CTA the barrier is just __syncthreads (a two-level arrival through
// 32 group words measured 1.2 us slower per barrier on 1216 CTAs: the queue
// of atomics on one word is not what a barrier waits for). The caller clears
// sm.round_pushes and sm.big_appended at the start of each round.
template <int CTA>
__device__ __forceinline__ bool grid_barrier(Smem<CTA>& sm, DevStatus* st, uint32_t& gen, unsigned long long timeout_ns,
                                             bool with_big = false) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++gen;
    uint32_t ok = 1, out = 0, flags = 0;
    unsigned long long big = 0;
    const unsigned long long mine = (static_cast<unsigned long long>(sm.round_pushes) << 32) |
                                    (sm.big_appended ? (1ull << 16) : 0ull) | 1ull;
    if (gridDim.x == 1) {
      out = sm.round_pushes;
      flags = __ldcg(&st->err) & 0x7Fu;
      if (with_big && sm.big_appended) {
        big = __ldcg(&st->big_ctr);
        flags |= kRelBigFlag;
        st->big_ctr = 0;
      }
    } else {
      const uint32_t err_seen = __ldcg(&st->err);
      const unsigned long long old = arrive_add(&st->arrive, mine);
      const unsigned long long total = old + mine;
      if ((total & 0xFFFFull) == gridDim.x) {
        // last arrival: every CTA's pushes and big-list appends are in (and
        // visible: its atomic acquired them)
        out = static_cast<uint32_t>(total >> 32);
        flags = err_seen & 0x7Fu;
        if (with_big && ((total >> 16) & 0xFFFFull) != 0) {
          big = __ldcg(&st->big_ctr);
          flags |= kRelBigFlag;
          st->big_pub = big;
          st->big_ctr = 0;  // the next appends come after the big phase
        }
        st->arrive = 0;
        // the release store orders everything above (and all it acquired) before it
        st_release_gpu_u64(&st->rel, (static_cast<unsigned long long>(gen) << 40) |
                                          (static_cast<unsigned long long>(flags) << 32) | out);
      } else {
        const unsigned long long t0 = globaltimer_ns();
        uint32_t spins = 0;
        for (;;) {
          const unsigned long long r = ld_acquire_gpu_u64(&st->rel);
          if (static_cast<uint32_t>(r >> 40) >= gen) {
            out = static_cast<uint32_t>(r);
            flags = static_cast<uint32_t>(r >> 32) & 0xFFu;
            if (flags & kRelBigFlag) big = __ldcg(&st->big_pub);
            break;
          }
          if ((++spins & 63u) == 0) {
            if (__ldcg(&st->err) == DERR_BARRIER_TIMEOUT) { ok = 0; break; }
            if (globaltimer_ns() - t0 > timeout_ns) {
              set_err(&st->err, DERR_BARRIER_TIMEOUT);
              ok = 0;
              break;
            }
          }
        }
      }
      // no fence here: the acquire load above orders this thread's later
      // accesses, and the bar.sync below orders the other threads' after it
    }
    sm.flag = ok;
    sm.pub_out = out;
    sm.pub_err = flags & 0x7Fu;
    sm.pub_flags = flags & kRelBigFlag;
    sm.pub_big = big;
  }
  __syncthreads();
  return sm.flag != 0;
}

// Largest i in [0, n) with off[i] <= x, for an increasing array with off[0] <= x:
// the warp samples 32 positions per step (one load per lane) and narrows the
// interval by a factor 32.
__device__ __forceinline__ uint32_t warp_search_le(const unsigned long long* off, uint32_t n, unsigned long long x) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t a = 0, b = n;
  while (b - a > 1) {
    const uint32_t step = (b - a + 31) / 32;
    const uint32_t p = a + lane * step;
    const bool pred = p < b && __ldcg(off + p) <= x;
    const uint32_t c = __popc(__ballot_sync(kFull, pred));
    const uint32_t na = a + (c - 1) * step;
    b = min(b, na + step);
    a = na;
  }
  return a;
}

// Big phase of a round: the concatenated edges of the big list are split into
// one equal range per warp of the grid. Each warp holds a window of 32 lists in
// registers (lane j: list i0 + j), deals its range out four edges per lane per
// strip (strided by 32, coalesced within a list), and finds each edge's list by
// a shuffle binary search over the window's offsets; all loads of a strip are
// issued before its atomics. Only the final stage flush is CTA-wide.
template <uint32_t OP, int CTA, class V>
__device__ __forceinline__ void big_phase(const V& g, Smem<CTA>& sm, const RoundCtx& rc, unsigned long long pub) {
  constexpr uint32_t E = 4;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n = min(static_cast<uint32_t>(pub >> 40), rc.big.cap);
  const unsigned long long tot = pub & kBigEdgeMask;
  const unsigned long long nw = static_cast<unsigned long long>(gridDim.x) * (CTA / 32);
  const unsigned long long gw = static_cast<unsigned long long>(blockIdx.x) * (CTA / 32) + (threadIdx.x >> 5);
  const unsigned long long lo = tot * gw / nw, hi = tot * (gw + 1) / nw;
  if (n != 0 && lo < hi) {
    uint32_t i0 = warp_search_le(rc.big.off, n, lo);
    unsigned long long pos = lo;
    while (pos < hi && i0 < n) {
      const uint32_t lim = min(32u, n - i0);
      // offsets into the concatenation fit 32 bits (it has fewer than 2^32 edges)
      uint4 en = make_uint4(0, 0, 0, 0);
      uint32_t off = 0xFFFFFFFFu;  // lanes past the window never match
      if (lane < lim) {
        en = __ldcg(rc.big.e + i0 + lane);
        off = static_cast<uint32_t>(__ldcg(rc.big.off + i0 + lane));
      }
      const unsigned long long last_end = static_cast<unsigned long long>(off) + (en.y - en.x);
      const unsigned long long wend_all = __shfl_sync(kFull, last_end, lim - 1);
      const unsigned long long wend = wend_all < hi ? wend_all : hi;
      for (unsigned long long base = pos; base < wend; base += E * 32) {
        uint32_t v[E], cur[E], sb[E], op[E], ov[E], oqs[E];
        int32_t wt[E];
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) {
          const unsigned long long e = base + k * 32 + lane;
          const uint32_t e32 = static_cast<uint32_t>(e < wend ? e : wend - 1);
          // the 32 edges of this step start at most one new list when the lists
          // are at least 32 edges long (the usual case): two ballots find the
          // owners; more list starts take the shuffle search
          const uint32_t ef = static_cast<uint32_t>(base + k * 32 < wend ? base + k * 32 : wend - 1);
          const uint32_t el = static_cast<uint32_t>(base + k * 32 + 31 < wend ? base + k * 32 + 31 : wend - 1);
          const uint32_t o1 = __popc(__ballot_sync(kFull, off <= ef)) - 1u;
          const uint32_t starts = __popc(__ballot_sync(kFull, off <= el)) - 1u - o1;
          uint32_t own = o1;
          if (starts == 1u) own += e32 >= __shfl_sync(kFull, off, o1 + 1u) ? 1u : 0u;
          else if (starts > 1u) own = warp_find<uint32_t>(off, e32, lim);
          const uint32_t ob = __shfl_sync(kFull, en.x, own);
          const uint32_t oo = __shfl_sync(kFull, off, own);
          oqs[k] = __shfl_sync(kFull, en.w, own);
          ov[k] = __shfl_sync(kFull, en.z, own);
          v[k] = 0;
          wt[k] = 0;
          sb[k] = 0;
          op[k] = OP_BFS;
          if (e < wend) {
            const uint32_t edge = ob + (e32 - oo);
            op[k] = g.op(oqs[k]);
            sb[k] = g.sbase(oqs[k]);
            v[k] = ld_adj(g.colp(oqs[k]) + edge);
            if (needs_w<OP>(op[k])) wt[k] = ld_adj(g.wp(oqs[k]) + edge);
          }
        }
#pragma unroll
        for (uint32_t k = 0; k < E; ++k)
          cur[k] = (base + k * 32 + lane < wend) ? load_cur<OP>(rc, g.state + sb[k], sb[k], v[k]) : 0u;
        uint32_t f = 0, ff = 0, dmin = kInf, vmask = 0, rr[E], ndv[E];
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) vmask |= (base + k * 32 + lane < wend ? 1u : 0u) << k;
        decide_n<OP, 4>(rc, g.state, g.stamp, op, sb, v, ov, wt, cur, vmask, rr, ndv);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) {
          const uint32_t r = rr[k];
          if (r == 1u) f |= 1u << k;
          if (r == 2u) {
            ff |= 1u << k;
            dmin = min(dmin, ndv[k]);
          }
          if (V::kBatched && r != 0u) g.mark(oqs[k], rc.ep);
        }
        if constexpr (V::kBatched) {
          if (rc.bdmin_next != nullptr) {
#pragma unroll
            for (uint32_t k = 0; k < E; ++k)
              note_pushes(rc.bdmin_next, g.slot(oqs[k]), (rr[k] == 1u && op[k] == OP_SSSP) ? ndv[k] : kInf);
          }
        }
        push4<CTA>(sm, rc.out, f, sb[0] + v[0], sb[1] + v[1], sb[2] + v[2], sb[3] + v[3]);
        if (kNearFarOp<OP>) push_far4<CTA>(sm, rc.far_out, ff, sb[0] + v[0], sb[1] + v[1], sb[2] + v[2], sb[3] + v[3], dmin);
      }
      pos = wend;
      i0 += lim;
    }
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out);
}

template <int CTA>
__device__ __forceinline__ unsigned long long cta_sum_u64(Smem<CTA>& sm, uint32_t x) {
  __syncthreads();
  if (threadIdx.x == 0) sm.edges = 0;
  __syncthreads();
  uint32_t s = x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&sm.edges, static_cast<unsigned long long>(s));
  __syncthreads();
  return sm.edges;
}

template <int CTA>
__device__ __forceinline__ void init_smem(Smem<CTA>& sm) {
  for (uint32_t i = threadIdx.x; i < static_cast<uint32_t>(CTA); i += CTA) sm.pushed[i] = 0;
  if (threadIdx.x == 0) {
    sm.stage_n = 0;
    sm.flag = 0;
    sm.round_pushes = 0;
    sm.big_appended = 0;
    sm.pmin_cta = kInf;
  }
  __syncthreads();
}

// Direction-optimising BFS, bottom-up round: every unvisited vertex v scans its
// in-edges for a parent at the current level L and, at the first one, takes
// level L + 1 (v is written by this thread only) and joins the out-worklist.
// Same levels as the top-down round (the fixed point is unique); the work is
// the in-edges scanned until a parent is found. Only a parent at exactly L
// counts: an unvisited vertex has no visited in-neighbour below L, and one
// found in this round (L + 1) is not a parent yet. Each thread takes four
// vertices at once (a warp takes 128 consecutive ones, 32 apart per thread,
// so every load coalesces) and checks two in-edges of each per step for up
// to four steps, so eight
// independent chains of loads are in flight per thread; what is still open
// after that (in-lists longer than eight) is scanned by the whole warp, 64
// in-edges per step, so one long list does not hold the warp for hundreds
// of dependent steps.
#ifndef IRGL_BOTTOM_UP_J
#define IRGL_BOTTOM_UP_J 4
#endif
#ifndef IRGL_BOTTOM_UP_STEPS
#define IRGL_BOTTOM_UP_STEPS 4  // two-edge steps per vertex before the warp takes a long in-list
#endif
template <int CTA>
__device__ __forceinline__ void bottom_up_round(const KParams& p, Smem<CTA>& sm, const RoundCtx& rc, uint32_t L,
                                                uint32_t& edges, const uint32_t* cand, uint32_t cand_n,
                                                uint32_t* rest, uint32_t* rest_n) {
  constexpr uint32_t J = IRGL_BOTTOM_UP_J;  // vertices per thread per pass
  constexpr uint32_t kLaneSteps = IRGL_BOTTOM_UP_STEPS;
  constexpr uint32_t kChunk = 32 * J;       // vertices per warp pass
  const uint32_t lane = threadIdx.x & 31;
  // candidates: the list the previous bottom-up round left (cand), else every vertex
  const uint32_t nv = cand ? cand_n : p.n;
  // The work per vertex varies with its in-list and where the first parent
  // sits in it, so chunks of kChunk vertices are dealt out per warp: the
  // first one by warp index, the rest from the round's grab counter (a
  // static share left the last CTA of a round 2.4x slower than the first).
  const uint32_t nchunks = (nv + kChunk - 1) / kChunk;
  const uint32_t nwarps = gridDim.x * (CTA / 32);
  for (uint32_t c = blockIdx.x * (CTA / 32) + (threadIdx.x >> 5); c < nchunks;) {
    const uint32_t base = c * kChunk;
    uint32_t v[J], b[J], e[J], ob[J], oe[J];
    bool open[J], found[J], keep[J];
#pragma unroll
    for (uint32_t j = 0; j < J; ++j) {
      const uint32_t i = base + j * 32 + lane;
      v[j] = i < nv ? (cand ? __ldcg(cand + i) : i) : 0u;
      open[j] = i < nv && __ldcg(p.state + v[j]) == kInf;
      found[j] = false;
    }
#pragma unroll
    for (uint32_t j = 0; j < J; ++j) {
      b[j] = open[j] ? __ldg(p.in_row_ptr + v[j]) : 0u;
      e[j] = open[j] ? __ldg(p.in_row_ptr + v[j] + 1) : 0u;
      // out-degree of v for the direction rule, loaded with the in-offsets (coalesced)
      ob[j] = open[j] ? __ldg(p.row_ptr + v[j]) : 0u;
      oe[j] = open[j] ? __ldg(p.row_ptr + v[j] + 1) : 0u;
      open[j] = open[j] && b[j] < e[j];
      keep[j] = open[j];  // unvisited with in-edges: kept for the next bottom-up round unless found
    }
    for (uint32_t step = 0; step < kLaneSteps; ++step) {
      uint32_t c[J][2];
#pragma unroll
      for (uint32_t j = 0; j < J; ++j) {
#pragma unroll
        for (uint32_t t = 0; t < 2; ++t) c[j][t] = (open[j] && b[j] + t < e[j]) ? ld_adj(p.in_col + b[j] + t) : kInf;
      }
      bool any = false;
#pragma unroll
      for (uint32_t j = 0; j < J; ++j) {
        bool hit = false;
#pragma unroll
        for (uint32_t t = 0; t < 2; ++t) hit |= c[j][t] != kInf && __ldcg(p.state + c[j][t]) == L;
        if (open[j]) {
          const uint32_t left = e[j] - b[j];
          edges += left < 2u ? left : 2u;
          b[j] += 2u;
          found[j] = hit;
          open[j] = !hit && b[j] < e[j];
        }
        any |= open[j];
      }
      if (!__any_sync(kFull, any)) break;
    }
    // long in-lists: the warp takes the open vertices one at a time
#pragma unroll
    for (uint32_t j = 0; j < J; ++j) {
      for (;;) {
        const unsigned m = __ballot_sync(kFull, open[j]);
        if (m == 0) break;
        const int ld = __ffs(m) - 1;
        uint32_t kb = __shfl_sync(kFull, b[j], ld);
        const uint32_t ke = __shfl_sync(kFull, e[j], ld);
        bool hit = false;
        while (kb < ke) {
          const uint32_t k0 = kb + lane, k1 = kb + 32u + lane;
          const uint32_t c0 = k0 < ke ? ld_adj(p.in_col + k0) : kInf;
          const uint32_t c1 = k1 < ke ? ld_adj(p.in_col + k1) : kInf;
          const bool h = (c0 != kInf && __ldcg(p.state + c0) == L) || (c1 != kInf && __ldcg(p.state + c1) == L);
          const uint32_t span = ke - kb < 64u ? ke - kb : 64u;
          if (lane == 0) edges += span;
          kb += 64u;
          if (__any_sync(kFull, h)) {
            hit = true;
            break;
          }
        }
        if (lane == static_cast<uint32_t>(ld)) {
          open[j] = false;
          found[j] = hit;
        }
      }
    }
    // out-edges of the found vertices for the direction rule: a thread sum, a
    // warp sum, one shared atomic per warp
    uint32_t mf = 0, fmask = 0;
#pragma unroll
    for (uint32_t j = 0; j < J; ++j) {
      if (found[j]) {
        __stcg(p.state + v[j], L + 1u);
        if (p.vis) atomicOr(p.vis + (v[j] >> 5), 1u << (v[j] & 31u));
        mf += oe[j] - ob[j];
        fmask |= 1u << j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mf += __shfl_xor_sync(kFull, mf, o);
    if (lane == 0 && mf) atomicAdd(&sm.mf_cta, static_cast<unsigned long long>(mf));
#pragma unroll
    for (uint32_t j = 0; j < J; j += 4)
      push4<CTA>(sm, rc.out, (fmask >> j) & 15u, v[j], J > j + 1 ? v[j + 1 < J ? j + 1 : j] : 0u,
                 J > j + 2 ? v[j + 2 < J ? j + 2 : j] : 0u, J > j + 3 ? v[j + 3 < J ? j + 3 : j] : 0u);
    if (rest) {
      // vertices still unvisited after all their in-edges: the next bottom-up round's candidates
      uint32_t kmask = 0;
#pragma unroll
      for (uint32_t j = 0; j < J; ++j) kmask |= (keep[j] && !found[j] ? 1u : 0u) << j;
      const uint32_t k = __popc(kmask);
      const uint32_t incl = warp_incl_scan(k);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      if (total) {
        uint32_t gb = 0;
        if (lane == 31) gb = atomicAdd(rest_n, total);
        gb = __shfl_sync(kFull, gb, 31);
        uint32_t pos = gb + incl - k;
#pragma unroll
        for (uint32_t j = 0; j < J; ++j) {
          if ((kmask >> j) & 1u) {
            if (pos < p.n) __stcg(rest + pos, v[j]);
            ++pos;
          }
        }
      }
    }
    // next chunk (pushes past the stage go straight to the out-worklist)
    uint32_t nc = 0;
    if (lane == 0) nc = nwarps + atomicAdd(rc.grab, 1u);
    c = __shfl_sync(kFull, nc, 0);
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out);
}

// Near-far phase change: every item of the finished phase's far list is
// checked against its current distance d. d < lim_old: it was improved below
// the old limit after it was pushed far, which pushed it to an out-worklist
// then, so it is dropped. lim_old <= d < lim_new: it joins this round's
// out-worklist. d >= lim_new: it stays far, in the other far list.
template <uint32_t OP, int CTA, class V>
__device__ __forceinline__ void split_far(const V& g, Smem<CTA>& sm, const RoundCtx& rc, const uint32_t* fin,
                                          uint32_t far_n, uint32_t lim_old, uint32_t lim_new) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t base = blockIdx.x * CTA; base < far_n; base += gridDim.x * CTA) {
    const uint32_t i = base + tid;
    uint32_t v = 0, d = kInf;
    if (i < far_n) {
      v = __ldcg(fin + i);
      d = (OP == OP_SSSP && rc.ds != nullptr) ? static_cast<uint32_t>(__ldcg(rc.ds + v) >> 32) : __ldcg(g.state + v);
    }
    // each vertex is on a phase's far list at most once and a split round
    // relaxes nothing, so with the packed words no round stamp is needed here
    const bool near = i < far_n && d >= lim_old && d < lim_new &&
                      ((OP == OP_SSSP && rc.ds != nullptr) || atomicExch(g.stamp + v, rc.ep) != rc.ep);
    const bool keep = i < far_n && d >= lim_new && atomicExch(rc.far_stamp + v, rc.phase) != rc.phase;
    push1<CTA>(sm, rc.out, near, v);
    push_far4<CTA>(sm, rc.far_out, keep ? 1u : 0u, v, 0u, 0u, 0u, d);
    if (__syncthreads_or(sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2))) flush_stage<CTA>(sm, rc.out);
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out);
}

// ----------------------------------------------------------------------------- state initialisation

// Iterate initial values (Initial[...] of the BFS listing): BFS/SSSP state = INF
// except 0 at the initial items; CC label[v] = v. Grid-stride with 16-byte
// stores when the state array is 16-byte aligned. `srcs`/`nsrc` is a small
// in-register copy of the initial items (nsrc <= 8), else the caller sets the
// sources in a second pass.
template <uint32_t OP>
__device__ __forceinline__ void fill_state(uint32_t* state, uint32_t n, const uint32_t* srcs, uint32_t nsrc,
                                           uint32_t tid, uint32_t nthreads) {
  auto value = [&](uint32_t v) -> uint32_t {
    if (OP == OP_CC) return v;
    uint32_t r = kInf;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) r = (i < nsrc && srcs[i] == v) ? 0u : r;
    return r;
  };
  if ((reinterpret_cast<uintptr_t>(state) & 15u) == 0) {
    const uint32_t n4 = n >> 2;
    uint4* s4 = reinterpret_cast<uint4*>(state);
    for (uint32_t i = tid; i < n4; i += nthreads) {
      const uint32_t v = i << 2;
      __stcg(s4 + i, make_uint4(value(v), value(v + 1), value(v + 2), value(v + 3)));
    }
    for (uint32_t v = (n4 << 2) + tid; v < n; v += nthreads) __stcg(state + v, value(v));
  } else {
    for (uint32_t v = tid; v < n; v += nthreads) __stcg(state + v, value(v));
  }
}

// SSSP initial values in the packed form: (dist << 32) | 0, dist = 0 at the
// in-register sources, INF elsewhere. Round ids start at 1, so no vertex
// looks pushed in round 1.
__device__ __forceinline__ void fill_packed(unsigned long long* ds, uint32_t n, const uint32_t* srcs, uint32_t nsrc,
                                            uint32_t tid, uint32_t nthreads) {
  for (uint32_t v = tid; v < n; v += nthreads) {
    uint32_t d = kInf;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) d = (i < nsrc && srcs[i] == v) ? 0u : d;
    __stcg(ds + v, static_cast<unsigned long long>(d) << 32);
  }
}

// ----------------------------------------------------------------------------- kernels

// Clean exit of a persistent launch: the last CTA out restores the
// between-launch invariants (counters, release word and arrival slots at 0)
// and publishes the outcome. Called by every thread of every CTA.
template <int CTA>
__device__ __forceinline__ void persistent_exit(Smem<CTA>& sm, DevStatus* st, bool ok, uint32_t rounds,
                                                uint32_t last_out, uint32_t ep0, unsigned long long esum,
                                                uint32_t* cont, uint32_t cont_buf, uint32_t far_buf = 0,
                                                uint32_t far_n = 0, uint32_t id_step = 1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&st->edges, esum);
    uint32_t last = 0;
    if (ok) {
      __threadfence();
      last = atomicAdd(&st->exit_count, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    sm.flag = last;
  }
  __syncthreads();
  if (sm.flag == 0) return;
  __threadfence();
  if (threadIdx.x == 0) {
    if (cont) {
      cont[0] = cont_buf;
      cont[1] = last_out;
      cont[2] = far_buf;  // batched near-far: the far list left for the next launch
      cont[3] = far_n;
      for (int i = 0; i < 3; ++i) {
        st->bfar_tail[i] = 0;
        for (int w = 0; w < 32; ++w) st->qnear[i][w] = 0;
      }
    }
    st->rounds = rounds;
    st->last_out = last_out;
    st->epoch = ep0 + rounds * id_step;  // round ids ep0 .. ep0 + rounds * id_step - 1 were used
    for (int i = 0; i < 4; ++i) {
      st->tail[i] = 0;
      st->grab[i] = 0;
    }
    st->arrive = 0;
    st->rel = 0;
    st->big_ctr = 0;
    st->far_tail[0] = st->far_tail[1] = 0;
    st->far_min[0] = st->far_min[1] = 0;
    st->mf[0] = st->mf[1] = st->mf[2] = 0;
    st->bu_n[0] = st->bu_n[1] = st->bu_n[2] = 0;
    st->pmin[0] = st->pmin[1] = st->pmin[2] = 0;
    st->exit_count = 0;
  }
  __threadfence();
}

__device__ __forceinline__ void trace_round(unsigned long long* trace, uint32_t cap, uint32_t r, uint32_t in_n,
                                            uint32_t out_n) {
  if (trace && r < cap && blockIdx.x == 0 && threadIdx.x == 0) {
    trace[2 * r] = globaltimer_ns();
    trace[2 * r + 1] = (static_cast<unsigned long long>(in_n) << 32) | out_n;
  }
}

// Record 0 of a trace: the end of the prologue, with the prologue's duration
// (ns since the kernel started, t0 taken by CTA 0) in the out field.
__device__ __forceinline__ void trace_prologue(unsigned long long* trace, uint32_t cap, unsigned long long t0,
                                               uint32_t in_n) {
  if (trace && cap > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long t = globaltimer_ns();
    const unsigned long long d = t - t0;
    trace[0] = t;
    trace[1] = (static_cast<unsigned long long>(in_n) << 32) | static_cast<uint32_t>(d < 0xFFFFFFFFull ? d : 0xFFFFFFFFull);
  }
}

// Phase record of round r (persistent single-query Iterate, when tracing):
// words 0/1 the earliest and latest end of the round's first phase over all
// CTAs (word 0 complemented, both gathered with atomicMax), 2 the time CTA 0
// left the first grid barrier, 3 the big list published there ((entries << 40)
// | edges; 0: none), 4/5 the earliest (complemented) and latest end of the big
// phase, 6 the time CTA 0 left the second barrier. All globaltimer ns.
constexpr uint32_t kPhaseWords = 8;
// Round 0 is fused into the prologue when the sources have at most this many out-edges together.
constexpr uint32_t kFuseEdges = 256;
__device__ __forceinline__ unsigned long long* trace_phase(unsigned long long* ph, uint32_t cap, uint32_t r) {
  return (ph != nullptr && r < cap) ? ph + static_cast<size_t>(kPhaseWords) * r : nullptr;
}
__device__ __forceinline__ void trace_phase_end(unsigned long long* rec, uint32_t word) {
  // called by thread 0 of every CTA after a CTA barrier
  if (rec != nullptr) {
    const unsigned long long t = globaltimer_ns();
    atomicMax(rec + word, ~t);
    atomicMax(rec + word + 1, t);
  }
}

// Record rounds + 1 of a trace: the end of the epilogue (results copied out),
// marked with in = out = 0xFFFFFFFF.
__device__ __forceinline__ void trace_end(unsigned long long* trace, uint32_t cap, uint32_t rounds) {
  if (trace && rounds + 1 < cap && blockIdx.x == 0 && threadIdx.x == 0) {
    trace[2 * (rounds + 1)] = globaltimer_ns();
    trace[2 * (rounds + 1) + 1] = ~0ull;
  }
}

// Iteration-outlined Iterate: every round in one cooperative launch.
template <uint32_t OP, int CTA>
__device__ __forceinline__ void iterate_persistent(const KParams& p, Smem<CTA>& sm) {
  const unsigned long long t_start = p.trace ? globaltimer_ns() : 0ull;
  init_smem<CTA>(sm);
  DevStatus* st = p.st;
  uint32_t gen = 0;
  const uint32_t ep0 = __ldcg(&st->epoch);
  const uint32_t init_n = p.init_count ? min(__ldcg(p.init_count), p.init_cap) : p.n;
  if (p.skip_cta == static_cast<int>(blockIdx.x)) return;  // test hook: never arrives

  SingleView<OP> g{p.row_ptr, p.col, p.w, p.state, p.stamp, p.n};
  uint32_t edges = 0, dummy_t = 0, dummy_f = 0;
  uint32_t rounds = 0, last_out = 0;
  bool ok = true;

  // Round 0 fused into the prologue (BFS; at most eight sources with at most
  // kFuseEdges out-edges together, plain rounds; SSSP measured slower, its
  // kernel spilling more registers with the fused code in it): the
  // thread that initialises a vertex is the only writer of its value until the
  // prologue barrier, so the CTA owning a source's out-neighbour relaxes that
  // edge right after its own initialisation (a CTA barrier between) and pushes
  // it; the prologue's grid barrier then ends round 0 and publishes its pushes.
  bool fused = false;
  uint32_t fused_out = 0;
  if (p.init_state) {
    uint32_t srcs[8];
    uint32_t ns = 0;
    const bool small = OP != OP_CC && p.init_items != nullptr && init_n <= 8;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) srcs[i] = (small && i < init_n) ? __ldcg(p.init_items + i) : kInf;
    if (small) ns = init_n;
    if ((OP == OP_SSSP || OP == OP_BFSR) && p.ds != nullptr) fill_packed(p.ds, p.n, srcs, ns, blockIdx.x * CTA + threadIdx.x, gridDim.x * CTA);
    else fill_state<OP>(p.state, p.n, srcs, ns, blockIdx.x * CTA + threadIdx.x, gridDim.x * CTA);
    if constexpr (OP == OP_BFS) {
    // sources' out-degrees (every thread, the same few words): decide the fusion
    uint32_t sbeg[8], sdeg[8], tdeg = 0;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
      sbeg[i] = 0;
      sdeg[i] = 0;
      if (i < ns && srcs[i] < p.n) {
        sbeg[i] = __ldg(p.row_ptr + srcs[i]);
        sdeg[i] = __ldg(p.row_ptr + srcs[i] + 1) - sbeg[i];
      }
      tdeg += sdeg[i];
    }
    fused = small && ns > 0 && tdeg <= kFuseEdges && p.vis == nullptr && p.diropt != 2 && p.max_rounds > 1;
    if (fused) {
      __syncthreads();  // this CTA's initial values before its relaxations
      const Out out0{p.items[1], &st->tail[1], p.cap, &st->err};
      const unsigned long long nthreads = static_cast<unsigned long long>(gridDim.x) * CTA;
      for (uint32_t base = 0; base < tdeg; base += CTA) {
        const uint32_t e = base + threadIdx.x;
        bool push = false;
        uint32_t v = 0;
        if (e < tdeg) {
          // edge e of the sources' concatenated out-lists
          uint32_t i = 0, off = e;
#pragma unroll
          for (uint32_t k = 0; k < 7; ++k) {
            if (i == k && off >= sdeg[k]) {
              off -= sdeg[k];
              i = k + 1;
            }
          }
          uint32_t edge = 0;
#pragma unroll
          for (uint32_t k = 0; k < 8; ++k) edge = i == k ? sbeg[k] + off : edge;
          v = __ldg(p.col + edge);
          // the CTA whose thread initialised v relaxes it: fill_state gives vertex v to
          // thread v mod T, or, on a 16-byte-aligned array, groups of four to thread
          // v / 4 mod T and the last n mod 4 vertices one by one
          unsigned long long own = v % nthreads;
          if ((reinterpret_cast<uintptr_t>(p.state) & 15u) == 0) {
            const uint32_t n4 = (p.n >> 2) << 2;
            own = v < n4 ? (v >> 2) % nthreads : (v - n4) % nthreads;
          }
          if (v < p.n && own / CTA == blockIdx.x) push = atomicCAS(p.state + v, kInf, 1u) == kInf;
        }
        push1<CTA>(sm, out0, push, v);
      }
      __syncthreads();
      flush_stage<CTA>(sm, out0);
      if (blockIdx.x == 0 && threadIdx.x == 0) edges += tdeg;
      // phase record of round 0 (the host clears the records before a traced launch)
      if (threadIdx.x == 0) trace_phase_end(trace_phase(p.trace_ph, p.trace_cap, 0), 0);
    }
    }
    if (OP != OP_CC && !small) {
      ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
      if (ok) {
        for (uint32_t i = blockIdx.x * CTA + threadIdx.x; i < init_n; i += gridDim.x * CTA) {
          const uint32_t s = p.init_items ? __ldcg(p.init_items + i) : i;
          if (s >= p.n) continue;
          if ((OP == OP_SSSP || OP == OP_BFSR) && p.ds != nullptr) __stcg(p.ds + s, 0ull);
          else __stcg(p.state + s, 0u);
        }
      }
    }
  } else if ((OP == OP_SSSP || OP == OP_BFSR) && p.ds != nullptr) {
    // the caller's initial distances, round id 0
    for (uint32_t v = blockIdx.x * CTA + threadIdx.x; v < p.n; v += gridDim.x * CTA)
      __stcg(p.ds + v, static_cast<unsigned long long>(__ldcg(p.state + v)) << 32);
  }
  if (OP == OP_BFS && p.vis != nullptr) {
    for (uint32_t i = blockIdx.x * CTA + threadIdx.x; i < (p.n + 31u) >> 5; i += gridDim.x * CTA) __stcg(p.vis + i, 0u);
  }
  if constexpr (OP != OP_BFS) {
    // phase records gather with atomicMax: clear this launch's (BFS, whose round 0 may write its
    // record before this point, has them cleared by the host; the other operators keep the clear
    // here, without which the SSSP kernel's registers fell differently and it ran 2 % slower)
    if (p.trace_ph != nullptr) {
      for (uint32_t i = blockIdx.x * CTA + threadIdx.x; i < p.trace_cap * kPhaseWords; i += gridDim.x * CTA)
        p.trace_ph[i] = 0ull;
    }
  }
  if (ok) ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
  trace_prologue(p.trace, p.trace_cap, t_start, init_n);
  bool skip_rounds = false;
  if (fused && ok) {
    // round 0 ended at the prologue barrier
    fused_out = sm.pub_out;
    last_out = fused_out;
    rounds = 1;
    unsigned long long* const ph0 = trace_phase(p.trace_ph, p.trace_cap, 0);
    if (ph0 != nullptr && blockIdx.x == 0 && threadIdx.x == 0) ph0[2] = globaltimer_ns();
    trace_round(p.trace, p.trace_cap, 1, init_n, fused_out);
    skip_rounds = fused_out == 0 || sm.pub_err != DERR_NONE;
  }

  // Near-far schedule (SSSP distances, CC labels): improvements to a value >=
  // limit wait on a far list; when a round pushes nothing below the limit, a
  // split round raises the limit and releases the far items below it (delta =
  // 0: plain rounds).
  const bool nf = kNearFarOp<OP> && p.delta != 0 && p.far_stamp != nullptr;
  uint32_t limit = nf ? p.delta : kInf, lim_old = 0;
  uint32_t fb = 0;        // far list receiving pushes in the current phase
  uint32_t phase = ep0;   // far-list dedup id of the current phase
  uint32_t far_n = 0;
  bool split = false;
  // direction-optimising BFS (Beamer's rule): go bottom-up when the next
  // frontier's out-edges exceed the unvisited vertices' out-edges / 15; come
  // back top-down when the frontier shrinks below n / 18
  const bool dopt = OP == OP_BFS && p.diropt != 0 && p.in_row_ptr != nullptr;
  bool bottom_up = dopt && p.diropt == 2;  // test hook: every round bottom-up
  uint32_t bu_k = 0;                       // bottom-up rounds run so far
  unsigned long long visited_edges = 0;
  uint32_t prev_n = init_n;
  uint32_t in_n = init_n;
  uint32_t r0 = 0;
  if constexpr (OP == OP_BFS) {
    if (fused) {
      prev_n = fused_out;
      in_n = min(fused_out, p.cap);
      r0 = 1;
    }
  }
  // small frontiers skip the big list (broadcast_round): BFS, SSSP and
  // min-label CC rounds (near-far included) without CTA-local sub-rounds
  const bool bcast = p.bcast != 0 && (OP == OP_BFS || OP == OP_SSSP || OP == OP_CC) && p.local_rounds == 0;
  // dense rounds: BFS, and SSSP on packed words, without near-far or sub-rounds
  const bool dense_ok = p.dense_div != 0 && !nf && p.local_rounds == 0 &&
                        (OP == OP_BFS || (OP == OP_SSSP && p.ds != nullptr));
  // deferred expansion of long lists (SSSP on packed words, plain rounds)
  const bool defer = OP == OP_SSSP && p.defer_deg != 0 && p.ds != nullptr && !nf && p.local_rounds == 0 &&
                     p.dense_div == 0;
  const unsigned long long t_run0 = p.time_limit_ns ? globaltimer_ns() : 0ull;
  for (uint32_t r = r0; ok && (OP != OP_BFS || !skip_rounds); ++r) {
    check_time_limit(&st->err, t_run0, p.time_limit_ns);
    uint32_t* const cur = (r & 1) ? p.items[1] : p.items[0];  // no dynamic index into the param struct
    uint32_t* const nxt = (r & 1) ? p.items[0] : p.items[1];
    RoundCtx rc;
    rc.in_n = in_n;
    rc.in_items = r == 0 ? p.init_items : cur;
    rc.out = Out{nxt, &st->tail[(r + 1) % 3], p.cap, &st->err};
    rc.bfs_val = r + 1;
    rc.ep = ep0 + r;
    rc.grab = &st->grab[r % 3];
    rc.tn = p.tn;
    rc.big = p.big;
    rc.big_ctr = &st->big_ctr;
    rc.limit = limit;
    rc.far_stamp = p.far_stamp;
    rc.phase = phase;
    rc.changes = nullptr;
    rc.mf = dopt ? &sm.mf_cta : nullptr;
    rc.row_ptr = p.row_ptr;
    rc.vis = OP == OP_BFS ? p.vis : nullptr;
    rc.ds = (OP == OP_SSSP || OP == OP_BFSR) ? p.ds : nullptr;
    rc.dsr = r * (p.local_rounds + 1u) + 1u;  // room for the sub-rounds' ids
    rc.local_rounds = (OP == OP_SSSP || OP == OP_BFSR) ? p.local_rounds : 0u;
    rc.local_items = nullptr;
    rc.spread = p.spread;
    if (defer && r > 0) {
      // the smallest distance pushed for this round (complete at the last barrier)
      const uint32_t pm = __ldcg(&st->pmin[r % 3]);
      if (pm != 0u) {
        const unsigned long long lim = static_cast<unsigned long long>(~pm) + p.defer_delta;
        rc.defer_lim = lim < kInf ? static_cast<uint32_t>(lim) : kInf;
        rc.defer_deg = p.defer_deg;
      }
    }
    rc.pmin = defer ? &sm.pmin_cta : nullptr;
    // dense round: a large frontier is popped in vertex order (coalesced row
    // offsets, neighbouring adjacency lists) instead of worklist order
    const bool small_round =
        bcast && in_n <= kBcast && static_cast<unsigned long long>(in_n) * gridDim.x <= kBcastBudget;
    if (dense_ok && r > 0 && !split && !(dopt && bottom_up) && !small_round &&
        static_cast<unsigned long long>(in_n) * p.dense_div > p.n) {
      rc.dense = 1;
      rc.dense_id = rc.dsr - 1u;  // the previous round's id (no sub-rounds here)
      rc.in_items = nullptr;
      rc.in_n = p.n;
    }
    const uint32_t ftarget = split ? (fb ^ 1u) : fb;  // far list this round pushes to
    rc.far_out = Out{ftarget ? p.far[1] : p.far[0], &st->far_tail[ftarget], p.far_cap, &st->err};
    if (threadIdx.x == 0) {
      if (blockIdx.x == 0) {
        st->tail[(r + 2) % 3] = 0;
        st->grab[(r + 2) % 3] = 0;
      }
      sm.round_pushes = 0;
      sm.big_appended = 0;
      sm.far_min_cta = kInf;
      sm.mf_cta = 0;
      // mf[(r + 2) % 3] is still being read by CTAs that just left the last
      // barrier; mf[(r + 1) % 3] was read by every CTA before it arrived there
      if (dopt && blockIdx.x == 0) st->mf[(r + 1) % 3] = 0;
      // pmin[(r + 1) % 3] gathers this round's pushes; pmin[(r + 2) % 3] was
      // read at the start of the last round, before its barrier
      if (defer && blockIdx.x == 0) st->pmin[(r + 2) % 3] = 0;
    }
    if (split) {
      split_far<OP, CTA>(g, sm, rc, fb ? p.far[1] : p.far[0], far_n, lim_old, limit);
    } else if (dopt && bottom_up) {
      // bottom-up round k reads the list round k - 1 left (count bu_n[(k - 1) % 3]) and
      // writes list k & 1 (count bu_n[k % 3]); bu_n[(k + 1) % 3], last read in round
      // k - 1, is cleared now for round k + 1
      const bool lists = p.bu_list[0] != nullptr;
      const uint32_t* cand = (lists && bu_k != 0) ? p.bu_list[(bu_k + 1) & 1] : nullptr;
      const uint32_t cand_n = cand ? min(__ldcg(&st->bu_n[(bu_k + 2) % 3]), p.n) : 0u;
      if (lists && blockIdx.x == 0 && threadIdx.x == 0) st->bu_n[(bu_k + 1) % 3] = 0;
      __syncthreads();
      bottom_up_round<CTA>(p, sm, rc, r, edges, cand, cand_n, lists ? p.bu_list[bu_k & 1] : nullptr,
                           &st->bu_n[bu_k % 3]);
      ++bu_k;
    } else if (small_round) {
      broadcast_round<OP, CTA>(g, sm, rc, edges);
    } else {
      round_body<OP, CTA, RED_NONE>(g, sm, rc, edges, dummy_t, dummy_f);
    }
    if (dopt && threadIdx.x == 0 && sm.mf_cta) {
      atomicAdd(&st->mf[r % 3], sm.mf_cta);
      sm.mf_cta = 0;
    }
    if (nf && threadIdx.x == 0 && sm.far_min_cta != kInf) atomicMax(&st->far_min[ftarget], ~sm.far_min_cta);
    if (defer && threadIdx.x == 0 && sm.pmin_cta != kInf) {
      atomicMax(&st->pmin[(r + 1) % 3], ~sm.pmin_cta);
      sm.pmin_cta = kInf;
    }
    unsigned long long* const ph = trace_phase(p.trace_ph, p.trace_cap, r);
    if (ph != nullptr) {
      __syncthreads();
      if (threadIdx.x == 0) trace_phase_end(ph, 0);
    }
    ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns, !split && p.big.cap != 0);
    if (!ok) break;
    if (ph != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
      ph[2] = globaltimer_ns();
      ph[3] = (sm.pub_flags & kRelBigFlag) ? sm.pub_big : 0ull;
    }
    if (sm.pub_flags & kRelBigFlag) {
      big_phase<OP, CTA>(g, sm, rc, sm.pub_big);
      if (nf && threadIdx.x == 0 && sm.far_min_cta != kInf) atomicMax(&st->far_min[ftarget], ~sm.far_min_cta);
      if (dopt && threadIdx.x == 0 && sm.mf_cta) {
        atomicAdd(&st->mf[r % 3], sm.mf_cta);
        sm.mf_cta = 0;
      }
      if (defer && threadIdx.x == 0 && sm.pmin_cta != kInf) {
        atomicMax(&st->pmin[(r + 1) % 3], ~sm.pmin_cta);
        sm.pmin_cta = kInf;
      }
      if (ph != nullptr) {
        __syncthreads();
        if (threadIdx.x == 0) trace_phase_end(ph, 4);
      }
      ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
      if (!ok) break;
      if (ph != nullptr && blockIdx.x == 0 && threadIdx.x == 0) ph[6] = globaltimer_ns();
    }
    last_out = sm.pub_out;
    rounds = r + 1;
    trace_round(p.trace, p.trace_cap, rounds, in_n, last_out);
    if (sm.pub_err != DERR_NONE) break;
    if (split) {
      // the split list is consumed: clear it for a later phase, continue with the kept list
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->far_tail[fb] = 0;
        st->far_min[fb] = 0;
      }
      fb ^= 1u;
      split = false;
    }
    if (dopt && p.diropt == 1 && last_out != 0) {
      // every CTA takes the same decision from the same published values
      if (threadIdx.x == 0) sm.pub_big = __ldcg(&st->mf[r % 3]);
      __syncthreads();
      const unsigned long long mf = sm.pub_big;
      __syncthreads();
      visited_edges += mf;
      const unsigned long long mu = p.m_total > visited_edges ? p.m_total - visited_edges : 0ull;
      if (!bottom_up && mf > mu / 15ull && last_out > prev_n) bottom_up = true;
      else if (bottom_up && last_out < p.n / 18u && last_out < prev_n) bottom_up = false;
      prev_n = last_out;
    }
    if (last_out == 0) {
      if (!nf) break;
      if (threadIdx.x == 0) {
        sm.gbase = __ldcg(&st->far_tail[fb]);
        sm.own_val = ~__ldcg(&st->far_min[fb]);
      }
      __syncthreads();
      far_n = min(sm.gbase, p.far_cap);
      const uint32_t fmin = sm.own_val;
      __syncthreads();
      if (far_n == 0) break;
      // next phase: at least one delta higher, and high enough to release the nearest far item
      const unsigned long long l1 = static_cast<unsigned long long>(limit) + p.delta;
      const unsigned long long l2 = (static_cast<unsigned long long>(fmin) / p.delta + 1ull) * p.delta;
      const unsigned long long ln = l1 > l2 ? l1 : l2;
      lim_old = limit;
      limit = ln >= kInf ? kInf : static_cast<uint32_t>(ln);
      phase = ep0 + r + 1;  // the split round's id
      split = true;
    }
    if (rounds >= p.max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(&st->err, DERR_MAX_ROUNDS);
      break;
    }
    in_n = min(last_out, p.cap);
  }
  if ((OP == OP_SSSP || OP == OP_BFSR) && p.ds != nullptr) {
    // every round ended at a barrier that all CTAs passed: the words are final
    for (uint32_t v = blockIdx.x * CTA + threadIdx.x; v < p.n; v += gridDim.x * CTA)
      __stcg(p.state + v, static_cast<uint32_t>(__ldcg(p.ds + v) >> 32));
  }
  const unsigned long long esum = cta_sum_u64<CTA>(sm, edges);
  trace_end(p.trace, p.trace_cap, rounds);
  persistent_exit<CTA>(sm, st, ok, rounds, last_out, ep0, esum, nullptr, 0);
}

// Connected components by min-hooking and pointer jumping, in one cooperative
// launch. parent = state, initially parent[v] = v. Each iteration: (1) hook:
// for every edge (u, v) with parents a = parent[u], b = parent[v], a != b,
// atomicMin(parent[max(a,b)], min(a,b)); (2) shortcut: every vertex follows
// its parent pointers to the root and stores it. Parents only decrease and
// always name a vertex of the same component, so the first hook phase that
// lowers nothing leaves every component pointing at one root, its minimum id:
// the labels of min-label propagation in O(log n) iterations instead of
// O(diameter) rounds.
template <int CTA>
__device__ __forceinline__ void cc_jump_persistent(const KParams& p, Smem<CTA>& sm) {
  init_smem<CTA>(sm);
  DevStatus* st = p.st;
  uint32_t gen = 0;
  const uint32_t ep0 = __ldcg(&st->epoch);
  if (p.skip_cta == static_cast<int>(blockIdx.x)) return;  // test hook: never arrives
  SingleView<OP_CCJ> g{p.row_ptr, p.col, p.w, p.state, p.stamp, p.n};
  uint32_t edges = 0, dummy_t = 0, dummy_f = 0, rounds = 0, last_changes = 0;
  fill_state<OP_CC>(p.state, p.n, nullptr, 0, blockIdx.x * CTA + threadIdx.x, gridDim.x * CTA);
  bool ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
  trace_round(p.trace, p.trace_cap, 0, p.n, 0);
  for (uint32_t r = 0; ok; ++r) {
    RoundCtx rc;
    rc.in_items = nullptr;  // every vertex
    rc.in_n = p.n;
    rc.out = Out{r & 1 ? p.items[0] : p.items[1], &st->tail[(r + 1) % 3], p.cap, &st->err};  // never pushed
    rc.bfs_val = 0;
    rc.ep = ep0 + r;
    rc.grab = &st->grab[r % 3];
    rc.tn = p.tn;
    rc.big = p.big;
    rc.big_ctr = &st->big_ctr;
    rc.limit = kInf;
    rc.far_out = Out{nullptr, nullptr, 0, &st->err};
    rc.far_stamp = nullptr;
    rc.phase = 0;
    rc.changes = &sm.round_pushes;  // the barrier publishes the grid's sum
    rc.mf = nullptr;
    rc.row_ptr = p.row_ptr;
    rc.vis = nullptr;
    rc.ds = nullptr;
    rc.dsr = 0;
    rc.local_rounds = 0;
    rc.local_items = nullptr;
    if (threadIdx.x == 0) {
      if (blockIdx.x == 0) {
        st->tail[(r + 2) % 3] = 0;
        st->grab[(r + 2) % 3] = 0;
      }
      sm.round_pushes = 0;
      sm.big_appended = 0;
    }
    round_body<OP_CCJ, CTA, RED_NONE>(g, sm, rc, edges, dummy_t, dummy_f);
    ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns, p.big.cap != 0);
    if (!ok) break;
    if (sm.pub_flags & kRelBigFlag) {
      big_phase<OP_CCJ, CTA>(g, sm, rc, sm.pub_big);
      ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
      if (!ok) break;
    }
    last_changes = sm.pub_out;
    // shortcut: every vertex points straight at its root
    for (uint32_t v = blockIdx.x * CTA + threadIdx.x; v < p.n; v += gridDim.x * CTA) {
      const uint32_t f0 = __ldcg(p.state + v);
      uint32_t x = f0;
      for (;;) {
        const uint32_t y = __ldcg(p.state + x);
        if (y == x) break;
        x = y;
      }
      if (x != f0) __stcg(p.state + v, x);
    }
    ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
    if (!ok) break;
    rounds = r + 1;
    trace_round(p.trace, p.trace_cap, rounds, p.n, last_changes);
    if (last_changes == 0 || sm.pub_err != DERR_NONE) break;
    if (rounds >= p.max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(&st->err, DERR_MAX_ROUNDS);
      break;
    }
  }
  const unsigned long long esum = cta_sum_u64<CTA>(sm, edges);
  trace_end(p.trace, p.trace_cap, rounds);
  persistent_exit<CTA>(sm, st, ok, rounds, 0, ep0, esum, nullptr, 0);
}

// One invocation (Invoke, or one round of a per-launch Iterate).
template <uint32_t OP, int CTA, int RED>
__device__ __forceinline__ void invoke_round(const KParams& p, const RoundArgs& a, Smem<CTA>& sm) {
  init_smem<CTA>(sm);
  DevStatus* st = p.st;
  SingleView<OP> g{p.row_ptr, p.col, p.w, p.state, p.stamp, p.n};
  RoundCtx rc;
  rc.in_items = a.in_items;
  rc.in_n = a.in_count ? min(__ldcg(a.in_count), a.in_cap) : p.n;
  rc.out = Out{a.out_items, a.out_tail, a.out_cap, &st->err};
  rc.bfs_val = a.level + 1;
  const uint32_t ep = __ldcg(&st->epoch);
  rc.ep = ep;
  rc.grab = &st->grab[0];
  rc.tn = p.tn;
  rc.big = BigList{nullptr, nullptr, 0};  // one launch, no grid barrier: long lists stay in the CTA bin
  rc.big_ctr = nullptr;
  rc.limit = kInf;
  rc.far_out = Out{nullptr, nullptr, 0, &st->err};
  rc.far_stamp = nullptr;
  rc.phase = 0;
  rc.changes = nullptr;
  rc.mf = nullptr;
  rc.row_ptr = p.row_ptr;
  rc.vis = nullptr;
  rc.ds = nullptr;
  rc.dsr = 0;
  rc.local_rounds = 0;
  rc.local_items = nullptr;
  uint32_t edges = 0, any_true = 0, any_false = 0;
  round_body<OP, CTA, RED>(g, sm, rc, edges, any_true, any_false);
  const int t = __syncthreads_or(any_true != 0);
  const int f = __syncthreads_or(any_false != 0);
  const unsigned long long esum = cta_sum_u64<CTA>(sm, edges);
  if (threadIdx.x == 0) {
    if (RED == RED_ANY && t) atomicOr(&st->any_true, 1u);
    if (RED == RED_ALL && f) atomicOr(&st->any_false, 1u);
    atomicAdd(&st->edges, esum);
    __threadfence();
    const uint32_t prev = atomicAdd(&st->exit_count, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      if (RED == RED_ANY) st->result = __ldcg(&st->any_true);
      if (RED == RED_ALL) st->result = __ldcg(&st->any_false) ? 0u : 1u;
      st->any_true = 0;
      st->any_false = 0;
      st->grab[0] = 0;
      if (a.in_consume) *a.in_consume = 0;
      if (OP != OP_BFS) st->epoch = ep + 1;
      st->exit_count = 0;
      __threadfence();
    }
  }
}

// Batched Iterate over many queries in one cooperative launch. Round 0 pops
// the pending worklist left by the admission kernels (or by the previous
// epoch); the launch stops when the worklist drains or after max_rounds
// rounds (an epoch), leaving the pending items and their buffer in p.cont.
template <int CTA>
__device__ __forceinline__ void iterate_batch(const BParams& p, BatchSmem<CTA>& bs) {
  Smem<CTA>& sm = bs.core;
  init_smem<CTA>(sm);
  const uint32_t nq = min(p.nq, static_cast<uint32_t>(kMaxBatchQueries));
  for (uint32_t i = threadIdx.x; i < nq; i += CTA) bs.sbases[i] = __ldg(p.sbases + i);
  __syncthreads();
  DevStatus* st = p.st;
  uint32_t gen = 0;
  const uint32_t ep0 = __ldcg(&st->epoch);
  const uint32_t cur0 = __ldcg(p.cont) & 1u;
  const uint32_t init_n = nq == 0 ? 0u : min(__ldcg(p.cont + 1), p.cap);
  // near-far (SSSP queries): limits in shared memory, advanced by delta after
  // every round in which the query pushed nothing to the out-worklist
  const bool nf = p.delta != 0 && p.ds != nullptr;
  // deferred expansion of long lists (SSSP queries, packed words, plain rounds)
  const bool bdefer = p.dmin != nullptr && p.defer_deg != 0 && p.ds != nullptr && !nf && p.local_rounds == 0;
  const uint32_t fcur0 = nf ? (__ldcg(p.cont + 2) & 1u) : 0u;
  uint32_t far_n = nf ? min(__ldcg(p.cont + 3), p.far_cap) : 0u;
  if (nf)
    for (uint32_t i = threadIdx.x; i < nq; i += CTA) bs.lim[i] = __ldcg(p.blim + __ldg(&p.desc[i].slot));
  BatchView g{p.desc, bs.sbases, nq, p.state, p.stamp, bs.qbits, bs.qfar, nf ? bs.lim : nullptr, p.far_stamp};
  if (threadIdx.x < kMaxBatchQueries / 32) {
    bs.qbits[threadIdx.x] = 0;
    bs.qfar[threadIdx.x] = 0;
  }
  __syncthreads();
  // fold this CTA's query bits into the round's global bitmaps (before a barrier)
  auto fold_marks = [&](uint32_t r) {
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < kMaxBatchQueries / 32; w += CTA) {
      const uint32_t bits = bs.qbits[w], fbits = bs.qfar[w];
      if (bits | fbits) {
        atomicOr(&st->qmask[r & 1][w], bits | fbits);
        if (nf && bits) atomicOr(&st->qnear[r % 3][w], bits);
        bs.qbits[w] = 0;
        bs.qfar[w] = 0;
      }
    }
  };
  // after round r's last barrier: CTA 0 turns the round's bitmap into qlast stamps
  auto publish_marks = [&](uint32_t r, uint32_t ep) {
    if (blockIdx.x != 0) return;
    for (uint32_t w = threadIdx.x; w < kMaxBatchQueries / 32; w += CTA) {
      uint32_t bits = __ldcg(&st->qmask[r & 1][w]);
      if (!bits) continue;
      st->qmask[r & 1][w] = 0;
      while (bits) {
        const uint32_t b = __ffs(bits) - 1;
        bits &= bits - 1;
        p.qlast[w * 32 + b] = ep;
      }
    }
  };
  uint32_t edges = 0, dummy_t = 0, dummy_f = 0, rounds = 0, last_out = 0;
  bool ok = true;
  trace_round(p.trace, p.trace_cap, 0, init_n, 0);
  uint32_t in_n = init_n;
  const uint32_t id_step = p.ds != nullptr ? p.local_rounds + 1u : 1u;
  const unsigned long long t_run0 = p.time_limit_ns ? globaltimer_ns() : 0ull;
  for (uint32_t r = 0; ok; ++r) {
    check_time_limit(&st->err, t_run0, p.time_limit_ns);
    RoundCtx rc;
    rc.in_n = in_n;
    const uint32_t b = (cur0 + r) & 1u;
    rc.in_items = b ? p.items[1] : p.items[0];
    rc.out = Out{b ? p.items[0] : p.items[1], &st->tail[(r + 1) % 3], p.cap, &st->err};
    rc.bfs_val = 0;
    rc.ep = ep0 + r * id_step;
    rc.grab = &st->grab[r % 3];
    rc.tn = p.tn;
    rc.big = p.big;
    rc.big_ctr = &st->big_ctr;
    rc.limit = kInf;
    rc.far_out = Out{nullptr, nullptr, 0, &st->err};
    rc.far_stamp = nullptr;
    rc.phase = 0;
    rc.changes = nullptr;
    rc.mf = nullptr;
    rc.row_ptr = nullptr;
    rc.vis = nullptr;
    rc.ds = p.ds;     // round ids are the global ones: admission writes id 0
    rc.dsr = rc.ep;
    rc.local_rounds = p.ds != nullptr ? p.local_rounds : 0u;
    rc.local_items = nullptr;
    rc.spread = p.spread;
    if (bdefer) {
      // round r reads the words round r - 1 noted, notes into (r + 1) % 3, and
      // clears (r + 2) % 3 (read in round r - 1); the first rounds of a launch
      // neither note into an uncleared buffer nor read one
      if (r >= 2) rc.bdmin_cur = p.dmin + (r % 3u) * kMaxBatchQueries;
      if (r >= 1) rc.bdmin_next = p.dmin + ((r + 1u) % 3u) * kMaxBatchQueries;
      rc.defer_deg = p.defer_deg;
      rc.defer_delta = p.defer_delta;
      if (blockIdx.x == 0) {
        uint32_t* clr = p.dmin + ((r + 2u) % 3u) * kMaxBatchQueries;
        for (uint32_t i = threadIdx.x; i < static_cast<uint32_t>(kMaxBatchQueries); i += CTA) clr[i] = 0u;
      }
    }
    rc.far_in = nullptr;
    rc.far_in_n = 0;
    if (nf) {
      rc.far_in = p.far_items[(fcur0 + r) & 1u];
      rc.far_in_n = far_n;
      rc.far_out = Out{p.far_items[(fcur0 + r + 1) & 1u], &st->bfar_tail[(r + 1) % 3], p.far_cap, &st->err};
      rc.far_stamp = p.far_stamp;
      if (r != 0) {
        // the previous round's out-worklist bits are complete after its barrier
        for (uint32_t i = threadIdx.x; i < nq; i += CTA) {
          const uint32_t slot = __ldg(&p.desc[i].slot);
          if (!((__ldcg(&st->qnear[(r - 1) % 3][slot >> 5]) >> (slot & 31u)) & 1u))
            bs.lim[i] = bs.lim[i] >= kInf - p.delta ? kInf : bs.lim[i] + p.delta;
        }
      }
      // round r - 2's bitmap and round r - 1's far-in size were read before the last barrier
      if (blockIdx.x == 0) {
        for (uint32_t w = threadIdx.x; w < 32; w += CTA) st->qnear[(r + 1) % 3][w] = 0;
        if (threadIdx.x == 0) st->bfar_tail[(r + 2) % 3] = 0;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (blockIdx.x == 0) {
        st->tail[(r + 2) % 3] = 0;
        st->grab[(r + 2) % 3] = 0;
      }
      sm.round_pushes = 0;
      sm.big_appended = 0;
    }
    round_body<OP_RUNTIME, CTA, RED_NONE>(g, sm, rc, edges, dummy_t, dummy_f);
    fold_marks(r);
    ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns, p.big.cap != 0);
    if (!ok) break;
    if (sm.pub_flags & kRelBigFlag) {
      big_phase<OP_RUNTIME, CTA>(g, sm, rc, sm.pub_big);
      fold_marks(r);
      ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
      if (!ok) break;
    }
    publish_marks(r, rc.ep);
    last_out = sm.pub_out;
    rounds = r + 1;
    if (nf) far_n = min(__ldcg(&st->bfar_tail[(r + 1) % 3]), p.far_cap);
    trace_round(p.trace, p.trace_cap, rounds, in_n, last_out);
    if ((last_out == 0 && far_n == 0) || sm.pub_err != DERR_NONE) break;
    if (rounds >= p.max_rounds) {
      if (p.rounds_cap_is_error && blockIdx.x == 0 && threadIdx.x == 0) set_err(&st->err, DERR_MAX_ROUNDS);
      break;
    }
    in_n = min(last_out, p.cap);
  }
  if (nf && blockIdx.x == 0)  // every CTA holds the same limits
    for (uint32_t i = threadIdx.x; i < nq; i += CTA) p.blim[__ldg(&p.desc[i].slot)] = bs.lim[i];
  const unsigned long long esum = cta_sum_u64<CTA>(sm, edges);
  trace_end(p.trace, p.trace_cap, rounds);
  persistent_exit<CTA>(sm, st, ok, rounds, last_out, ep0, esum, p.cont, (cur0 + rounds) & 1u,
                       (fcur0 + rounds) & 1u, far_n, id_step);
}

// Admission of new queries into a batch: per new query j, arena range
// [base_j, base_j + n_j) gets its Iterate initial values (BFS/SSSP: INF; CC:
// label v and every vertex on the pending worklist), then its sources get 0
// and go onto the pending worklist.
struct QNew {
  uint32_t base;
  uint32_t n;
  uint32_t op;
  uint32_t slot;
  uint32_t src_off;  // first source in the flat source array
  uint32_t nsrc;
  uint32_t pre;      // exclusive prefix of n over the new queries
  uint32_t pad;
};

struct AdmitParams {
  const QNew* qn;
  uint32_t nnew;
  uint32_t total;         // sum of n over the new queries
  const uint32_t* srcs;   // flat sources (vertex ids local to each query's graph)
  uint32_t* state;
  unsigned long long* ds; // packed arena (when set, the initial values go here)
  uint32_t* qlast;
  uint32_t* qfirst;       // optional, per query id: the round id it was admitted at
  uint32_t* blim;         // optional (near-far): per slot limit, set to delta
  uint32_t* items[2];
  uint32_t cap;
  uint32_t* cont;
  DevStatus* st;
  uint32_t delta;
  uint32_t id_step;       // round ids per round (1 + CTA-local sub-rounds)
};

__device__ __forceinline__ uint32_t find_new(const QNew* qn, uint32_t nnew, uint32_t i) {
  uint32_t lo = 0, hi = nnew - 1;
  while (lo < hi) {
    const uint32_t md = (lo + hi + 1) >> 1;
    if (__ldg(&qn[md].pre) <= i) lo = md;
    else hi = md - 1;
  }
  return lo;
}

// Warp-aggregated append of one optional item per lane to the pending worklist.
__device__ __forceinline__ void append_pending(const AdmitParams& a, uint32_t* buf, bool p, uint32_t v) {
  const unsigned m = __ballot_sync(kFull, p);
  if (m == 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const int ld = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == static_cast<uint32_t>(ld)) base = atomicAdd(a.cont + 1, static_cast<uint32_t>(__popc(m)));
  base = __shfl_sync(kFull, base, ld);
  if (p) {
    const uint32_t idx = base + __popc(m & lanemask_lt());
    if (idx < a.cap) __stcg(buf + idx, v);
    else set_err(&a.st->err, DERR_WL_OVERFLOW);
  }
}

__device__ __forceinline__ void admit_fill(const AdmitParams& a) {
  // grid-stride over the concatenated new ranges; trip count uniform per warp
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t* buf = (__ldcg(a.cont) & 1u) ? a.items[1] : a.items[0];
  for (uint32_t base = tid - (threadIdx.x & 31); base < a.total; base += nthreads) {
    const uint32_t i = base + (threadIdx.x & 31);
    bool push = false;
    uint32_t item = 0;
    if (i < a.total) {
      const uint32_t j = find_new(a.qn, a.nnew, i);
      const QNew q = a.qn[j];
      const uint32_t v = i - q.pre;
      item = q.base + v;
      const uint32_t init = q.op == OP_CC ? v : kInf;
      if (a.ds != nullptr) __stcg(a.ds + item, static_cast<unsigned long long>(init) << 32);
      else __stcg(a.state + item, init);
      push = q.op == OP_CC;
    }
    append_pending(a, buf, push, item);
  }
}

__device__ __forceinline__ void admit_sources(const AdmitParams& a) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  uint32_t* buf = (__ldcg(a.cont) & 1u) ? a.items[1] : a.items[0];
  const uint32_t ep = __ldcg(&a.st->epoch);
  for (uint32_t j = tid; j < a.nnew; j += nthreads) {
    a.qlast[a.qn[j].slot] = ep - a.id_step;  // "last pushed" one round before admission
    if (a.qfirst != nullptr) a.qfirst[a.qn[j].slot] = ep;
    if (a.blim != nullptr) a.blim[a.qn[j].slot] = a.delta;
  }
  // one warp per new query walks its sources
  const uint32_t warp = tid >> 5, nwarps = nthreads >> 5, lane = threadIdx.x & 31;
  for (uint32_t j = warp; j < a.nnew; j += nwarps) {
    const QNew q = a.qn[j];
    if (q.op == OP_CC) continue;
    for (uint32_t k0 = 0; k0 < q.nsrc; k0 += 32) {
      const uint32_t k = k0 + lane;
      bool p = false;
      uint32_t item = 0;
      if (k < q.nsrc) {
        const uint32_t v = __ldg(a.srcs + q.src_off + k);
        if (v < q.n) {
          item = q.base + v;
          // a repeated source is pushed once
          p = a.ds != nullptr ? (atomicExch(a.ds + item, 0ull) >> 32) != 0u : atomicExch(a.state + item, 0u) != 0u;
        }
      }
      append_pending(a, buf, p, item);
    }
  }
}

}  // namespace irgl
