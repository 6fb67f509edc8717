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
enum : uint32_t { OP_BFS = 0, OP_SSSP = 1, OP_CC = 2, OP_RUNTIME = 3 };
enum : int { RED_NONE = 0, RED_ANY = 1, RED_ALL = 2 };
// Device error codes (first one wins).
enum : uint32_t {
  DERR_NONE = 0,
  DERR_WL_OVERFLOW = 1,
  DERR_BARRIER_TIMEOUT = 2,
  DERR_MAX_ROUNDS = 3,
  DERR_BAD_ITEM = 4,
};

// Device status block. Each contended family sits on its own 128-byte line.
// Invariant between launches: bar_count, exit_count, tail[], grab[],
// any_true and any_false are 0 (every kernel restores them on a clean exit;
// the host clears the block after an error).
struct alignas(128) DevStatus {
  uint32_t bar_count;
  uint32_t exit_count;
  uint32_t pad0[30];
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
};
static_assert(sizeof(DevStatus) == 512, "status layout");

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
};

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
  int skip_cta;                // test hook: this CTA never reaches the first barrier
  int init_state;              // write the Iterate initial values in the prologue
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

// ----------------------------------------------------------------------------- small helpers

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
  static constexpr int kStage = 4 * CTA;  // push stage capacity (items)
  static constexpr int kWarps = CTA / 32;
  uint32_t stage[kStage];
  uint32_t s_off[CTA];   // scan bin: exclusive offset of each thread's short list
  uint32_t s_beg[CTA];   //           first edge of the list
  uint32_t s_val[CTA];   //           operator value of the popped vertex
  uint32_t s_q[CTA];     //           query slot (batched)
  uint32_t warp_sums[kWarps + 1];
  uint32_t stage_n;
  uint32_t gbase;
  uint32_t grab_base;
  uint32_t flag;
  uint32_t own_tid, own_beg, own_end, own_val, own_q;
  uint32_t red;
  unsigned long long edges;
  uint8_t pushed[CTA];   // ReduceAndReturn All: item pushed something
};

// ----------------------------------------------------------------------------- cooperative-conversion push

// Flush the stage to the out-worklist: one global atomicAdd, coalesced stores.
// Called by every thread of the CTA at a CTA-uniform point, after a barrier.
template <int CTA>
__device__ __forceinline__ void flush_stage(Smem<CTA>& sm, const Out& out) {
  const uint32_t n = min(sm.stage_n, static_cast<uint32_t>(Smem<CTA>::kStage));
  if (n == 0) return;
  if (threadIdx.x == 0) sm.gbase = atomicAdd(out.tail, n);
  __syncthreads();
  const uint32_t gb = sm.gbase;
  for (uint32_t i = threadIdx.x; i < n; i += CTA) {
    const uint32_t idx = gb + i;
    if (idx < out.cap) __stcg(out.items + idx, sm.stage[i]);
    else set_err(out.err, DERR_WL_OVERFLOW);
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.stage_n = 0;
  __syncthreads();
}

// Items that did not fit the stage go straight to global memory, aggregated per warp.
__device__ __forceinline__ void push_global_warp(const Out& out, uint32_t cnt_lane, uint32_t incl_unused,
                                                 uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
  (void)incl_unused;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t incl = warp_incl_scan(cnt_lane);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  uint32_t gb = 0;
  if (lane == 31) gb = atomicAdd(out.tail, total);
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
    push_global_warp(out, ov ? 1u : 0u, 0u, v, 0u, 0u, 0u);
  }
}

// Up to four candidate items per lane (flags f bits 0..3): warp scan aggregation.
template <int CTA>
__device__ __forceinline__ void push4(Smem<CTA>& sm, const Out& out, uint32_t f, uint32_t v0, uint32_t v1,
                                      uint32_t v2, uint32_t v3) {
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
    push_global_warp(out, ov, 0u, g0, g1, g2, g3);
  }
}

// ----------------------------------------------------------------------------- CTA-wide scan

template <int CTA>
__device__ __forceinline__ uint32_t cta_excl_scan(Smem<CTA>& sm, uint32_t x, uint32_t& total) {
  constexpr int NW = Smem<CTA>::kWarps;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(x);
  if (lane == 31) sm.warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t s = lane < static_cast<uint32_t>(NW) ? sm.warp_sums[lane] : 0u;
    const uint32_t si = warp_incl_scan(s);
    if (lane < static_cast<uint32_t>(NW)) sm.warp_sums[lane] = si - s;
    if (lane == static_cast<uint32_t>(NW) - 1) sm.warp_sums[NW] = si;
  }
  __syncthreads();
  total = sm.warp_sums[NW];
  return sm.warp_sums[wid] + incl - x;
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
  __device__ __forceinline__ uint32_t nverts(uint32_t) const { return n; }
  __device__ __forceinline__ uint32_t op(uint32_t) const { return OP; }
  __device__ __forceinline__ const uint32_t* rowp(uint32_t) const { return row_ptr; }
  __device__ __forceinline__ const uint32_t* colp(uint32_t) const { return col; }
  __device__ __forceinline__ const int32_t* wp(uint32_t) const { return w; }
  __device__ __forceinline__ uint32_t sbase(uint32_t) const { return 0u; }
  __device__ __forceinline__ void decode(uint32_t item, uint32_t& q, uint32_t& u) const { q = 0; u = item; }
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

template <uint32_t OP>
__device__ __forceinline__ bool needs_w(uint32_t op_rt) {
  return (OP == OP_RUNTIME ? op_rt : OP) == OP_SSSP;
}

// Edges [beg, end) of one owner, GROUP threads cooperating (GROUP = 32: a warp,
// GROUP = CTA: the whole CTA); `rank` in [0, GROUP). 16-byte vector loads of
// col (and w) after an alignment peel; the loop trip count is uniform across
// the group so the warp-level pushes see converged warps.
template <uint32_t OP, int CTA, int GROUP, class V>
__device__ __forceinline__ bool group_edges(const V& g, Smem<CTA>& sm, const Out& out, uint32_t q, uint32_t beg,
                                            uint32_t end, uint32_t val, uint32_t ep, uint32_t rank) {
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
  {  // head: up to 3 edges before the 16-byte boundary
    const uint32_t e = beg + rank;
    bool p = false;
    uint32_t v = 0;
    if (e < a) {
      v = __ldg(col + e);
      p = relax<OP>(op, state, stamp, v, val, nw ? __ldg(w + e) : 0, ep);
    }
    push1<CTA>(sm, out, p, sb + v);
    any |= p;
  }
  for (uint32_t base = a; base < b; base += 4u * GROUP) {
    const uint32_t e = base + 4u * rank;
    uint32_t f = 0;
    uint4 c = make_uint4(0, 0, 0, 0);
    if (e < b) {
      c = __ldg(reinterpret_cast<const uint4*>(col + e));
      int4 ww = make_int4(0, 0, 0, 0);
      if (nw) ww = __ldg(reinterpret_cast<const int4*>(w + e));
      f |= relax<OP>(op, state, stamp, c.x, val, ww.x, ep) ? 1u : 0u;
      f |= relax<OP>(op, state, stamp, c.y, val, ww.y, ep) ? 2u : 0u;
      f |= relax<OP>(op, state, stamp, c.z, val, ww.z, ep) ? 4u : 0u;
      f |= relax<OP>(op, state, stamp, c.w, val, ww.w, ep) ? 8u : 0u;
    }
    push4<CTA>(sm, out, f, sb + c.x, sb + c.y, sb + c.z, sb + c.w);
    any |= f != 0;
    if (GROUP == CTA) {
      // the predicate is taken at the barrier, when every warp's pushes are in
      if (__syncthreads_or(sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2))) flush_stage<CTA>(sm, out);
    }
  }
  {  // tail: up to 3 edges after the last full vector
    const uint32_t e = b + rank;
    bool p = false;
    uint32_t v = 0;
    if (e < end) {
      v = __ldg(col + e);
      p = relax<OP>(op, state, stamp, v, val, nw ? __ldg(w + e) : 0, ep);
    }
    push1<CTA>(sm, out, p, sb + v);
    any |= p;
  }
  return any;
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
};

template <uint32_t OP, int CTA, int RED, class V>
__device__ __forceinline__ void process_tile(const V& g, Smem<CTA>& sm, const RoundCtx& rc, uint32_t idx,
                                             uint32_t& edges, uint32_t& any_true, uint32_t& any_false) {
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31;
  bool valid = idx < rc.in_n;
  uint32_t q = 0, beg = 0, end = 0, val = 0;
  if (valid) {
    const uint32_t item = rc.in_items ? __ldcg(rc.in_items + idx) : idx;
    uint32_t u;
    g.decode(item, q, u);
    if (u >= g.nverts(q)) {  // a caller-pushed item outside the graph: report and skip it
      set_err(rc.out.err, DERR_BAD_ITEM);
      valid = false;
    } else {
      const uint32_t* rp = g.rowp(q);
      beg = __ldg(rp + u);
      end = __ldg(rp + u + 1);
      const uint32_t op = g.op(q);
      if (op == OP_BFS) val = V::kBatched ? __ldcg(g.state + item) + 1u : rc.bfs_val;
      else val = __ldcg(g.state + item);
    }
  }
  const uint32_t deg = end - beg;
  edges += deg;
  bool pushed = false;

  // CTA bin: the whole CTA walks one long list at a time.
  bool big = deg >= rc.tn.cta_thresh;
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
    const bool p = group_edges<OP, CTA, CTA>(g, sm, rc.out, sm.own_q, sm.own_beg, sm.own_end, sm.own_val, rc.ep, tid);
    if (RED == RED_ALL && p) sm.pushed[sm.own_tid] = 1;
    pushed |= p;
  }

  // Warp bin: each warp walks its members' medium lists one at a time.
  bool mid = valid && deg >= rc.tn.warp_thresh && deg < rc.tn.cta_thresh;
  for (;;) {
    const unsigned m = __ballot_sync(kFull, mid);
    if (m == 0) break;
    const int ld = __ffs(m) - 1;
    const uint32_t wb = __shfl_sync(kFull, beg, ld);
    const uint32_t we = __shfl_sync(kFull, end, ld);
    const uint32_t wv = __shfl_sync(kFull, val, ld);
    const uint32_t wq = __shfl_sync(kFull, q, ld);
    if (lane == static_cast<uint32_t>(ld)) mid = false;
    const bool p = group_edges<OP, CTA, 32>(g, sm, rc.out, wq, wb, we, wv, rc.ep, lane);
    if (RED == RED_ALL && p) sm.pushed[(tid & ~31u) + ld] = 1;
    pushed |= p;
  }

  // Scan bin: short lists of the whole tile, one edge per thread per strip.
  const bool small = valid && deg > 0 && deg < rc.tn.warp_thresh && deg < rc.tn.cta_thresh;
  uint32_t total = 0;
  const uint32_t excl = cta_excl_scan<CTA>(sm, small ? deg : 0u, total);
  if (total > 0) {
    sm.s_off[tid] = excl;
    sm.s_beg[tid] = beg;
    sm.s_val[tid] = val;
    sm.s_q[tid] = q;
    __syncthreads();
    for (uint32_t base = 0; base < total; base += CTA) {
      const uint32_t e = base + tid;
      bool p = false;
      uint32_t pv = 0;
      if (e < total) {
        uint32_t lo = 0, hi = CTA - 1;
        while (lo < hi) {
          const uint32_t md = (lo + hi + 1) >> 1;
          if (sm.s_off[md] <= e) lo = md;
          else hi = md - 1;
        }
        const uint32_t oq = sm.s_q[lo];
        const uint32_t edge = sm.s_beg[lo] + (e - sm.s_off[lo]);
        const uint32_t op = g.op(oq);
        const uint32_t sb = g.sbase(oq);
        const uint32_t v = __ldg(g.colp(oq) + edge);
        const int32_t wt = needs_w<OP>(op) ? __ldg(g.wp(oq) + edge) : 0;
        p = relax<OP>(op, g.state + sb, g.stamp + sb, v, sm.s_val[lo], wt, rc.ep);
        pv = sb + v;
        if (RED == RED_ALL && p) sm.pushed[lo] = 1;
      }
      push1<CTA>(sm, rc.out, p, pv);
      pushed |= p;
      if (__syncthreads_or(sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2))) flush_stage<CTA>(sm, rc.out);
    }
  }

  if (RED == RED_ANY) any_true |= pushed ? 1u : 0u;
  const bool full = __syncthreads_or(sm.stage_n >= static_cast<uint32_t>(Smem<CTA>::kStage / 2));
  if (RED == RED_ALL) {
    if (valid && !sm.pushed[tid]) any_false = 1u;
    sm.pushed[tid] = 0;
  }
  if (full) flush_stage<CTA>(sm, rc.out);
}

// ForAll over the in-worklist: CTAs grab `chunk` tiles of CTA items at a time.
template <uint32_t OP, int CTA, int RED, class V>
__device__ __forceinline__ void round_body(const V& g, Smem<CTA>& sm, const RoundCtx& rc, uint32_t& edges,
                                           uint32_t& any_true, uint32_t& any_false) {
  const uint32_t span = CTA * rc.tn.chunk;
  for (;;) {
    if (threadIdx.x == 0) sm.grab_base = atomicAdd(rc.grab, span);
    __syncthreads();
    const uint32_t gb = sm.grab_base;
    __syncthreads();
    if (gb >= rc.in_n) break;
    for (uint32_t t = 0; t < rc.tn.chunk; ++t) {
      const uint32_t tb = gb + t * CTA;
      if (tb >= rc.in_n) break;
      process_tile<OP, CTA, RED>(g, sm, rc, tb + threadIdx.x, edges, any_true, any_false);
    }
  }
  __syncthreads();
  flush_stage<CTA>(sm, rc.out);
}

// ----------------------------------------------------------------------------- grid barrier

// SyncRunningThreads: valid only because the launch is cooperative (all CTAs
// co-resident). Arrival counter is monotonic within a launch; the spin is
// bounded by timeout_ns and gives up as soon as any CTA reported an error.
template <int CTA>
__device__ __forceinline__ bool grid_barrier(Smem<CTA>& sm, DevStatus* st, uint32_t& target,
                                             unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += gridDim.x;
    __threadfence();
    atomicAdd(&st->bar_count, 1u);
    uint32_t ok = 1;
    const unsigned long long t0 = globaltimer_ns();
    uint32_t spins = 0;
    for (;;) {
      const uint32_t c = ld_acquire_gpu(&st->bar_count);
      if (static_cast<int32_t>(c - target) >= 0) break;
      if ((++spins & 31u) == 0) {
        if (__ldcg(&st->err) == DERR_BARRIER_TIMEOUT) { ok = 0; break; }
        if (globaltimer_ns() - t0 > timeout_ns) {
          set_err(&st->err, DERR_BARRIER_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    sm.flag = ok;
  }
  __syncthreads();
  return sm.flag != 0;
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
  }
  __syncthreads();
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

// ----------------------------------------------------------------------------- kernels

// Iteration-outlined Iterate: every round in one cooperative launch.
template <uint32_t OP, int CTA>
__device__ __forceinline__ void iterate_persistent(const KParams& p, Smem<CTA>& sm) {
  init_smem<CTA>(sm);
  DevStatus* st = p.st;
  const uint32_t G = gridDim.x;
  uint32_t target = 0;
  const uint32_t ep0 = __ldcg(&st->epoch);
  const uint32_t init_n = p.init_count ? min(__ldcg(p.init_count), p.init_cap) : p.n;
  if (p.skip_cta == static_cast<int>(blockIdx.x)) return;  // test hook: never arrives

  SingleView<OP> g{p.row_ptr, p.col, p.w, p.state, p.stamp, p.n};
  uint32_t edges = 0, dummy_t = 0, dummy_f = 0;
  uint32_t rounds = 0;
  bool ok = true;

  if (p.init_state) {
    uint32_t srcs[8];
    uint32_t ns = 0;
    const bool small = OP != OP_CC && p.init_items != nullptr && init_n <= 8;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) srcs[i] = (small && i < init_n) ? __ldcg(p.init_items + i) : kInf;
    if (small) ns = init_n;
    fill_state<OP>(p.state, p.n, srcs, ns, blockIdx.x * CTA + threadIdx.x, G * CTA);
    if (OP != OP_CC && !small) {
      ok = grid_barrier<CTA>(sm, st, target, p.timeout_ns);
      if (ok) {
        for (uint32_t i = blockIdx.x * CTA + threadIdx.x; i < init_n; i += G * CTA) {
          const uint32_t s = p.init_items ? __ldcg(p.init_items + i) : i;
          if (s < p.n) __stcg(p.state + s, 0u);
        }
      }
    }
  }
  if (ok) ok = grid_barrier<CTA>(sm, st, target, p.timeout_ns);

  uint32_t last_out = 0;
  for (uint32_t r = 0; ok; ++r) {
    RoundCtx rc;
    rc.in_n = r == 0 ? init_n : min(__ldcg(&st->tail[r % 3]), p.cap);
    uint32_t* const cur = (r & 1) ? p.items[1] : p.items[0];  // no dynamic index into the param struct
    uint32_t* const nxt = (r & 1) ? p.items[0] : p.items[1];
    rc.in_items = r == 0 ? p.init_items : cur;
    rc.out = Out{nxt, &st->tail[(r + 1) % 3], p.cap, &st->err};
    rc.bfs_val = r + 1;
    rc.ep = ep0 + r;
    rc.grab = &st->grab[r % 3];
    rc.tn = p.tn;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->tail[(r + 2) % 3] = 0;
      st->grab[(r + 2) % 3] = 0;
    }
    round_body<OP, CTA, RED_NONE>(g, sm, rc, edges, dummy_t, dummy_f);
    ok = grid_barrier<CTA>(sm, st, target, p.timeout_ns);
    if (!ok) break;
    last_out = __ldcg(&st->tail[(r + 1) % 3]);
    const uint32_t err = __ldcg(&st->err);
    rounds = r + 1;
    if (last_out == 0 || err != DERR_NONE) break;
    if (rounds >= p.max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(&st->err, DERR_MAX_ROUNDS);
      break;
    }
  }

  const unsigned long long esum = cta_sum_u64<CTA>(sm, edges);
  if (threadIdx.x == 0) {
    atomicAdd(&st->edges, esum);
    if (ok) {
      __threadfence();
      const uint32_t prev = atomicAdd(&st->exit_count, 1u);
      if (prev == G - 1) {
        __threadfence();
        st->rounds = rounds;
        st->last_out = last_out;
        st->epoch = ep0 + rounds + 1;
        for (int i = 0; i < 4; ++i) {
          st->tail[i] = 0;
          st->grab[i] = 0;
        }
        st->bar_count = 0;
        st->exit_count = 0;
        __threadfence();
      }
    }
  }
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

}  // namespace irgl
