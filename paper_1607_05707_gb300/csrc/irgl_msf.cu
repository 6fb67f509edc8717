// Minimum spanning forest by Boruvka's algorithm (Sec. 3.3) as an outlined
// multi-kernel Pipe (Sec. 4.3, 4.4):
//
//   Pipe {                                    // until no component has a cross edge
//     Invoke find_min(in -> out, retry)       // Atomic(component_lock) { keep the lighter edge }
//       [Invoke find_min(retry -> retry')]*   // Retry items re-run (Retry Backoff mapping)
//     Invoke link(components)                 // record the edges, hook the components
//     Iterate jump(all vertices)              // pointer jumping, Until !Any(changed)
//   }
//
// Edge order: the key (w, min(u,v), max(u,v)) is a strict order on distinct
// undirected edges, so every component has one lightest cross edge and the
// forest is unique. A component's lightest edge is a multi-word record (weight,
// both endpoints, CSR index, the other component), which no single atomic can
// update: the find_min kernel updates it inside an Atomic section on the
// component's lock, in one of three forms:
//   IRGL_LOCK_BLOCKING  divergence-safe atomicCAS retry loop (the lock attempt
//                       and the critical section share one branch), bounded
//   IRGL_LOCK_TICKET    ticket lock (take a ticket, wait for it to be served),
//                       bounded
//   IRGL_LOCK_RETRY     one atomicCAS attempt (Atomic ... Else); a vertex that
//                       misses the lock is pushed to the retry worklist and
//                       find_min is invoked again on that list, with contiguous
//                       blocks of items per thread (Retry Backoff), until it is
//                       empty.
// Before taking a lock a thread compares its weight with the component's
// current one (weights only fall within an iteration), so most vertices never
// lock.
//
// Outlined (IRGL_PERSISTENT): the three kernels run back to back in one
// cooperative launch, separated by the grid barrier; the CTA size is chosen by
// the T_control rule over the kernels' block-size sets. IRGL_PER_LAUNCH: one
// launch per kernel invocation, with the host reading the counters in between.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

namespace irgl {

constexpr uint32_t kMsfMaxIters = 64;  // Boruvka halves the components with cross edges: 32 suffice

// Per-invocation counters, a ring of three: invocation j counts into slot j % 3
// and CTA 0 clears slot (j + 1) % 3 at its start (every CTA read that slot
// after the barrier that ended invocation j - 2, before arriving at the one
// that ended j - 1).
struct __align__(16) MsfSlot {
  uint32_t out;      // vertices pushed to the out-worklist (found a cross edge)
  uint32_t retry;    // vertices pushed to the retry worklist
  uint32_t comp;     // components whose record got its first edge this iteration
  uint32_t changed;  // pointer-jumping updates
};

struct MsfStatus {
  unsigned long long weight;  // total forest weight
  uint32_t edges;             // forest edges written
  uint32_t retries;           // retry pushes over the whole run
  uint32_t iterations;        // Boruvka iterations (Pipe repetitions)
  uint32_t invocations;       // kernel invocations inside the Pipe
  uint32_t locks;             // lock acquisitions
  uint32_t pad0[25];
  MsfSlot slot[3];
  uint32_t pad1[20];
};
static_assert(sizeof(MsfStatus) % 128 == 0, "status layout");

struct MsfParams {
  const uint32_t* __restrict__ row_ptr;
  const uint32_t* __restrict__ col;
  const int32_t* __restrict__ w;
  uint32_t n;
  uint32_t* comp;    // component (root vertex) of each vertex
  unsigned long long* cwl;  // per component: lightest cross edge's (w << 32) | min(u,v) (~0: none yet),
                            // one word so the pre-lock test reads a consistent prefix of the key
  uint32_t* chi;     //   its larger endpoint
  uint32_t* cedge;   //   its CSR index
  uint32_t* cother;  //   the component at its other end
  uint32_t* lock;    // per component: 0/1 (BLOCKING, RETRY) or now-serving (TICKET)
  uint32_t* ticket;  // per component: next ticket (TICKET)
  uint32_t* items[2];  // in/out worklists of vertices (capacity n each)
  uint32_t* retry[2];  // retry worklists (capacity n each)
  uint32_t* comps;     // components with a record this iteration (capacity n)
  uint32_t* out_edges;
  uint32_t out_cap;
  uint32_t lock_mode;
  DevStatus* st;
  MsfStatus* ms;
  unsigned long long timeout_ns;       // grid barrier waits
  unsigned long long lock_timeout_ns;  // lock waits and one find_min's retries: half the barrier's, so a
                                       // stuck lock is reported as such before the barrier gives up
  uint32_t held_lock;  // test hook: this component's lock starts held and is never released (kInf: none)
};

// Lexicographic order on (w, lo, hi).
__device__ __forceinline__ bool key_less(uint32_t w1, uint32_t l1, uint32_t h1, uint32_t w2, uint32_t l2, uint32_t h2) {
  if (w1 != w2) return w1 < w2;
  if (l1 != l2) return l1 < l2;
  return h1 < h2;
}

struct MinEdge {
  uint32_t w, lo, hi, e, other;
};

__device__ __forceinline__ MinEdge no_edge() { return MinEdge{kInf, kInf, kInf, 0u, 0u}; }

// Lightest cross-component edge among u's edges [beg, end), lanes taking
// every stride-th edge from beg + rank.
__device__ __forceinline__ void scan_edges(const MsfParams& p, uint32_t u, uint32_t cu, uint32_t beg, uint32_t end,
                                           uint32_t rank, uint32_t stride, MinEdge& best) {
  for (uint32_t e = beg + rank; e < end; e += stride) {
    const uint32_t v = __ldg(p.col + e);
    const uint32_t cv = __ldcg(p.comp + v);
    if (cv == cu) continue;
    const uint32_t wt = static_cast<uint32_t>(__ldg(p.w + e));
    const uint32_t lo = min(u, v), hi = max(u, v);
    if (key_less(wt, lo, hi, best.w, best.lo, best.hi)) best = MinEdge{wt, lo, hi, e, cv};
  }
}

__device__ __forceinline__ MinEdge warp_min_edge(MinEdge b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    MinEdge x;
    x.w = __shfl_xor_sync(kFull, b.w, o);
    x.lo = __shfl_xor_sync(kFull, b.lo, o);
    x.hi = __shfl_xor_sync(kFull, b.hi, o);
    x.e = __shfl_xor_sync(kFull, b.e, o);
    x.other = __shfl_xor_sync(kFull, b.other, o);
    if (key_less(x.w, x.lo, x.hi, b.w, b.lo, b.hi)) b = x;
  }
  return b;
}

// Warp-aggregated push of `item` (where pred) to list[base + ...], counting in *ctr.
__device__ __forceinline__ void warp_push(uint32_t* list, uint32_t base, uint32_t cap, uint32_t* ctr, bool pred,
                                          uint32_t item, uint32_t* err) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (m == 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  uint32_t pos = 0;
  if (lane == static_cast<uint32_t>(leader)) pos = atomicAdd(ctr, static_cast<uint32_t>(__popc(m)));
  pos = __shfl_sync(kFull, pos, leader) + __popc(m & lanemask_lt());
  if (pred) {
    if (base + pos < cap) __stcg(list + base + pos, item);
    else set_err(err, DERR_WL_OVERFLOW);
  }
}

constexpr unsigned long long kNoRecord = ~0ull;

__device__ __forceinline__ unsigned long long wl_of(const MinEdge& k) {
  return (static_cast<unsigned long long>(k.w) << 32) | k.lo;
}

// The critical section of the Atomic: keep the lighter of the component's
// record and this edge. The first edge of the iteration lists the component.
__device__ __forceinline__ void record_update(const MsfParams& p, uint32_t c, const MinEdge& k, MsfSlot* slot,
                                              uint32_t comp_base) {
  const unsigned long long wl0 = __ldcg(p.cwl + c), wl = wl_of(k);
  if (wl > wl0 || (wl == wl0 && k.hi >= __ldcg(p.chi + c))) return;
  if (wl0 == kNoRecord) {
    const uint32_t pos = comp_base + atomicAdd(&slot->comp, 1u);
    if (pos < p.n) __stcg(p.comps + pos, c);
    else set_err(&p.st->err, DERR_WL_OVERFLOW);
  }
  __stcg(p.cwl + c, wl);
  __stcg(p.chi + c, k.hi);
  __stcg(p.cedge + c, k.e);
  __stcg(p.cother + c, k.other);
}

__device__ __forceinline__ unsigned long long msf_now() { return globaltimer_ns(); }

// Atomic(lock[c]) { record_update } in the configured form. Returns false when
// the lock was missed in RETRY mode (the caller retries the vertex).
__device__ __forceinline__ bool atomic_update(const MsfParams& p, uint32_t c, const MinEdge& k, MsfSlot* slot,
                                              uint32_t comp_base) {
  // test before locking: the record only gets lighter within an iteration, and
  // its (w, lo) prefix is one word, so a heavier prefix can never win
  if (wl_of(k) > __ldcg(p.cwl + c)) return true;
  if (p.lock_mode == IRGL_LOCK_TICKET) {
    const uint32_t t = atomicAdd(p.ticket + c, 1u);
    const unsigned long long t0 = msf_now();
    for (uint32_t spins = 1;; ++spins) {
      uint32_t serving;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(serving) : "l"(p.lock + c) : "memory");
      if (serving == t) break;
      if ((spins & 63u) == 0 && (msf_now() - t0 > p.lock_timeout_ns || __ldcg(&p.st->err) == DERR_LOCK_TIMEOUT)) {
        set_err(&p.st->err, DERR_LOCK_TIMEOUT);
        return true;
      }
    }
    record_update(p, c, k, slot, comp_base);
    atomicAdd(&p.ms->locks, 1u);
    asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p.lock + c), "r"(t + 1u) : "memory");
    return true;
  }
  const bool blocking = p.lock_mode == IRGL_LOCK_BLOCKING;
  const unsigned long long t0 = blocking ? msf_now() : 0ull;
  for (uint32_t spins = 1;; ++spins) {
    // the attempt and the critical section in one branch: no thread waits on
    // a lock held by a lane of its own warp that cannot be scheduled
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], 0, 1;" : "=r"(old) : "l"(p.lock + c) : "memory");
    if (old == 0u) {
      record_update(p, c, k, slot, comp_base);
      atomicAdd(&p.ms->locks, 1u);
      asm volatile("st.release.gpu.global.u32 [%0], 0;" : : "l"(p.lock + c) : "memory");
      return true;
    }
    if (!blocking) return false;  // Atomic ... Else: Retry
    if ((spins & 63u) == 0 && (msf_now() - t0 > p.lock_timeout_ns || __ldcg(&p.st->err) == DERR_LOCK_TIMEOUT)) {
      set_err(&p.st->err, DERR_LOCK_TIMEOUT);
      return true;
    }
    __nanosleep(min(32u << min(spins, 5u), 1024u));  // exponential backoff: waiters leave the line to the holder
  }
}

// Lanes of a warp whose vertices share a component send only the lightest of
// their edges to the Atomic section (the others cannot change the record).
// Returns true when that lane missed the lock in RETRY mode.
__device__ __forceinline__ bool aggregate_update(const MsfParams& p, bool found, uint32_t cu, const MinEdge& best,
                                                 MsfSlot* slot, uint32_t comp_base) {
  const unsigned active = __ballot_sync(kFull, found);
  if (!found) return false;
  const unsigned peers = __match_any_sync(active, cu);
  const uint32_t mw = __reduce_min_sync(peers, best.w);
  const uint32_t ml = __reduce_min_sync(peers, best.w == mw ? best.lo : kInf);
  const uint32_t mh = __reduce_min_sync(peers, best.w == mw && best.lo == ml ? best.hi : kInf);
  if (best.w != mw || best.lo != ml || best.hi != mh) return false;
  return !atomic_update(p, cu, best, slot, comp_base);
}

// find_min over a worklist: `in` (nullptr = vertices 0..in_n-1). Default
// mapping: a warp takes 32 consecutive items; lists of 32 edges or more are
// scanned by the whole warp. Retry mapping (Retry Backoff): thread t takes the
// contiguous block [t * B, (t + 1) * B) and scans each list alone.
__device__ void msf_find_min(const MsfParams& p, const uint32_t* in, uint32_t in_n, bool backoff, uint32_t* out,
                             uint32_t out_base, uint32_t* retry_out, MsfSlot* slot, uint32_t comp_base,
                             uint32_t gtid, uint32_t nthreads) {
  const uint32_t lane = threadIdx.x & 31;
  if (backoff) {
    const uint32_t B = (in_n + nthreads - 1) / nthreads;
    const uint32_t lo = min(gtid * B, in_n), hi = min(lo + B, in_n);
    // warp-uniform trip count so the warp-aggregated pushes see converged warps
    uint32_t trips = hi - lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) trips = max(trips, __shfl_xor_sync(kFull, trips, o));
    for (uint32_t t = 0; t < trips; ++t) {
      const uint32_t i = lo + t;
      const bool valid = i < hi;
      uint32_t u = 0, cu = 0;
      bool found = false, missed = false;
      MinEdge best = no_edge();
      if (valid) {
        u = __ldcg(in + i);
        cu = __ldcg(p.comp + u);
        best = no_edge();
        scan_edges(p, u, cu, __ldg(p.row_ptr + u), __ldg(p.row_ptr + u + 1), 0, 1, best);
        found = best.w != kInf;
      }
      missed = aggregate_update(p, found, cu, best, slot, comp_base);
      warp_push(out, out_base, p.n, &slot->out, found && !missed, u, &p.st->err);
      warp_push(retry_out, 0, p.n, &slot->retry, missed, u, &p.st->err);
    }
    return;
  }
  const uint32_t wid = gtid >> 5, nwarps = nthreads >> 5;
  for (uint32_t base = wid * 32; base < in_n; base += nwarps * 32) {
    const uint32_t idx = base + lane;
    const bool valid = idx < in_n;
    uint32_t u = 0, cu = 0, beg = 0, end = 0;
    if (valid) {
      u = in ? __ldcg(in + idx) : idx;
      cu = __ldcg(p.comp + u);
      beg = __ldg(p.row_ptr + u);
      end = __ldg(p.row_ptr + u + 1);
    }
    MinEdge best = no_edge();
    const bool big = valid && end - beg >= 32u;
    if (valid && !big) scan_edges(p, u, cu, beg, end, 0, 1, best);
    for (unsigned m = __ballot_sync(kFull, big); m; m &= m - 1) {
      const int l = __ffs(m) - 1;
      MinEdge wb = no_edge();
      scan_edges(p, __shfl_sync(kFull, u, l), __shfl_sync(kFull, cu, l), __shfl_sync(kFull, beg, l),
                 __shfl_sync(kFull, end, l), lane, 32, wb);
      wb = warp_min_edge(wb);
      if (lane == static_cast<uint32_t>(l)) best = wb;
    }
    const bool found = best.w != kInf;
    const bool missed = aggregate_update(p, found, cu, best, slot, comp_base);
    warp_push(out, out_base, p.n, &slot->out, found && !missed, u, &p.st->err);
    warp_push(retry_out, 0, p.n, &slot->retry, missed, u, &p.st->err);
  }
}

// link over the components with a record: record the edge (once per mutual
// pair: by the smaller component) and hook the component to the other one
// (a mutual pair's smaller component stays the root), then clear the record.
__device__ void msf_link(const MsfParams& p, uint32_t comp_n, uint32_t gtid, uint32_t nthreads) {
  for (uint32_t i = gtid; i < comp_n; i += nthreads) {
    const uint32_t c = __ldcg(p.comps + i);
    const uint32_t c2 = __ldcg(p.cother + c);
    const bool mutual = __ldcg(p.cother + c2) == c;
    if (!mutual || c < c2) {
      const uint32_t pos = atomicAdd(&p.ms->edges, 1u);
      if (pos < p.out_cap) __stcg(p.out_edges + pos, __ldcg(p.cedge + c));
      else set_err(&p.st->err, DERR_WL_OVERFLOW);
      atomicAdd(&p.ms->weight, __ldcg(p.cwl + c) >> 32);
    }
    if (!mutual || c > c2) __stcg(p.comp + c, c2);
    __stcg(p.cwl + c, kNoRecord);
  }
}

// One pointer-jumping pass over every vertex; returns this thread's updates.
__device__ uint32_t msf_jump(const MsfParams& p, uint32_t gtid, uint32_t nthreads) {
  uint32_t changed = 0;
  for (uint32_t v = gtid; v < p.n; v += nthreads) {
    const uint32_t c = __ldcg(p.comp + v);
    const uint32_t cc = __ldcg(p.comp + c);
    if (cc != c) {
      __stcg(p.comp + v, cc);
      ++changed;
    }
  }
  return changed;
}

__device__ void msf_init(const MsfParams& p, uint32_t gtid, uint32_t nthreads) {
  for (uint32_t v = gtid; v < p.n; v += nthreads) {
    __stcg(p.comp + v, v);
    __stcg(p.cwl + v, kNoRecord);
    // a held lock: 1 for the CAS forms, a now-serving value no ticket reaches
    __stcg(p.lock + v, v == p.held_lock ? (p.ticket ? kInf : 1u) : 0u);
    if (p.ticket) __stcg(p.ticket + v, 0u);
  }
}

template <int CTA>
__device__ __forceinline__ uint32_t cta_sum_u32(Smem<CTA>& sm, uint32_t x) {
  unsigned long long s = cta_sum_u64<CTA>(sm, x);
  return static_cast<uint32_t>(s);
}

// The outlined Pipe: every kernel invocation of every iteration in one
// cooperative launch.
template <int CTA>
__global__ void __launch_bounds__(CTA, MinBlocks<CTA>::value) k_msf(MsfParams p) {
  __shared__ Smem<CTA> sm;
  init_smem<CTA>(sm);
  DevStatus* st = p.st;
  MsfStatus* ms = p.ms;
  const uint32_t gtid = blockIdx.x * CTA + threadIdx.x, nthreads = gridDim.x * CTA;
  const uint32_t ep0 = __ldcg(&st->epoch);
  uint32_t gen = 0, inv = 0;
  bool ok = true;

  auto begin_invocation = [&]() {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      MsfSlot* s = &ms->slot[(inv + 1) % 3];
      s->out = s->retry = s->comp = s->changed = 0;
    }
    sm.round_pushes = 0;
  };
  auto end_invocation = [&]() -> MsfSlot {
    ok = grid_barrier<CTA>(sm, st, gen, p.timeout_ns);
    MsfSlot r{0, 0, 0, 0};
    if (ok && sm.pub_err == DERR_NONE) {
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(&ms->slot[inv % 3]));
      r = MsfSlot{v.x, v.y, v.z, v.w};
    } else {
      ok = false;
    }
    ++inv;
    return r;
  };

  begin_invocation();
  msf_init(p, gtid, nthreads);
  end_invocation();

  uint32_t cur = 0, in_n = p.n, iters = 0, retries = 0;
  const uint32_t* in = nullptr;  // iteration 0: every vertex
  while (ok) {
    if (iters >= kMsfMaxIters) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(&st->err, DERR_MSF_ITERS);
      break;
    }
    ++iters;
    uint32_t* out = p.items[cur ^ 1u];
    // find_min, then its retries
    uint32_t out_total = 0, comp_total = 0, rb = 0;
    const uint32_t* fin = in;
    uint32_t fin_n = in_n;
    bool backoff = false;
    const unsigned long long t_retry0 = msf_now();
    for (;;) {
      begin_invocation();
      msf_find_min(p, fin, fin_n, backoff, out, out_total, p.retry[rb], &ms->slot[inv % 3], comp_total, gtid,
                   nthreads);
      const MsfSlot s = end_invocation();
      if (!ok) break;
      out_total += s.out;
      comp_total += s.comp;
      retries += s.retry;
      if (s.retry == 0) break;
      // the retries of one find_min end within the lock time limit (every CTA
      // reads the same clock values closely enough; the flag makes it uniform)
      if (threadIdx.x == 0 && msf_now() - t_retry0 > p.lock_timeout_ns) set_err(&st->err, DERR_LOCK_TIMEOUT);
      fin = p.retry[rb];
      fin_n = min(s.retry, p.n);
      rb ^= 1u;
      backoff = true;
    }
    if (!ok || out_total == 0) break;  // no component has a cross edge: the forest is complete
    begin_invocation();
    msf_link(p, min(comp_total, p.n), gtid, nthreads);
    end_invocation();
    for (uint32_t pass = 0; ok; ++pass) {
      begin_invocation();
      sm.round_pushes = 0;
      const uint32_t changed = cta_sum_u32<CTA>(sm, msf_jump(p, gtid, nthreads));
      if (threadIdx.x == 0 && changed) atomicAdd(&ms->slot[inv % 3].changed, changed);
      const MsfSlot s = end_invocation();
      if (s.changed == 0) break;
    }
    in = out;
    in_n = min(out_total, p.n);
    cur ^= 1u;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ms->iterations = iters;
    ms->invocations = inv;
    ms->retries = retries;
  }
  persistent_exit<CTA>(sm, st, ok, inv, 0u, ep0, 0ull, nullptr, 0);
}

// Per-launch form: one kernel per invocation; the host clears the slot it
// counts into and reads it afterwards.
enum : uint32_t { MSF_INIT = 0, MSF_FIND = 1, MSF_FIND_RETRY = 2, MSF_LINK = 3, MSF_JUMP = 4 };

struct MsfStep {
  uint32_t phase;
  const uint32_t* in;
  uint32_t in_n;
  uint32_t* out;
  uint32_t out_base;
  uint32_t* retry_out;
  uint32_t comp_base;
  uint32_t comp_n;
  uint32_t slot;
};

template <int CTA>
__global__ void __launch_bounds__(CTA, MinBlocks<CTA>::value) k_msf_step(MsfParams p, MsfStep s) {
  const uint32_t gtid = blockIdx.x * CTA + threadIdx.x, nthreads = gridDim.x * CTA;
  MsfSlot* slot = &p.ms->slot[s.slot];
  switch (s.phase) {
    case MSF_INIT: msf_init(p, gtid, nthreads); break;
    case MSF_FIND:
    case MSF_FIND_RETRY:
      msf_find_min(p, s.in, s.in_n, s.phase == MSF_FIND_RETRY, s.out, s.out_base, s.retry_out, slot, s.comp_base, gtid,
                   nthreads);
      break;
    case MSF_LINK: msf_link(p, s.comp_n, gtid, nthreads); break;
    case MSF_JUMP: {
      const uint32_t c = msf_jump(p, gtid, nthreads);
      if (c) atomicAdd(&slot->changed, c);
      break;
    }
  }
}

// Block-size sets of the Pipe's kernels (bit b = CTA 128 << b). Each is a
// FixedBlock template (CTA is a template parameter: launch bounds and the
// shared-memory layout of the barrier depend on it) compiled for the four sizes.
constexpr uint32_t kMsfFindMask = 0xFu, kMsfLinkMask = 0xFu, kMsfJumpMask = 0xFu;

template <int CTA>
cudaError_t msf_occupancy(bool outlined, int* nb) {
  return outlined ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_msf<CTA>, CTA, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_msf_step<CTA>, CTA, 0);
}

cudaError_t msf_occupancy_cta(uint32_t cta, bool outlined, int* nb) {
  switch (cta) {
    case 128: return msf_occupancy<128>(outlined, nb);
    case 256: return msf_occupancy<256>(outlined, nb);
    case 512: return msf_occupancy<512>(outlined, nb);
    case 1024: return msf_occupancy<1024>(outlined, nb);
  }
  return cudaErrorInvalidValue;
}

template <int CTA>
cudaError_t msf_launch_outlined(uint32_t grid, const MsfParams& p, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(CTA);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_msf<CTA>, p);
}

cudaError_t msf_launch_outlined_cta(uint32_t cta, uint32_t grid, const MsfParams& p, cudaStream_t s) {
  switch (cta) {
    case 128: return msf_launch_outlined<128>(grid, p, s);
    case 256: return msf_launch_outlined<256>(grid, p, s);
    case 512: return msf_launch_outlined<512>(grid, p, s);
    case 1024: return msf_launch_outlined<1024>(grid, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t msf_launch_step_cta(uint32_t cta, uint32_t grid, const MsfParams& p, const MsfStep& st, cudaStream_t s) {
  switch (cta) {
    case 128: k_msf_step<128><<<grid, 128, 0, s>>>(p, st); break;
    case 256: k_msf_step<256><<<grid, 256, 0, s>>>(p, st); break;
    case 512: k_msf_step<512><<<grid, 512, 0, s>>>(p, st); break;
    case 1024: k_msf_step<1024><<<grid, 1024, 0, s>>>(p, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace irgl

using namespace irgl;

extern "C" {

irgl_status irgl_msf(irgl_ctx* ctx, irgl_graph* g, irgl_mode mode, irgl_lock lock, uint32_t* out_edges,
                     uint32_t cap, int out_on_host, const irgl_tuning* tin, irgl_msf_stats* stats) {
  if (!ctx || !g || !out_edges) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (!g->w) return fail(IRGL_ERR_INVALID_ARG, "the minimum spanning forest needs edge weights");
  if (!(g->flags & IRGL_SYMMETRIC))
    return fail(IRGL_ERR_NOT_SYMMETRIC, "the minimum spanning forest needs a graph loaded with IRGL_SYMMETRIC");
  if (mode != IRGL_PERSISTENT && mode != IRGL_PER_LAUNCH) return fail(IRGL_ERR_INVALID_ARG, "unknown mode");
  if (lock != IRGL_LOCK_BLOCKING && lock != IRGL_LOCK_TICKET && lock != IRGL_LOCK_RETRY)
    return fail(IRGL_ERR_INVALID_ARG, "unknown lock form %d", static_cast<int>(lock));
  const uint32_t n = g->n;
  const uint32_t need = n > 0 ? n - 1 : 0;
  if (cap < need) return fail(IRGL_ERR_INVALID_ARG, "out_edges holds %u edges, a forest may need %u", cap, need);
  irgl_tuning t;
  irgl_status s = resolve_tuning(tin, &t);
  if (s != IRGL_OK) return s;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return IRGL_OK;
  DeviceGuard guard(ctx->device);

  // T_control over find_min, link and jump (Sec. 4.4)
  const uint32_t masks[3] = {kMsfFindMask, kMsfLinkMask, kMsfJumpMask};
  uint32_t cta = 0;
  s = control_cta(masks, 3, t.cta_size, &cta);
  if (s != IRGL_OK) return s;

  // workspace: the status block, then 14 arrays of N words (N a multiple of
  // 64, so every array starts on a 256-byte boundary; cwl takes two)
  const uint64_t n_round = (static_cast<uint64_t>(n) + 63u) & ~63ull;
  if (n_round > 0xFFFFFFC0ull) return fail(IRGL_ERR_INVALID_ARG, "n = %u is too large for the forest workspace", n);
  if (ctx->msf_n < n_round || !ctx->msf_buf) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->msf_buf);
    ctx->msf_buf = nullptr;
    ctx->msf_n = 0;
    const size_t words = static_cast<size_t>(n_round) * 14 + sizeof(MsfStatus) / 4;
    cudaError_t e = cudaMalloc(&ctx->msf_buf, words * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "minimum spanning forest workspace");
    ctx->msf_n = static_cast<uint32_t>(n_round);
  }
  if (!ctx->msf_host) {
    cudaError_t e = cudaMallocHost(&ctx->msf_host, sizeof(MsfStatus));
    if (e != cudaSuccess) return cuda_fail(e, "status staging");
  }
  uint32_t* b = ctx->msf_buf;
  const size_t N = ctx->msf_n;
  MsfParams p;
  std::memset(&p, 0, sizeof(p));
  p.row_ptr = g->row_ptr;
  p.col = g->col;
  p.w = g->w;
  p.n = n;
  MsfStatus* ms = reinterpret_cast<MsfStatus*>(b);  // 128-byte multiple at the start
  uint32_t* a = b + sizeof(MsfStatus) / 4;
  p.comp = a + 0 * N;
  p.cwl = reinterpret_cast<unsigned long long*>(a + 1 * N);  // two arrays' worth
  p.chi = a + 3 * N;
  p.cedge = a + 4 * N;
  p.cother = a + 5 * N;
  p.lock = a + 6 * N;
  p.ticket = lock == IRGL_LOCK_TICKET ? a + 7 * N : nullptr;
  p.items[0] = a + 8 * N;
  p.items[1] = a + 9 * N;
  p.retry[0] = a + 10 * N;
  p.retry[1] = a + 11 * N;
  p.comps = a + 12 * N;
  uint32_t* dev_out = out_on_host ? a + 13 * N : out_edges;
  p.out_edges = dev_out;
  p.out_cap = out_on_host ? n : cap;
  p.lock_mode = static_cast<uint32_t>(lock);
  p.st = ctx->st;
  p.ms = ms;
  p.timeout_ns = ctx->dbg_timeout_us ? ctx->dbg_timeout_us * 1000ull : 2000000000ull;
  p.lock_timeout_ns = p.timeout_ns / 2;
  p.held_lock = ctx->dbg_held_lock < n ? ctx->dbg_held_lock : kInf;
  cudaError_t e = cudaMemsetAsync(ms, 0, sizeof(MsfStatus), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status clear");

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, ctx->stream);
  irgl_msf_stats local;
  std::memset(&local, 0, sizeof(local));
  local.cta_size = cta;
  uint32_t launches = 0, invocations = 0, iters = 0, retries = 0;

  int nb = 0;
  e = msf_occupancy_cta(cta, mode == IRGL_PERSISTENT, &nb);
  if (e != cudaSuccess || nb <= 0) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return e != cudaSuccess ? cuda_fail(e, "occupancy") : fail(IRGL_ERR_CUDA, "MSF kernel cannot be made resident");
  }
  if (t.blocks_per_sm && static_cast<int>(t.blocks_per_sm) < nb) nb = static_cast<int>(t.blocks_per_sm);
  uint32_t grid = static_cast<uint32_t>(nb) * static_cast<uint32_t>(ctx->sm_count);
  if (t.max_blocks && t.max_blocks < grid) grid = t.max_blocks;
  grid = std::max<uint32_t>(1, std::min<uint32_t>(grid, kMaxGrid));
  local.grid = grid;

  if (mode == IRGL_PERSISTENT) {
    e = msf_launch_outlined_cta(cta, grid, p, ctx->stream);
    if (e != cudaSuccess) {
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      return cuda_fail(e, "MSF launch");
    }
    launches = 1;
  } else {
    // the host drives the Pipe: one launch per invocation, counters read in between
    MsfStep st;
    std::memset(&st, 0, sizeof(st));
    auto step = [&](MsfStep& x) -> irgl_status {
      x.slot = 0;
      cudaError_t er = cudaMemsetAsync(&ms->slot[0], 0, sizeof(MsfSlot), ctx->stream);
      if (er == cudaSuccess) er = msf_launch_step_cta(cta, grid, p, x, ctx->stream);
      if (er == cudaSuccess)
        er = cudaMemcpyAsync(ctx->msf_host, ms, sizeof(MsfStatus), cudaMemcpyDeviceToHost, ctx->stream);
      if (er == cudaSuccess) er = cudaStreamSynchronize(ctx->stream);
      if (er != cudaSuccess) return cuda_fail(er, "MSF step");
      ++launches;
      ++invocations;
      return read_status(ctx, nullptr);
    };
    st.phase = MSF_INIT;
    s = step(st);
    uint32_t cur = 0, in_n = n;
    const uint32_t* in = nullptr;
    while (s == IRGL_OK) {
      if (iters >= kMsfMaxIters) {
        s = fail(IRGL_ERR_CUDA, "Boruvka did not converge within %u iterations", kMsfMaxIters);
        break;
      }
      ++iters;
      uint32_t* out = p.items[cur ^ 1u];
      uint32_t out_total = 0, comp_total = 0, rb = 0;
      const uint32_t* fin = in;
      uint32_t fin_n = in_n;
      bool backoff = false;
      const auto t_retry0 = std::chrono::steady_clock::now();
      for (;;) {
        st.phase = backoff ? MSF_FIND_RETRY : MSF_FIND;
        st.in = fin;
        st.in_n = fin_n;
        st.out = out;
        st.out_base = out_total;
        st.retry_out = p.retry[rb];
        st.comp_base = comp_total;
        s = step(st);
        if (s != IRGL_OK) break;
        const MsfSlot r = static_cast<MsfStatus*>(ctx->msf_host)->slot[0];
        out_total += r.out;
        comp_total += r.comp;
        retries += r.retry;
        if (r.retry == 0) break;
        if (std::chrono::steady_clock::now() - t_retry0 > std::chrono::nanoseconds(p.lock_timeout_ns)) {
          s = fail(IRGL_ERR_LOCK_TIMEOUT, "retries of a component lock exceeded the time limit");
          break;
        }
        fin = p.retry[rb];
        fin_n = std::min(r.retry, n);
        rb ^= 1u;
        backoff = true;
      }
      if (s != IRGL_OK || out_total == 0) break;
      st.phase = MSF_LINK;
      st.comp_n = std::min(comp_total, n);
      s = step(st);
      while (s == IRGL_OK) {
        st.phase = MSF_JUMP;
        s = step(st);
        if (s != IRGL_OK || static_cast<MsfStatus*>(ctx->msf_host)->slot[0].changed == 0) break;
      }
      in = out;
      in_n = std::min(out_total, n);
      cur ^= 1u;
    }
    if (s != IRGL_OK) {
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      if (stats) *stats = local;
      return s;
    }
  }
  cudaEventRecord(ev1, ctx->stream);
  e = cudaMemcpyAsync(ctx->msf_host, ms, sizeof(MsfStatus), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return cuda_fail(e, "MSF status readback");
  }
  float ms_elapsed = 0.f;
  cudaEventElapsedTime(&ms_elapsed, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  s = read_status(ctx, nullptr);
  if (s != IRGL_OK) {
    if (stats) *stats = local;
    return s;
  }
  const MsfStatus& h = *static_cast<MsfStatus*>(ctx->msf_host);
  local.edges = h.edges;
  local.weight = h.weight;
  local.locks = h.locks;
  if (mode == IRGL_PERSISTENT) {
    local.iterations = h.iterations;
    local.invocations = h.invocations;
    local.retries = h.retries;
  } else {
    local.iterations = iters;
    local.invocations = invocations;
    local.retries = retries;
  }
  local.launches = launches;
  local.device_ms = ms_elapsed;
  if (h.edges > need) {
    if (stats) *stats = local;
    return fail(IRGL_ERR_CUDA, "forest has %u edges, more than n - 1 = %u", h.edges, need);
  }
  if (out_on_host && h.edges) {
    e = cudaMemcpyAsync(out_edges, dev_out, sizeof(uint32_t) * h.edges, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "forest copy");
  }
  if (stats) *stats = local;
  return IRGL_OK;
}

}  // extern "C"
