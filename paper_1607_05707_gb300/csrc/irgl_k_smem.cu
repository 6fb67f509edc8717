// Iteration-outlined Iterate for graphs that fit in one CTA's shared memory.
//
// The Sec. 3.4 outlining puts every round of an Iterate into one launch and
// separates the rounds by SyncRunningThreads; on a graph of a few thousand
// vertices the rounds are then a chain of dependent global-memory round trips
// (pop, row offsets, column, value, atomic, push) plus a grid barrier, each
// round a few microseconds although it touches a few hundred bytes. When the
// whole graph, its values and both worklists fit in the 227 KB of shared
// memory one CTA may use, a single CTA of 1024 threads copies the CSR in once
// and runs every round there: the grid barrier becomes __syncthreads, every
// access is a shared-memory one, and the values are written back at the end.
// Same operator, worklist discipline (pops from `in`, pushes to `out`, swapped
// each round) and fixed point as the grid-wide kernels; only the schedule of
// the pops differs, which the unique fixed point does not see.
//
// Shared-memory layout (32-bit words): row_ptr[n + 1], col[m], w[m] (SSSP),
// value[n], stamp[n] (SSSP and CC: the round that last pushed the vertex, so
// each vertex is pushed at most once per round), wl[2][n].
#include <algorithm>

#include "irgl_launch.h"

namespace irgl {

namespace {

constexpr int kSmemCta = 1024;
constexpr uint32_t kInitMark = 0xFFFFFFFEu;  // stamp of the round-0 items (CC)

template <uint32_t OP>
__device__ __forceinline__ void smem_push(uint32_t* out, uint32_t* out_n, uint32_t cap, uint32_t v, uint32_t* err) {
  const uint32_t pos = atomicAdd(out_n, 1u);
  if (pos < cap) out[pos] = v;
  else atomicCAS(err, DERR_NONE, DERR_WL_OVERFLOW);
}

// Relax edge k of a popped vertex whose operator value is `val`
// (BFS: the level to assign; SSSP: its distance; CC: its label).
template <uint32_t OP>
__device__ __forceinline__ void smem_relax(const uint32_t* col, const uint32_t* w, uint32_t* val_arr,
                                           uint32_t* stamp, uint32_t k, uint32_t val, uint32_t r, uint32_t* out,
                                           uint32_t* out_n, uint32_t cap, uint32_t* err) {
  const uint32_t v = col[k];
  if (OP == OP_BFS) {
    if (val_arr[v] == kInf && atomicCAS(val_arr + v, kInf, val) == kInf) smem_push<OP>(out, out_n, cap, v, err);
    return;
  }
  const uint32_t nd = OP == OP_SSSP ? val + w[k] : val;
  if (nd >= val_arr[v]) return;
  if (nd < atomicMin(val_arr + v, nd) && atomicExch(stamp + v, r) != r) smem_push<OP>(out, out_n, cap, v, err);
}

template <uint32_t OP>
__global__ void __launch_bounds__(kSmemCta, 1) k_smem_iterate(KParams p) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t s_n[2];
  __shared__ uint32_t s_err;
  __shared__ unsigned long long s_edges;
  const unsigned long long t_start = p.trace ? globaltimer_ns() : 0ull;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t n = p.n;
  const uint32_t m = __ldg(p.row_ptr + n);
  uint32_t* rp = sh;
  uint32_t* col = rp + n + 1;
  uint32_t* w = col + m;
  uint32_t* val = w + (OP == OP_SSSP ? m : 0u);
  uint32_t* stamp = val + n;
  uint32_t* wl0 = stamp + (OP == OP_BFS ? 0u : n);
  uint32_t* wl1 = wl0 + n;
  if (tid == 0) {
    s_n[0] = 0;
    s_n[1] = 0;
    s_err = DERR_NONE;
    s_edges = 0;
  }
  // the graph, once (plain loads; the CSR arrays are read-only here)
  for (uint32_t i = tid; i <= n; i += kSmemCta) rp[i] = __ldg(p.row_ptr + i);
  for (uint32_t i = tid; i < m; i += kSmemCta) col[i] = __ldg(p.col + i);
  if (OP == OP_SSSP)
    for (uint32_t i = tid; i < m; i += kSmemCta) w[i] = static_cast<uint32_t>(__ldg(p.w + i));
  // Iterate initial values: BFS/SSSP INF (sources 0 below), CC label v
  for (uint32_t v = tid; v < n; v += kSmemCta) {
    val[v] = OP == OP_CC ? v : kInf;
    if (OP != OP_BFS) stamp[v] = kInf;
  }
  __syncthreads();
  // round-0 worklist: the caller's initial items (CC without them: every vertex)
  const uint32_t init_n = p.init_count ? min(__ldcg(p.init_count), p.init_cap) : n;
  for (uint32_t i = tid; i < init_n; i += kSmemCta) {
    const uint32_t s = p.init_items ? __ldcg(p.init_items + i) : i;
    if (s >= n) {
      atomicCAS(&s_err, DERR_NONE, DERR_BAD_ITEM);
      continue;
    }
    if (OP == OP_CC) {
      // a repeated item is pushed once (a mark no round id reaches: rounds stay below n)
      if (atomicExch(stamp + s, kInitMark) != kInitMark) smem_push<OP>(wl0, &s_n[0], n, s, &s_err);
    } else if (atomicExch(val + s, 0u) != 0u) {  // a repeated source is pushed once
      smem_push<OP>(wl0, &s_n[0], n, s, &s_err);
    }
  }
  __syncthreads();
  trace_prologue(p.trace, p.trace_cap, t_start, s_n[0]);
  uint32_t edges = 0, rounds = 0, last_out = 0;
  for (uint32_t r = 0;; ++r) {
    uint32_t* in = (r & 1) ? wl1 : wl0;
    uint32_t* out = (r & 1) ? wl0 : wl1;
    uint32_t* out_n = &s_n[(r + 1) & 1];
    const uint32_t in_n = min(s_n[r & 1], n);  // a worklist holds at most n items
    // every thread has read in_n before the counter is reused two rounds on
    __syncthreads();
    if (tid == 0) *out_n = 0;
    __syncthreads();
    for (uint32_t base = 0; base < in_n; base += kSmemCta) {
      const uint32_t i = base + tid;
      uint32_t b = 0, e = 0, x = 0;
      if (i < in_n) {
        const uint32_t u = in[i];
        b = rp[u];
        e = rp[u + 1];
        x = OP == OP_BFS ? r + 1u : val[u];
      }
      edges += e - b;
      // short lists by their own thread, long ones by the whole warp
      bool lng = e - b > 8u;
      if (!lng)
        for (uint32_t k = b; k < e; ++k) smem_relax<OP>(col, w, val, stamp, k, x, r, out, out_n, n, &s_err);
      for (;;) {
        const unsigned mk = __ballot_sync(kFull, lng);
        if (mk == 0) break;
        const int ld = __ffs(mk) - 1;
        const uint32_t lb = __shfl_sync(kFull, b, ld), le = __shfl_sync(kFull, e, ld);
        const uint32_t lx = __shfl_sync(kFull, x, ld);
        for (uint32_t k = lb + lane; k < le; k += 32) smem_relax<OP>(col, w, val, stamp, k, lx, r, out, out_n, n, &s_err);
        if (lane == static_cast<uint32_t>(ld)) lng = false;
      }
    }
    __syncthreads();
    last_out = min(*out_n, n);
    rounds = r + 1;
    trace_round(p.trace, p.trace_cap, rounds, in_n, last_out);
    if (last_out == 0 || s_err != DERR_NONE) break;
    if (rounds >= p.max_rounds) {
      if (tid == 0) atomicCAS(&s_err, DERR_NONE, DERR_MAX_ROUNDS);
      break;
    }
  }
  for (uint32_t v = tid; v < n; v += kSmemCta) __stcg(p.state + v, val[v]);
  atomicAdd(&s_edges, static_cast<unsigned long long>(edges));
  __syncthreads();
  trace_end(p.trace, p.trace_cap, rounds);
  if (tid == 0) {
    DevStatus* st = p.st;
    atomicAdd(&st->edges, s_edges);
    st->rounds = rounds;
    st->last_out = last_out;
    if (s_err != DERR_NONE) atomicCAS(&st->err, DERR_NONE, s_err);
  }
}

template <uint32_t OP>
cudaError_t launch_op(const KParams& p, size_t bytes, cudaStream_t s) {
  // the opt-in size is set per launch: cheap, and correct on any device current
  cudaError_t e = cudaFuncSetAttribute(k_smem_iterate<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  k_smem_iterate<OP><<<1, kSmemCta, bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t smem_iterate_bytes(uint32_t op, uint32_t n, uint64_t m) {
  const uint64_t words = (n + 1ull) + m + (op == OP_SSSP ? m : 0ull) + n + (op == OP_BFS ? 0ull : n) + 2ull * n;
  return static_cast<size_t>(4ull * words);
}

bool smem_iterate_fits(uint32_t op, uint32_t n, uint64_t m, size_t limit) {
  if (op != OP_BFS && op != OP_SSSP && op != OP_CC) return false;
  if (n == 0 || m >= 0xFFFFFFFFull) return false;
  return smem_iterate_bytes(op, n, m) <= limit;
}

cudaError_t launch_smem_iterate(uint32_t op, const KParams& p, uint64_t m, cudaStream_t s) {
  const size_t bytes = smem_iterate_bytes(op, p.n, m);
  switch (op) {
    case OP_BFS: return launch_op<OP_BFS>(p, bytes, s);
    case OP_SSSP: return launch_op<OP_SSSP>(p, bytes, s);
    case OP_CC: return launch_op<OP_CC>(p, bytes, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace irgl
