// Serving loop: continuous batching of BFS/SSSP queries into epochs of the
// batched persistent kernel.
//
// A host worker thread repeats:
//   1. admission: take queued queries in arrival order while a slot is free and
//      the query's state (20 bytes per vertex: the packed (value, round id)
//      word, the u32 result and two worklist entries; 32 with near-far, which
//      adds two far-list entries and a far stamp) fits in the device arena
//      (first-fit over free ranges); the arena is sized from free HBM when the
//      server starts;
//   2. upload the sorted descriptor table of the active queries and the new
//      queries' sources; the admission kernels write their initial values and
//      append their sources to the pending worklist, which still holds the
//      unfinished work of the queries already running;
//   3. one epoch: the batched persistent kernel runs at most epoch_rounds
//      rounds over the union of all active queries' worklist items; the next
//      step launches the following epoch before it reads this one back, so
//      the host's bookkeeping overlaps the GPU's work (a query found finished
//      one epoch late sat inert in that epoch: it had no items);
//   4. queries that pushed nothing in the epoch's last round are finished:
//      one kernel extracts all their results and counts their reached edges,
//      then their results are copied to the callers' host buffers (or a
//      scratch buffer) on a second stream while the next epochs run; once a
//      copy has landed, the query's completion time is stamped and its arena
//      range and slot are released (at most 8 epochs' copies in flight).
// The host/device boundary is crossed once per epoch and every device wait is
// bounded, so no kernel spins indefinitely while the server idles.
//
// Queries on large graphs (solo_min_n vertices or more; by default those whose
// state and stamps exceed half the L2) do not join the arena: between epochs
// the worker runs one of them alone as a persistent single-query Iterate on a
// private context bound to the server's stream. Such a query has enough
// parallelism per round to fill the GPU, and alone its state stays in L2,
// where in the arena every state access of every query would miss it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

using namespace irgl;

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  irgl_graph* g = nullptr;
  uint32_t op = 0;
  uint32_t src = 0;
  uint32_t* host_out = nullptr;
  double t_submit = 0;
};

struct Active {
  Request rq;
  uint32_t slot = 0;
  uint32_t base = 0;
  uint32_t n = 0;
};

// An epoch launched and not yet read back: the queries it ran over.
struct EpochRec {
  bool live = false;
  std::vector<Active> set;
};

// Queries that finished in one epoch whose results are still being copied to
// host memory on the copy stream: their slots and arena ranges are released,
// and their completion published, once `ev` has completed.
struct Pending {
  std::vector<Active> fin;
  std::vector<uint32_t> rounds;
  unsigned long long* h_edges = nullptr;  // per slot, from the ring of pinned buffers
  cudaEvent_t ev = nullptr;
  uint32_t ring = 0;                       // ring entry holding h_edges and ev
  // a query that ran alone: its request, rounds and edge count (h_edges[0])
  bool solo = false;
  Request rq;
  uint32_t solo_rounds = 0;
};

struct Done {
  int32_t status = IRGL_OK;
  uint32_t rounds = 0;
  double t_submit = 0;
  double t_done = 0;
  uint64_t edges = 0;  // out-edges of reached vertices (when counting is on)
};

// First-fit allocator over [0, cap) in entries.
struct Arena {
  std::map<uint64_t, uint64_t> free_;  // base -> size
  uint64_t cap = 0;
  void init(uint64_t c) {
    cap = c;
    free_.clear();
    if (c) free_[0] = c;
  }
  bool alloc(uint64_t n, uint64_t* base) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *base = it->first;
        const uint64_t rest = it->second - n;
        const uint64_t nb = it->first + n;
        free_.erase(it);
        if (rest) free_[nb] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t base, uint64_t n) {
    if (n == 0) return;
    auto it = free_.emplace(base, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

// Out-edges of reached vertices of one finished query: sum of out-degrees over
// state[v] != INF (measurement only).
__global__ void k_reached_edges(const uint32_t* __restrict__ state, const uint32_t* __restrict__ row_ptr, uint32_t n,
                                unsigned long long* out) {
  unsigned long long s = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (__ldcg(state + v) != kInf) s += __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// One finished query of an epoch: its arena range, the exclusive prefix of n
// over the epoch's finished queries, its slot and its graph's row offsets.
struct FinDesc {
  const uint32_t* row_ptr;
  uint32_t base, n, pre, slot;
};

// Every query that finished in an epoch at once: results from the packed words
// (when ds is set) into the u32 arena and, with count_edges, the out-edges of
// reached vertices per slot (one atomic per run of same-query lanes in a warp).
__global__ void k_finish(const FinDesc* __restrict__ fd, uint32_t nf, uint32_t total,
                         const unsigned long long* __restrict__ ds, uint32_t* state, unsigned long long* edge_cnt,
                         int count_edges) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t w0 = tid - lane; w0 < total; w0 += nthreads) {  // warp-uniform trip count
    const uint32_t i = static_cast<uint32_t>(w0) + lane;
    uint32_t j = 0, e = 0;
    if (i < total) {
      uint32_t lo = 0, hi = nf - 1;
      while (lo < hi) {
        const uint32_t md = (lo + hi + 1) >> 1;
        if (__ldg(&fd[md].pre) <= i) lo = md;
        else hi = md - 1;
      }
      j = lo;
      const uint32_t v = i - __ldg(&fd[j].pre);
      const uint32_t item = __ldg(&fd[j].base) + v;
      uint32_t val;
      if (ds != nullptr) {
        val = static_cast<uint32_t>(__ldcg(ds + item) >> 32);
        __stcg(state + item, val);
      } else {
        val = __ldcg(state + item);
      }
      if (count_edges && val != kInf) {
        const uint32_t* rp = fd[j].row_ptr;
        e = __ldg(rp + v + 1) - __ldg(rp + v);
      }
    }
    if (count_edges) {
      const unsigned act = __ballot_sync(kFull, i < total);
      if (i < total) {
        // lanes of one query: their degrees summed in two 16-bit halves (no overflow in 32 lanes)
        const unsigned grp = __match_any_sync(act, j);
        const unsigned long long sum = static_cast<unsigned long long>(__reduce_add_sync(grp, e & 0xFFFFu)) +
                                       (static_cast<unsigned long long>(__reduce_add_sync(grp, e >> 16)) << 16);
        if (static_cast<uint32_t>(__ffs(grp) - 1) == lane && sum) atomicAdd(edge_cnt + fd[j].slot, sum);
      }
    }
  }
}

struct irgl_server {
  irgl_ctx* ctx = nullptr;
  irgl_server_config cfg{};
  cudaStream_t stream = nullptr;
  // result copies of finished queries run here, overlapping the next epochs
  cudaStream_t copy_stream = nullptr;
  static constexpr uint32_t kRing = 8;      // epochs whose copies may be in flight
  unsigned long long* h_edge_ring = nullptr;  // kRing x max_slots pinned edge counts
  cudaEvent_t ring_ev[kRing] = {};
  std::vector<uint32_t> ring_free;
  std::deque<Pending> pending;               // worker thread only
  // device
  DevStatus* st = nullptr;
  DevStatus* st_host = nullptr;        // pinned, two: one per launch parity
  uint32_t* state = nullptr;           // results (extracted from ds when a query finishes)
  uint32_t* stamp = nullptr;           // two-array form only (IRGL_TUNE_NO_PACKED)
  unsigned long long* ds = nullptr;    // packed (value, round id) arena
  uint32_t* items[2] = {nullptr, nullptr};
  uint32_t* qlast = nullptr;
  uint32_t* cont = nullptr;
  uint32_t* far_items[2] = {nullptr, nullptr};  // near-far (tuning delta != 0): far lists
  uint32_t* far_stamp = nullptr;                //   arena: round id of the far list a vertex was last put on
  uint32_t* blim = nullptr;                     //   per slot: the SSSP query's limit
  QDesc* desc = nullptr;
  uint32_t* sbases = nullptr;
  QNew* qnew = nullptr;
  uint32_t* srcs = nullptr;
  unsigned long long* edge_cnt = nullptr;
  FinDesc* fin = nullptr;              // the epoch's finished queries (k_finish)
  uint4* big_e = nullptr;
  unsigned long long* big_off = nullptr;
  uint32_t big_cap = 0;
  // pinned staging
  // pinned staging, two halves of max_slots entries each (by launch parity), so an epoch's
  // uploads and read-backs never share a buffer with the next epoch's
  QDesc* h_desc = nullptr;
  uint32_t* h_sbases = nullptr;
  QNew* h_qnew = nullptr;
  uint32_t* h_srcs = nullptr;
  uint32_t* h_qlast = nullptr;
  uint32_t* h_qfirst = nullptr;
  FinDesc* h_fin = nullptr;
  uint32_t* qfirst = nullptr;  // device, per slot: the round id the query was admitted at
  // epochs in flight: epoch k+1 is launched before epoch k is read back
  EpochRec rec[2];
  uint32_t par = 0;            // parity of the next launch
  cudaEvent_t ep_ev[4] = {};   // start / end of the epoch kernel, per parity
  cudaEvent_t st_ev[2] = {};   // the epoch's status read-back has landed, per parity
  uint32_t* h_scratch = nullptr;  // result sink for queries without a host buffer
  uint64_t scratch_n = 0;
  uint64_t arena_n = 0;
  uint32_t grid = 0;
  uint32_t sub_rounds = 0;  // CTA-local sub-rounds of the batched kernel (packed arena only)
  uint32_t id_step = 1;     // round ids per round: 1 + sub_rounds
  irgl_tuning t{};
  Arena arena;
  std::vector<uint32_t> free_slots;
  std::vector<Active> active;  // sorted by base
  // queue and results
  std::mutex mu;
  std::condition_variable cv;
  std::condition_variable cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0, rejected = 0, epochs = 0, rounds_total = 0;
  uint64_t edges_total = 0;
  double busy_s = 0;
  double kernel_s = 0;  // CUDA-event time of the epoch kernels
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int32_t fatal = IRGL_OK;
  bool stop = false;
  std::thread worker;
  // queries that run alone
  uint32_t solo_min_n = 0xFFFFFFFFu;
  irgl_ctx* solo_ctx = nullptr;
  std::deque<Request> solo_q;
  uint32_t* solo_state[2] = {nullptr, nullptr};  // device result buffers, alternated so a
  uint64_t solo_cap[2] = {0, 0};                  // result copy overlaps the next solo query
  cudaEvent_t solo_copied[2] = {nullptr, nullptr};  // the last copy out of each buffer
  uint32_t solo_next = 0;
  uint64_t solo_done = 0;
};

namespace {

void server_free(irgl_server* s) {
  cudaFree(s->st);
  cudaFree(s->state);
  cudaFree(s->stamp);
  cudaFree(s->ds);
  cudaFree(s->items[0]);
  cudaFree(s->items[1]);
  cudaFree(s->qlast);
  cudaFree(s->cont);
  cudaFree(s->far_items[0]);
  cudaFree(s->far_items[1]);
  cudaFree(s->far_stamp);
  cudaFree(s->blim);
  cudaFree(s->desc);
  cudaFree(s->sbases);
  cudaFree(s->qnew);
  cudaFree(s->srcs);
  cudaFree(s->edge_cnt);
  cudaFree(s->fin);
  cudaFree(s->big_e);
  cudaFree(s->big_off);
  if (s->st_host) cudaFreeHost(s->st_host);
  if (s->h_desc) cudaFreeHost(s->h_desc);
  if (s->h_sbases) cudaFreeHost(s->h_sbases);
  if (s->h_qnew) cudaFreeHost(s->h_qnew);
  if (s->h_srcs) cudaFreeHost(s->h_srcs);
  if (s->h_qlast) cudaFreeHost(s->h_qlast);
  if (s->h_fin) cudaFreeHost(s->h_fin);
  if (s->h_scratch) cudaFreeHost(s->h_scratch);
  if (s->ev[0]) cudaEventDestroy(s->ev[0]);
  if (s->ev[1]) cudaEventDestroy(s->ev[1]);
  for (int i = 0; i < 4; ++i)
    if (s->ep_ev[i]) cudaEventDestroy(s->ep_ev[i]);
  for (int i = 0; i < 2; ++i)
    if (s->st_ev[i]) cudaEventDestroy(s->st_ev[i]);
  cudaFree(s->qfirst);
  if (s->h_qfirst) cudaFreeHost(s->h_qfirst);
  for (uint32_t i = 0; i < irgl_server::kRing; ++i)
    if (s->ring_ev[i]) cudaEventDestroy(s->ring_ev[i]);
  if (s->h_edge_ring) cudaFreeHost(s->h_edge_ring);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (int i = 0; i < 2; ++i) {
    cudaFree(s->solo_state[i]);
    if (s->solo_copied[i]) cudaEventDestroy(s->solo_copied[i]);
  }
  if (s->solo_ctx) irgl_ctx_destroy(s->solo_ctx);
  if (s->stream) cudaStreamDestroy(s->stream);
}

// Ensure the pinned result sink holds n entries (worker thread only).
cudaError_t ensure_scratch(irgl_server* s, uint64_t n) {
  if (n <= s->scratch_n) return cudaSuccess;
  cudaStreamSynchronize(s->copy_stream);  // copies into the old sink may still be in flight
  if (s->h_scratch) cudaFreeHost(s->h_scratch);
  s->h_scratch = nullptr;
  s->scratch_n = 0;
  cudaError_t e = cudaMallocHost(&s->h_scratch, sizeof(uint32_t) * n);
  if (e == cudaSuccess) s->scratch_n = n;
  return e;
}

// One query alone: persistent single-query Iterate on the private context,
// then the reached-edge count and the result copy, all on the server's stream.
void retire_pending(irgl_server* s, bool wait);

// One query on a large graph, alone: a persistent single-query Iterate on the
// private context (the server's stream), its reached edges counted, then its
// result copied to host memory on the copy stream while the worker moves on;
// the query is published when the copy lands. Two result buffers alternate,
// the stream waiting for a buffer's last copy before reusing it.
void solo_step(irgl_server* s, const Request& rq) {
  const double t0 = now_s();
  const uint32_t n = rq.g->n;
  const uint32_t k = s->solo_next;
  s->solo_next ^= 1u;
  cudaError_t e = cudaSuccess;
  if (!s->solo_copied[k]) e = cudaEventCreateWithFlags(&s->solo_copied[k], cudaEventDisableTiming);
  if (e == cudaSuccess && n > s->solo_cap[k]) {
    cudaEventSynchronize(s->solo_copied[k]);  // nothing may still read the old buffer
    cudaFree(s->solo_state[k]);
    s->solo_state[k] = nullptr;
    s->solo_cap[k] = 0;
    e = cudaMalloc(&s->solo_state[k], sizeof(uint32_t) * std::max<uint32_t>(n, 4));
    if (e == cudaSuccess) s->solo_cap[k] = n;
  }
  uint32_t* dst = rq.host_out;
  if (!dst && e == cudaSuccess) {
    e = ensure_scratch(s, n);
    dst = s->h_scratch;
  }
  if (e == cudaSuccess && s->ring_free.empty()) retire_pending(s, true);
  // the buffer's previous result copy finishes before this query writes it
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->solo_copied[k], 0);
  irgl_stats st;
  std::memset(&st, 0, sizeof(st));
  irgl_status r = e == cudaSuccess ? IRGL_OK : IRGL_ERR_OOM;
  float kms = 0.f;
  if (r == IRGL_OK) {
    cudaEventRecord(s->ev[0], s->stream);
    const uint32_t src = rq.src;
    // alone, a query takes the single-query defaults plus the server's
    // direction-optimising BFS and round-form flags (the batched kernel's CTA
    // size and sub-rounds are choices for many small queries, not for this one)
    irgl_tuning solo_t = default_tuning();
    solo_t.flags = s->t.flags & (IRGL_TUNE_NO_BCAST | IRGL_TUNE_THREAD_BIN |
                                 (rq.op == IRGL_BFS ? IRGL_TUNE_DIROPT : 0u));
    r = irgl_run(s->solo_ctx, static_cast<irgl_kernel>(rq.op), rq.g, &src, 1, s->solo_state[k], 0, IRGL_PERSISTENT,
                 &solo_t, 0, &st);
    cudaEventRecord(s->ev[1], s->stream);
  }
  if (r == IRGL_OK) {
    Pending pd;
    pd.solo = true;
    pd.rq = rq;
    pd.solo_rounds = st.rounds;
    pd.ring = s->ring_free.back();
    s->ring_free.pop_back();
    pd.h_edges = s->h_edge_ring + static_cast<size_t>(pd.ring) * s->cfg.max_slots;
    pd.ev = s->ring_ev[pd.ring];
    e = cudaMemsetAsync(s->edge_cnt, 0, sizeof(unsigned long long), s->stream);
    if (e == cudaSuccess && s->cfg.count_edges) {
      k_reached_edges<<<static_cast<uint32_t>(s->ctx->sm_count), 256, 0, s->stream>>>(s->solo_state[k],
                                                                                     rq.g->row_ptr, n, s->edge_cnt);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pd.h_edges, s->edge_cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, pd.ev, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, s->solo_state[k], sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                          s->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->solo_copied[k], s->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->copy_stream);
    if (e == cudaSuccess) cudaEventElapsedTime(&kms, s->ev[0], s->ev[1]);  // irgl_run waited for the kernel
    if (e == cudaSuccess) {
      s->pending.push_back(std::move(pd));
    } else {
      s->ring_free.push_back(pd.ring);
      r = IRGL_ERR_CUDA;
    }
  }
  const double t_done = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  s->rounds_total += st.rounds;
  s->busy_s += t_done - t0;
  s->kernel_s += kms * 1e-3;
  if (r != IRGL_OK) {  // published now, with its error
    Done d;
    d.status = r;
    d.t_submit = rq.t_submit;
    d.t_done = t_done;
    s->done[rq.ticket] = d;
    s->completed += 1;
    s->solo_done += 1;
    s->cv_done.notify_all();
  }
}

// Publish the queries of finished epochs whose result copies have completed
// (in epoch order; `wait`: block on the oldest), releasing their slots and
// arena ranges. Worker thread only.
void retire_pending(irgl_server* s, bool wait) {
  while (!s->pending.empty()) {
    Pending& pd = s->pending.front();
    cudaError_t e = wait ? cudaEventSynchronize(pd.ev) : cudaEventQuery(pd.ev);
    if (e == cudaErrorNotReady) return;
    const double t_done = now_s();
    if (pd.solo) {
      std::lock_guard<std::mutex> lk(s->mu);
      Done d;
      d.status = e == cudaSuccess ? IRGL_OK : IRGL_ERR_CUDA;
      d.rounds = pd.solo_rounds;
      d.t_submit = pd.rq.t_submit;
      d.t_done = t_done;
      d.edges = (e == cudaSuccess && s->cfg.count_edges) ? pd.h_edges[0] : 0;
      s->edges_total += d.edges;
      s->done[pd.rq.ticket] = d;
      s->completed += 1;
      s->solo_done += 1;
    } else {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t k = 0; k < pd.fin.size(); ++k) {
        const Active& a = pd.fin[k];
        Done d;
        d.status = e == cudaSuccess ? IRGL_OK : IRGL_ERR_CUDA;
        d.rounds = pd.rounds[k];
        d.t_submit = a.rq.t_submit;
        d.t_done = t_done;
        d.edges = s->cfg.count_edges ? pd.h_edges[a.slot] : 0;
        s->edges_total += d.edges;
        s->done[a.rq.ticket] = d;
        s->completed += 1;
        s->arena.release(a.base, a.n ? a.n : 1);
        s->free_slots.push_back(a.slot);
      }
    }
    s->ring_free.push_back(pd.ring);
    s->pending.pop_front();
    s->cv_done.notify_all();
    wait = false;  // block on one epoch at most
  }
}

// One scheduling step of the worker: admit, launch the next epoch over every
// active query, then read back the epoch launched by the previous step (its
// status copies precede this launch on the stream, so the GPU stays busy while
// the host decides which of its queries finished). A query found finished is
// inert in the epoch already running (it has no items), and is dropped from the
// following one. Returns false when there was nothing to do.
bool server_step(irgl_server* s) {
  const uint32_t S = s->cfg.max_slots;
  const uint32_t p = s->par;  // parity of this step's launch
  const uint32_t q = p ^ 1u;  // the epoch launched by the previous step
  std::vector<Active> fresh;
  retire_pending(s, false);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->queue.empty() && s->active.empty() && !s->rec[q].live) {  // no batched work: finish the copies
      lk.unlock();
      retire_pending(s, true);
      return false;
    }
    while (!s->queue.empty() && !s->free_slots.empty()) {
      Request& rq = s->queue.front();
      uint64_t base = 0;
      if (!s->arena.alloc(rq.g->n ? rq.g->n : 1, &base)) break;  // wait for memory to free up
      Active a;
      a.rq = rq;
      a.slot = s->free_slots.back();
      s->free_slots.pop_back();
      a.base = static_cast<uint32_t>(base);
      a.n = rq.g->n;
      fresh.push_back(a);
      s->queue.pop_front();
    }
  }
  const double t0 = now_s();
  cudaError_t e = cudaSuccess;
  // admission of new queries: descriptors, sources, initial values, pending items
  if (!fresh.empty()) {
    QNew* hq = s->h_qnew + static_cast<size_t>(p) * S;
    uint32_t* hs = s->h_srcs + static_cast<size_t>(p) * S;
    uint32_t nsrc = 0, pre = 0;
    for (size_t j = 0; j < fresh.size(); ++j) {
      const Active& a = fresh[j];
      hq[j] = QNew{a.base, a.n, a.rq.op, a.slot, nsrc, 1, pre, 0};
      hs[nsrc++] = a.rq.src;
      pre += a.n;
    }
    AdmitParams ap{};
    ap.qn = s->qnew;
    ap.nnew = static_cast<uint32_t>(fresh.size());
    ap.total = pre;
    ap.srcs = s->srcs;
    ap.state = s->state;
    ap.ds = s->ds;
    ap.qlast = s->qlast;
    ap.qfirst = s->qfirst;
    ap.items[0] = s->items[0];
    ap.items[1] = s->items[1];
    ap.cap = static_cast<uint32_t>(s->arena_n);
    ap.cont = s->cont;
    ap.st = s->st;
    ap.blim = s->blim;
    ap.delta = s->blim ? s->t.delta : 0u;
    ap.id_step = s->id_step;
    e = cudaMemcpyAsync(s->qnew, hq, sizeof(QNew) * fresh.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->srcs, hs, sizeof(uint32_t) * nsrc, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_admit(ap, static_cast<uint32_t>(s->ctx->sm_count) * 4, s->stream);
    for (auto& a : fresh) s->active.push_back(a);
    std::sort(s->active.begin(), s->active.end(), [](const Active& x, const Active& y) { return x.base < y.base; });
  }
  // one epoch over every active query, sorted by base
  const uint32_t nq = static_cast<uint32_t>(s->active.size());
  if (nq && e == cudaSuccess) {
    QDesc* hd = s->h_desc + static_cast<size_t>(p) * S;
    uint32_t* hb = s->h_sbases + static_cast<size_t>(p) * S;
    QDesc* dd = s->desc + static_cast<size_t>(p) * S;
    uint32_t* db = s->sbases + static_cast<size_t>(p) * S;
    for (uint32_t i = 0; i < nq; ++i) {
      const Active& a = s->active[i];
      hd[i] = QDesc{a.rq.g->row_ptr, a.rq.g->col, a.rq.g->w, a.n, a.rq.op, a.base, a.slot};
      hb[i] = a.base;
    }
    e = cudaMemcpyAsync(dd, hd, sizeof(QDesc) * nq, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, hb, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, s->stream);
    BParams bp{};
    bp.desc = dd;
    bp.sbases = db;
    bp.nq = nq;
    bp.state = s->state;
    bp.stamp = s->stamp;
    bp.ds = s->ds;
    bp.qlast = s->qlast;
    bp.items[0] = s->items[0];
    bp.items[1] = s->items[1];
    bp.cap = static_cast<uint32_t>(s->arena_n);
    bp.cont = s->cont;
    bp.st = s->st;
    bp.tn = Tune{s->t.warp_thresh, s->t.cta_thresh, s->t.chunk, thread_bin(s->t)};
    bp.max_rounds = s->cfg.epoch_rounds;
    bp.rounds_cap_is_error = 0;
    bp.timeout_ns = 2000000000ull;
    bp.time_limit_ns = run_time_limit_ns(s->ctx);
    bp.spread = s->ctx->dbg_no_spread ? 0u : 1u;
    bp.big = (s->t.flags & IRGL_TUNE_NO_SPLIT) ? BigList{nullptr, nullptr, 0} : BigList{s->big_e, s->big_off, s->big_cap};
    bp.delta = s->blim ? s->t.delta : 0u;
    bp.blim = s->blim;
    bp.far_items[0] = s->far_items[0];
    bp.far_items[1] = s->far_items[1];
    bp.far_cap = s->blim ? static_cast<uint32_t>(s->arena_n) : 0u;
    bp.far_stamp = s->far_stamp;
    bp.local_rounds = s->sub_rounds;
    if (e == cudaSuccess) e = cudaEventRecord(s->ep_ev[2 * p], s->stream);
    if (e == cudaSuccess) e = launch_batch_iterate(s->t.cta_size, s->grid, bp, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ep_ev[2 * p + 1], s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->st_host + p, s->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->h_qlast + static_cast<size_t>(p) * S, s->qlast, sizeof(uint32_t) * S,
                          cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->h_qfirst + static_cast<size_t>(p) * S, s->qfirst, sizeof(uint32_t) * S,
                          cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->st_ev[p], s->stream);
    s->rec[p].live = true;
    s->rec[p].set = s->active;
    s->par = q;
  }
  // read back the previous step's epoch
  uint32_t rounds = 0;
  bool read_back = false;
  if (s->rec[q].live && e == cudaSuccess) {
    read_back = true;
    e = cudaEventSynchronize(s->st_ev[q]);
    const DevStatus& sh = s->st_host[q];
    if (e != cudaSuccess || sh.err != DERR_NONE) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->fatal = e != cudaSuccess ? IRGL_ERR_CUDA
                                  : (sh.err == DERR_WL_OVERFLOW ? IRGL_ERR_WL_OVERFLOW : IRGL_ERR_BARRIER_TIMEOUT);
      s->stop = true;
      s->cv_done.notify_all();
      return false;
    }
    rounds = sh.rounds;
    float kms = 0.f;
    if (cudaEventElapsedTime(&kms, s->ep_ev[2 * q], s->ep_ev[2 * q + 1]) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->kernel_s += kms * 1e-3;
    }
    const uint32_t last_ep = sh.epoch - s->id_step;  // round id of the epoch's last round
    const uint32_t* hl = s->h_qlast + static_cast<size_t>(q) * S;
    const uint32_t* hf = s->h_qfirst + static_cast<size_t>(q) * S;
    // finished queries: no push in the epoch's last round. Only queries still
    // active count: one already finished by the previous read-back also sat,
    // inert, in this epoch's set
    std::vector<uint64_t> live_ticket(S, ~uint64_t{0});
    for (auto& a : s->active) live_ticket[a.slot] = a.rq.ticket;
    std::vector<Active> fin;
    std::vector<char> done_slot(S, 0);
    for (auto& a : s->rec[q].set) {
      if (live_ticket[a.slot] != a.rq.ticket) continue;
      if (hl[a.slot] < last_ep || rounds == 0) {
        fin.push_back(a);
        done_slot[a.slot] = 1;
      }
    }
    s->rec[q].live = false;
    s->rec[q].set.clear();
    if (!fin.empty()) {
      std::vector<Active> keep;
      keep.reserve(s->active.size());
      for (auto& a : s->active)
        if (!done_slot[a.slot]) keep.push_back(a);
      s->active.swap(keep);
    }
    // result sink for queries without a caller buffer (only this thread touches it)
    uint64_t need = 0;
    for (auto& a : fin)
      if (!a.rq.host_out) need = std::max<uint64_t>(need, a.n);
    if (e == cudaSuccess) e = ensure_scratch(s, need);
    // every finished query's result and reached edges in one kernel (after the
    // epoch now running: these queries are inert in it); the result copies run
    // on the copy stream, and the queries are published (slots and arena
    // released) once they have landed
    if (!fin.empty() && e == cudaSuccess) {
      if (s->ring_free.empty()) retire_pending(s, true);  // at most kRing epochs in flight
      Pending pd;
      pd.ring = s->ring_free.back();
      s->ring_free.pop_back();
      pd.h_edges = s->h_edge_ring + static_cast<size_t>(pd.ring) * S;
      pd.ev = s->ring_ev[pd.ring];
      FinDesc* hfd = s->h_fin + static_cast<size_t>(q) * S;
      uint64_t total = 0;
      for (size_t k = 0; k < fin.size(); ++k) {
        const Active& a = fin[k];
        hfd[k] = FinDesc{a.rq.g->row_ptr, a.base, a.n, static_cast<uint32_t>(total), a.slot};
        total += a.n;
        pd.rounds.push_back(static_cast<uint32_t>(static_cast<int32_t>(hl[a.slot] - hf[a.slot]) /
                                                  static_cast<int32_t>(s->id_step) + 2));
      }
      e = cudaMemcpyAsync(s->fin, hfd, sizeof(FinDesc) * fin.size(), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess && s->cfg.count_edges)
        e = cudaMemsetAsync(s->edge_cnt, 0, sizeof(unsigned long long) * S, s->stream);
      if (e == cudaSuccess && total) {
        k_finish<<<static_cast<uint32_t>(s->ctx->sm_count) * 4, 256, 0, s->stream>>>(
            s->fin, static_cast<uint32_t>(fin.size()), static_cast<uint32_t>(total), s->ds, s->state, s->edge_cnt,
            s->cfg.count_edges ? 1 : 0);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && s->cfg.count_edges)
        e = cudaMemcpyAsync(pd.h_edges, s->edge_cnt, sizeof(unsigned long long) * S, cudaMemcpyDeviceToHost,
                            s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, pd.ev, 0);
      for (auto& a : fin) {
        uint32_t* dst = a.rq.host_out ? a.rq.host_out : s->h_scratch;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dst, s->state + a.base, sizeof(uint32_t) * (size_t)a.n, cudaMemcpyDeviceToHost,
                              s->copy_stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->copy_stream);
      pd.fin = std::move(fin);
      s->pending.push_back(std::move(pd));
    }
  }
  const double t_done = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (read_back) {
      s->epochs += 1;
      s->rounds_total += rounds;
    }
    s->busy_s += t_done - t0;
    if (e != cudaSuccess) {
      s->fatal = IRGL_ERR_CUDA;
      s->stop = true;
      s->cv_done.notify_all();
    }
  }
  return true;
}

void server_loop(irgl_server* s) {
  DeviceGuard guard(s->ctx->device);
  for (;;) {
    Request solo;
    bool have_solo = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      if (s->queue.empty() && s->active.empty() && s->solo_q.empty() && s->pending.empty() && !s->rec[0].live &&
          !s->rec[1].live)
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
      if (s->stop) break;
    }
    server_step(s);  // one epoch of the batched queries, if any
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->fatal != IRGL_OK) break;
      if (!s->solo_q.empty()) {
        solo = s->solo_q.front();
        s->solo_q.pop_front();
        have_solo = true;
      }
    }
    if (have_solo) solo_step(s, solo);  // then one large query alone
  }
}

}  // namespace

extern "C" {

irgl_status irgl_server_create(irgl_ctx* ctx, const irgl_server_config* cfg, irgl_server** out) {
  if (!ctx || !cfg || !out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots == 0 || cfg->max_slots > static_cast<uint32_t>(kMaxBatchQueries))
    return fail(IRGL_ERR_INVALID_ARG, "max_slots must be in 1..%d", kMaxBatchQueries);
  if (cfg->epoch_rounds == 0) return fail(IRGL_ERR_INVALID_ARG, "epoch_rounds must be > 0");
  DeviceGuard guard(ctx->device);
  irgl_tuning t;
  irgl_status st = resolve_tuning(&cfg->tuning, &t);
  if (st != IRGL_OK) return st;
  irgl_server* s = new (std::nothrow) irgl_server();
  if (!s) return fail(IRGL_ERR_OOM, "server allocation");
  s->ctx = ctx;
  s->cfg = *cfg;
  s->t = t;
  uint64_t bytes = cfg->arena_bytes;
  if (bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    bytes = static_cast<uint64_t>(fr * 0.4);
  }
  const bool packed = !(t.flags & IRGL_TUNE_NO_PACKED);
  // near-far for SSSP queries (packed words only): two far lists and a far stamp per vertex
  const bool nf = packed && t.delta != 0;
  s->sub_rounds = packed ? (t.flags >> 8) & 15u : 0u;
  s->id_step = s->sub_rounds + 1u;
  s->arena_n = std::min<uint64_t>(bytes / (nf ? 32 : (packed ? 20 : 16)), 0xFFFFFFF0ull);
  const uint32_t S = cfg->max_slots;
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaMallocHost(&s->h_edge_ring, sizeof(unsigned long long) * irgl_server::kRing * cfg->max_slots);
  for (uint32_t i = 0; i < irgl_server::kRing && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&s->ring_ev[i], cudaEventDisableTiming);
    s->ring_free.push_back(irgl_server::kRing - 1 - i);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev[1]);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->ep_ev[i]);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->st_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&s->st, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&s->st_host, 2 * sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMalloc(&s->state, sizeof(uint32_t) * s->arena_n);
  if (e == cudaSuccess) {
    if (packed) e = cudaMalloc(&s->ds, sizeof(unsigned long long) * s->arena_n);
    else e = cudaMalloc(&s->stamp, sizeof(uint32_t) * s->arena_n);
  }
  if (e == cudaSuccess) e = cudaMalloc(&s->items[0], sizeof(uint32_t) * s->arena_n);
  if (e == cudaSuccess) e = cudaMalloc(&s->items[1], sizeof(uint32_t) * s->arena_n);
  if (e == cudaSuccess) e = cudaMalloc(&s->qlast, sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->cont, 128);
  if (nf && e == cudaSuccess) e = cudaMalloc(&s->far_items[0], sizeof(uint32_t) * s->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&s->far_items[1], sizeof(uint32_t) * s->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&s->far_stamp, sizeof(uint32_t) * s->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&s->blim, sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->desc, 2 * sizeof(QDesc) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->sbases, 2 * sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->qfirst, sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->qnew, sizeof(QNew) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->srcs, sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->edge_cnt, sizeof(unsigned long long) * S);
  if (e == cudaSuccess) e = cudaMalloc(&s->fin, sizeof(FinDesc) * S);
  if (e == cudaSuccess) {
    s->big_cap = big_capacity(s->arena_n);
    e = alloc_big(s->big_cap, &s->big_e, &s->big_off);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_desc, 2 * sizeof(QDesc) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_sbases, 2 * sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_qnew, 2 * sizeof(QNew) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_srcs, 2 * sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_qlast, 2 * sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_qfirst, 2 * sizeof(uint32_t) * S);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_fin, 2 * sizeof(FinDesc) * S);
  if (e != cudaSuccess) {
    server_free(s);
    delete s;
    return cuda_fail(e, "server allocation");
  }
  DevStatus z;
  std::memset(&z, 0, sizeof(z));
  z.epoch = 1;
  *s->st_host = z;
  e = cudaMemcpyAsync(s->st, s->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && s->stamp) e = cudaMemsetAsync(s->stamp, 0, sizeof(uint32_t) * s->arena_n, s->stream);
  if (e == cudaSuccess && s->far_stamp) e = cudaMemsetAsync(s->far_stamp, 0, sizeof(uint32_t) * s->arena_n, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->cont, 0, 128, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->qlast, 0, sizeof(uint32_t) * S, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  int nb = 0;
  if (e == cudaSuccess) e = occupancy_batch(t.cta_size, &nb);
  if (e != cudaSuccess || nb <= 0) {
    server_free(s);
    delete s;
    return e != cudaSuccess ? cuda_fail(e, "server setup") : fail(IRGL_ERR_CUDA, "batched kernel cannot be resident");
  }
  if (t.blocks_per_sm && static_cast<int>(t.blocks_per_sm) < nb) nb = static_cast<int>(t.blocks_per_sm);
  s->grid = static_cast<uint32_t>(nb) * static_cast<uint32_t>(ctx->sm_count);
  if (t.max_blocks && t.max_blocks < s->grid) s->grid = t.max_blocks;
  s->grid = std::min<uint32_t>(s->grid, kMaxGrid);
  s->arena.init(s->arena_n);
  for (uint32_t i = 0; i < S; ++i) s->free_slots.push_back(S - 1 - i);
  // queries that run alone: private context on the server's stream (used by the worker only)
  if (cfg->solo_min_n == 0) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
    s->solo_min_n = static_cast<uint32_t>(std::max<int64_t>(int64_t{l2} / 16, 1));  // 8 B of state + stamp per vertex > L2 / 2
  } else {
    s->solo_min_n = cfg->solo_min_n;
  }
  if (s->solo_min_n != 0xFFFFFFFFu) {
    st = irgl_ctx_create(ctx->device, s->stream, &s->solo_ctx);
    if (st != IRGL_OK) {
      server_free(s);
      delete s;
      return st;
    }
  }
  s->worker = std::thread(server_loop, s);
  *out = s;
  return IRGL_OK;
}

irgl_status irgl_server_submit(irgl_server* s, irgl_graph* g, irgl_kernel k, uint32_t src, uint32_t* host_out,
                               uint64_t* ticket) {
  if (!s || !g || !ticket) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (k != IRGL_BFS && k != IRGL_SSSP) return fail(IRGL_ERR_UNSUPPORTED, "the server runs BFS and SSSP queries");
  irgl_status st = check_kernel_graph(k, g);
  if (st != IRGL_OK) return st;
  if (src >= g->n) return fail(IRGL_ERR_INVALID_ARG, "source %u out of range", src);
  if (g->ctx != s->ctx) return fail(IRGL_ERR_INVALID_ARG, "graph belongs to another context");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != IRGL_OK) return fail(s->fatal, "server stopped after a device error");
  const bool solo = g->n >= s->solo_min_n && s->solo_ctx != nullptr;
  if (!solo && static_cast<uint64_t>(g->n) > s->arena_n) {
    s->rejected += 1;
    return fail(IRGL_ERR_ADMISSION, "query needs %u arena entries, the arena holds %llu", g->n,
                (unsigned long long)s->arena_n);
  }
  Request rq;
  rq.ticket = s->next_ticket++;
  rq.g = g;
  rq.op = static_cast<uint32_t>(k);
  rq.src = src;
  rq.host_out = host_out;
  rq.t_submit = now_s();
  if (solo) s->solo_q.push_back(rq);
  else s->queue.push_back(rq);
  s->submitted += 1;
  *ticket = rq.ticket;
  s->cv.notify_one();
  return IRGL_OK;
}

irgl_status irgl_server_poll(irgl_server* s, uint64_t ticket, irgl_query_info* info) {
  if (!s) return fail(IRGL_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return s->fatal != IRGL_OK ? fail(s->fatal, "server stopped") : IRGL_ERR_NOT_READY;
  if (info) {
    info->status = it->second.status;
    info->rounds = it->second.rounds;
    info->latency_s = it->second.t_done - it->second.t_submit;
    info->t_submit_s = it->second.t_submit;
    info->t_done_s = it->second.t_done;
    info->edges = it->second.edges;
  }
  return IRGL_OK;
}

irgl_status irgl_server_drain(irgl_server* s, uint32_t timeout_ms) {
  if (!s) return fail(IRGL_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (s->completed + s->rejected < s->submitted && s->fatal == IRGL_OK) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return fail(IRGL_ERR_NOT_READY, "drain timed out");
  }
  if (s->fatal != IRGL_OK) return fail(s->fatal, "server stopped after a device error");
  return IRGL_OK;
}

irgl_status irgl_server_stats(irgl_server* s, irgl_server_counters* out) {
  if (!s || !out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->epochs = s->epochs;
  out->rounds = s->rounds_total;
  out->edges = s->edges_total;
  out->busy_s = s->busy_s;
  out->kernel_s = s->kernel_s;
  out->active = static_cast<uint32_t>(s->active.size());
  out->queued = static_cast<uint32_t>(s->queue.size() + s->solo_q.size());
  out->solo = s->solo_done;
  out->arena_entries = s->arena_n;
  out->grid = s->grid;
  out->cta_size = s->t.cta_size;
  return IRGL_OK;
}

irgl_status irgl_server_destroy(irgl_server* s) {
  if (!s) return IRGL_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  DeviceGuard guard(s->ctx->device);
  cudaStreamSynchronize(s->stream);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  server_free(s);
  delete s;
  return IRGL_OK;
}

}  // extern "C"
