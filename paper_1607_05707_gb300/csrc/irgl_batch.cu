// Batching: many independent queries (instances) in one persistent cooperative
// launch, captured once in a CUDA graph and replayed.
//
// Waves (optional; the autotuner measures them): the queries are split, in add
// order, into consecutive groups whose packed state fits in a byte budget; a
// run admits and iterates one group after another, each one persistent launch,
// so the random state accesses of the active group stay in L2 (256 R-MAT
// instances of 16.4 M vertices in all: 8.4 ms as one wave, 6.6 ms as two with
// half the L2 each). High-diameter queries lose: their rounds repeat per wave.
//
// Layout: instance q owns arena[base_q, base_q + n_q) of the packed arena (one
// 64-bit word per vertex: value and the id of the round that last lowered it;
// with IRGL_TUNE_NO_PACKED a state and a stamp arena instead) and the same
// range of the u32 result arena, filled from the packed words after each run;
// its worklist items are arena indices on the
// shared double-buffered worklist; its termination flag is qlast[q], the round
// of its last push. Bases are assigned in insertion order, so the descriptor
// table is sorted by base and an item maps back to its instance by binary
// search (the per-instance offset table).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

using namespace irgl;

namespace {

struct BQuery {
  irgl_graph* g = nullptr;
  uint32_t op = 0;
  std::vector<uint32_t> srcs;
  uint32_t base = 0;
  uint32_t n = 0;
  uint32_t rounds = 0;
};

struct Wave {
  uint32_t q0, q1;  // query ids [q0, q1)
  uint64_t n;       // vertices
};

}  // namespace

struct irgl_batch {
  irgl_ctx* ctx = nullptr;
  uint32_t max_q = 0;
  std::vector<BQuery> qs;
  bool prepared = false;
  uint64_t arena_n = 0;
  uint64_t wl_cap = 0;  // entries of each worklist
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevStatus* st = nullptr;
  DevStatus* st_host = nullptr;
  uint32_t* state = nullptr;
  uint32_t* stamp = nullptr;          // two-array form only (IRGL_TUNE_NO_PACKED)
  unsigned long long* ds = nullptr;   // packed (value, round id) arena
  uint32_t* items[2] = {nullptr, nullptr};
  uint32_t* qlast = nullptr;
  uint32_t* qlast_host = nullptr;
  uint32_t* qfirst = nullptr;         // per query: the round id its wave started at
  uint32_t* far_items[2] = {nullptr, nullptr};  // near-far (tuning delta != 0): far lists
  uint32_t* far_stamp = nullptr;      //   arena: round id of the far list a vertex was last put on
  uint32_t* blim = nullptr;           //   per query: its limit
  uint32_t* dmin = nullptr;           // deferred expansion: 3 x kMaxBatchQueries smallest pushed distances
  uint32_t* qfirst_host = nullptr;
  uint64_t wave_bytes = 0;            // 0: one wave
  std::vector<Wave> waves;
  std::vector<AdmitParams> aps;       // one admission per wave
  uint32_t epoch_prev = 1;            // device epoch after the previous run
  uint32_t* cont = nullptr;
  uint32_t* srcs = nullptr;
  uint32_t* sbases = nullptr;
  QDesc* desc = nullptr;
  QNew* qnew = nullptr;
  uint4* big_e = nullptr;
  unsigned long long* big_off = nullptr;
  uint32_t big_cap = 0;
  irgl_tuning t{};
  uint32_t grid = 0;
  uint32_t id_step = 1;  // round ids per round: 1 + CTA-local sub-rounds
  BParams bp{};
  uint32_t admit_grid = 0;
  bool graph_ok = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace irgl {

// Sec. 4.4: the control kernel's block size must lie in the intersection of
// the block sizes every kernel of the outlined Pipe accepts; empty means no
// outlining; with several candidates the highest is taken, unless the caller's
// preferred size is in the set.
irgl_status control_cta(const uint32_t* masks, uint32_t count, uint32_t preferred, uint32_t* out) {
  uint32_t inter = 0xFu;  // bit i <=> CTA size 128 << i
  for (uint32_t i = 0; i < count; ++i) inter &= masks[i];
  if (inter == 0) return fail(IRGL_ERR_UNSUPPORTED, "no block size satisfies every kernel: outlining impossible");
  if (preferred) {
    for (uint32_t b = 0; b < 4; ++b)
      if ((128u << b) == preferred && (inter >> b & 1u)) {
        *out = preferred;
        return IRGL_OK;
      }
  }
  for (int b = 3; b >= 0; --b)
    if (inter >> b & 1u) {
      *out = 128u << b;
      return IRGL_OK;
    }
  return fail(IRGL_ERR_UNSUPPORTED, "empty block-size set");
}

// Block sizes each kernel instance is compiled for (FixedBlock templates).
uint32_t kernel_cta_mask(uint32_t op) {
  (void)op;
  return 0xFu;  // 128, 256, 512, 1024 for BFS, SSSP and CC alike
}

}  // namespace irgl

namespace {

void batch_free_device(irgl_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaFree(b->state);
  cudaFree(b->stamp);
  cudaFree(b->ds);
  cudaFree(b->items[0]);
  cudaFree(b->items[1]);
  cudaFree(b->qlast);
  cudaFree(b->qfirst);
  cudaFree(b->far_items[0]);
  cudaFree(b->far_items[1]);
  cudaFree(b->far_stamp);
  cudaFree(b->blim);
  b->far_items[0] = b->far_items[1] = b->far_stamp = b->blim = nullptr;
  cudaFree(b->cont);
  cudaFree(b->srcs);
  cudaFree(b->sbases);
  cudaFree(b->desc);
  cudaFree(b->qnew);
  cudaFree(b->big_e);
  cudaFree(b->big_off);
  b->big_e = nullptr;
  b->big_off = nullptr;
  b->big_cap = 0;
  if (b->qlast_host) cudaFreeHost(b->qlast_host);
  if (b->qfirst_host) cudaFreeHost(b->qfirst_host);
  b->qfirst = b->qfirst_host = nullptr;
  b->waves.clear();
  b->aps.clear();
  b->state = b->stamp = b->items[0] = b->items[1] = b->qlast = b->cont = b->srcs = b->sbases = nullptr;
  b->ds = nullptr;
  b->qlast_host = nullptr;
  b->desc = nullptr;
  b->qnew = nullptr;
  b->prepared = false;
}

void batch_reset_status(irgl_batch* b) {
  DevStatus z;
  std::memset(&z, 0, sizeof(z));
  z.epoch = 1;
  *b->st_host = z;
  b->epoch_prev = z.epoch;
  cudaMemcpyAsync(b->st, b->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, b->stream);
  if (b->stamp) cudaMemsetAsync(b->stamp, 0, sizeof(uint32_t) * b->arena_n, b->stream);
  if (b->far_stamp) cudaMemsetAsync(b->far_stamp, 0, sizeof(uint32_t) * b->arena_n, b->stream);
  cudaStreamSynchronize(b->stream);
}

cudaError_t enqueue(irgl_batch* b) {
  cudaError_t e = cudaSuccess;
  for (const AdmitParams& ap : b->aps) {  // one wave after another
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cont, 0, 4 * sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = launch_admit(ap, b->admit_grid, b->stream);
    if (e == cudaSuccess) e = launch_batch_iterate(b->t.cta_size, b->grid, b->bp, b->stream);
  }
  // results: the value halves of the packed words
  if (e == cudaSuccess && b->ds) e = launch_extract_values(b->ds, b->state, b->arena_n, b->admit_grid, b->stream);
  return e;
}

}  // namespace

extern "C" {

irgl_status irgl_control_cta(const uint32_t* masks, uint32_t count, uint32_t preferred, uint32_t* out) {
  if ((count && !masks) || !out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  return control_cta(masks, count, preferred, out);
}

irgl_status irgl_batch_create(irgl_ctx* ctx, uint32_t max_queries, irgl_batch** out) {
  if (!ctx || !out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (max_queries == 0 || max_queries > static_cast<uint32_t>(kMaxBatchQueries))
    return fail(IRGL_ERR_INVALID_ARG, "max_queries must be in 1..%d", kMaxBatchQueries);
  DeviceGuard guard(ctx->device);
  irgl_batch* b = new (std::nothrow) irgl_batch();
  if (!b) return fail(IRGL_ERR_OOM, "batch allocation");
  b->ctx = ctx;
  b->max_q = max_queries;
  b->stream = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (!b->stream) {  // the legacy default stream cannot be captured: use a private one
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->st, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&b->st_host, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMalloc(&b->dmin, sizeof(uint32_t) * 3 * kMaxBatchQueries);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dmin, 0, sizeof(uint32_t) * 3 * kMaxBatchQueries, b->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
  if (e != cudaSuccess) {
    irgl_batch_destroy(b);
    return cuda_fail(e, "batch setup");
  }
  batch_reset_status(b);
  *out = b;
  return IRGL_OK;
}

irgl_status irgl_batch_destroy(irgl_batch* b) {
  if (!b) return IRGL_OK;
  DeviceGuard guard(b->ctx->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free_device(b);
  cudaFree(b->st);
  cudaFree(b->dmin);
  if (b->st_host) cudaFreeHost(b->st_host);
  if (b->ev[0]) cudaEventDestroy(b->ev[0]);
  if (b->ev[1]) cudaEventDestroy(b->ev[1]);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return IRGL_OK;
}

irgl_status irgl_batch_add(irgl_batch* b, irgl_graph* g, irgl_kernel k, const uint32_t* srcs_host, uint32_t nsrc,
                           uint32_t* query_id) {
  if (!b || !g || (nsrc && !srcs_host)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (b->prepared) return fail(IRGL_ERR_INVALID_ARG, "batch already prepared");
  if (b->qs.size() >= b->max_q) return fail(IRGL_ERR_INVALID_ARG, "batch is full (%u queries)", b->max_q);
  if (g->ctx != b->ctx) return fail(IRGL_ERR_INVALID_ARG, "graph belongs to another context");
  if (k == IRGL_CC_JUMP) return fail(IRGL_ERR_UNSUPPORTED, "batches host BFS, SSSP and CC queries");
  irgl_status s = check_kernel_graph(k, g);
  if (s != IRGL_OK) return s;
  if (k != IRGL_CC && nsrc == 0) return fail(IRGL_ERR_INVALID_ARG, "BFS/SSSP need at least one source");
  for (uint32_t i = 0; i < nsrc; ++i)
    if (srcs_host[i] >= g->n) return fail(IRGL_ERR_INVALID_ARG, "source %u out of range", srcs_host[i]);
  BQuery q;
  q.g = g;
  q.op = static_cast<uint32_t>(k);
  q.n = g->n;
  if (k != IRGL_CC) q.srcs.assign(srcs_host, srcs_host + nsrc);
  if (query_id) *query_id = static_cast<uint32_t>(b->qs.size());
  b->qs.push_back(std::move(q));
  return IRGL_OK;
}

irgl_status irgl_batch_prepare(irgl_batch* b, const irgl_tuning* tin, int use_cuda_graph) {
  if (!b) return fail(IRGL_ERR_INVALID_ARG, "batch is NULL");
  if (b->qs.empty()) return fail(IRGL_ERR_INVALID_ARG, "batch has no queries");
  DeviceGuard guard(b->ctx->device);
  irgl_ctx* ctx = b->ctx;
  irgl_tuning t;
  irgl_status s = resolve_tuning(tin, &t);
  if (s != IRGL_OK) return s;
  // T_control: one CTA size valid for every kernel hosted by the launch; the
  // preference is the caller's size or else the default one (128 measured
  // 12 % faster than the set's highest, 1024, on the 256-instance batch)
  std::vector<uint32_t> masks;
  for (auto& q : b->qs) masks.push_back(kernel_cta_mask(q.op));
  uint32_t cta = 0;
  s = control_cta(masks.data(), static_cast<uint32_t>(masks.size()), t.cta_size, &cta);
  if (s != IRGL_OK) return s;
  t.cta_size = cta;
  if (b->prepared) {
    cudaStreamSynchronize(b->stream);
    batch_free_device(b);
  }
  // arena
  uint64_t total = 0, nsrc = 0;
  for (auto& q : b->qs) {
    q.base = static_cast<uint32_t>(total);
    total += q.n;
    nsrc += q.srcs.size();
    if (total >= 0xFFFFFFFFull) return fail(IRGL_ERR_INVALID_ARG, "batch arena exceeds 2^32 - 1 entries");
  }
  b->arena_n = std::max<uint64_t>(total, 1);
  const uint32_t Q = static_cast<uint32_t>(b->qs.size());
  // waves: consecutive queries while their packed state fits the budget
  const uint64_t budget = b->wave_bytes == 0 ? ~uint64_t{0} : b->wave_bytes;  // 0: one wave
  b->waves.clear();
  for (uint32_t i = 0; i < Q; ++i) {
    const uint64_t bytes = 8ull * b->qs[i].n;
    if (b->waves.empty() || 8ull * b->waves.back().n + bytes > budget) b->waves.push_back(Wave{i, i, 0});
    b->waves.back().q1 = i + 1;
    b->waves.back().n += b->qs[i].n;
  }
  std::vector<QDesc> desc(Q);
  std::vector<QNew> qn(Q);
  std::vector<uint32_t> bases(Q), flat;
  flat.reserve(nsrc);
  for (const Wave& wv : b->waves) {
    for (uint32_t i = wv.q0; i < wv.q1; ++i) {
      const BQuery& q = b->qs[i];
      desc[i] = QDesc{q.g->row_ptr, q.g->col, q.g->w, q.n, q.op, q.base, i};
      bases[i] = q.base;
      // pre: exclusive prefix of n within the wave (the admission kernels' index space)
      qn[i] = QNew{q.base, q.n, q.op, i, static_cast<uint32_t>(flat.size()), static_cast<uint32_t>(q.srcs.size()),
                   q.base - b->qs[wv.q0].base, 0};
      flat.insert(flat.end(), q.srcs.begin(), q.srcs.end());
    }
  }
  // packed (value, round id) words unless the two-array form is asked for; the
  // u32 state arena then holds the results, extracted after each run
  const bool packed = !(t.flags & IRGL_TUNE_NO_PACKED);
  cudaError_t e = cudaMalloc(&b->state, sizeof(uint32_t) * b->arena_n);
  if (e == cudaSuccess) {
    if (packed) e = cudaMalloc(&b->ds, sizeof(unsigned long long) * b->arena_n);
    else e = cudaMalloc(&b->stamp, sizeof(uint32_t) * b->arena_n);
  }
  // worklists: one entry per arena vertex; with CTA-local sub-rounds a vertex
  // lowered again in a later sub-round of the same round can be on the next
  // round's worklist twice, so they get twice the room (a round that still
  // overflows reports IRGL_ERR_WL_OVERFLOW)
  const bool sub = packed && ((t.flags >> 8) & 15u) != 0;
  b->wl_cap = std::min<uint64_t>(b->arena_n * (sub ? 2u : 1u), 0xFFFFFFF0ull);
  if (e == cudaSuccess) e = cudaMalloc(&b->items[0], sizeof(uint32_t) * b->wl_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->items[1], sizeof(uint32_t) * b->wl_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->qlast, sizeof(uint32_t) * Q);
  if (e == cudaSuccess) e = cudaMallocHost(&b->qlast_host, sizeof(uint32_t) * Q);
  if (e == cudaSuccess) e = cudaMalloc(&b->qfirst, sizeof(uint32_t) * Q);
  // near-far for the SSSP queries (packed words only): two far lists, a far stamp per vertex
  const bool nf = t.delta != 0 && packed;
  if (nf && e == cudaSuccess) e = cudaMalloc(&b->far_items[0], sizeof(uint32_t) * b->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&b->far_items[1], sizeof(uint32_t) * b->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&b->far_stamp, sizeof(uint32_t) * b->arena_n);
  if (nf && e == cudaSuccess) e = cudaMalloc(&b->blim, sizeof(uint32_t) * Q);
  if (e == cudaSuccess) e = cudaMallocHost(&b->qfirst_host, sizeof(uint32_t) * Q);
  if (e == cudaSuccess) e = cudaMalloc(&b->cont, 128);
  if (e == cudaSuccess) e = cudaMalloc(&b->srcs, sizeof(uint32_t) * std::max<size_t>(flat.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->sbases, sizeof(uint32_t) * Q);
  if (e == cudaSuccess) e = cudaMalloc(&b->desc, sizeof(QDesc) * Q);
  if (e == cudaSuccess) e = cudaMalloc(&b->qnew, sizeof(QNew) * Q);
  if (e == cudaSuccess) {
    b->big_cap = big_capacity(b->arena_n);
    e = alloc_big(b->big_cap, &b->big_e, &b->big_off);
  }
  if (e != cudaSuccess) {
    batch_free_device(b);
    return cuda_fail(e, "batch arena allocation");
  }
  if (b->stamp) e = cudaMemsetAsync(b->stamp, 0, sizeof(uint32_t) * b->arena_n, b->stream);
  if (e == cudaSuccess && b->far_stamp) e = cudaMemsetAsync(b->far_stamp, 0, sizeof(uint32_t) * b->arena_n, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->cont, 0, 128, b->stream);
  if (e == cudaSuccess && !flat.empty())
    e = cudaMemcpyAsync(b->srcs, flat.data(), sizeof(uint32_t) * flat.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->sbases, bases.data(), sizeof(uint32_t) * Q, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->desc, desc.data(), sizeof(QDesc) * Q, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->qnew, qn.data(), sizeof(QNew) * Q, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    batch_free_device(b);
    return cuda_fail(e, "batch upload");
  }
  // persistent grid
  int nb = 0;
  e = occupancy_batch(t.cta_size, &nb);
  if (e != cudaSuccess || nb <= 0) {
    batch_free_device(b);
    return fail(IRGL_ERR_CUDA, "batched kernel cannot be made resident");
  }
  if (t.blocks_per_sm && static_cast<int>(t.blocks_per_sm) < nb) nb = static_cast<int>(t.blocks_per_sm);
  b->grid = static_cast<uint32_t>(nb) * static_cast<uint32_t>(ctx->sm_count);
  if (t.max_blocks && t.max_blocks < b->grid) b->grid = t.max_blocks;
  b->grid = std::min<uint32_t>(b->grid, kMaxGrid);
  b->t = t;
  b->bp = BParams{};
  b->bp.desc = b->desc;
  b->bp.sbases = b->sbases;
  b->bp.nq = Q;
  b->bp.state = b->state;
  b->bp.stamp = b->stamp;
  b->bp.ds = b->ds;
  b->bp.qlast = b->qlast;
  b->bp.items[0] = b->items[0];
  b->bp.items[1] = b->items[1];
  b->bp.cap = static_cast<uint32_t>(b->wl_cap);
  b->bp.cont = b->cont;
  b->bp.st = b->st;
  b->bp.tn = Tune{t.warp_thresh, t.cta_thresh, t.chunk, thread_bin(t)};
  b->bp.max_rounds = 0xFFFFFFFFu;
  b->bp.rounds_cap_is_error = 1;
  b->bp.timeout_ns = ctx->dbg_timeout_us ? ctx->dbg_timeout_us * 1000ull : 2000000000ull;
  b->bp.time_limit_ns = run_time_limit_ns(ctx);
  b->bp.spread = ctx->dbg_no_spread ? 0u : 1u;
  b->bp.trace = ctx->trace;
  b->bp.trace_cap = ctx->trace_cap;
  b->bp.big = (t.flags & IRGL_TUNE_NO_SPLIT) ? BigList{nullptr, nullptr, 0} : BigList{b->big_e, b->big_off, b->big_cap};
  b->bp.delta = nf ? t.delta : 0u;
  b->bp.blim = b->blim;
  b->bp.far_items[0] = b->far_items[0];
  b->bp.far_items[1] = b->far_items[1];
  b->bp.far_cap = nf ? static_cast<uint32_t>(b->arena_n) : 0u;
  b->bp.far_stamp = b->far_stamp;
  b->bp.local_rounds = b->ds ? (t.flags >> 8) & 15u : 0u;
  b->id_step = b->bp.local_rounds + 1u;
  if (b->ds && !nf && b->bp.local_rounds == 0 && !(t.flags & IRGL_TUNE_NO_DEFER)) {
    // deferred expansion of long lists for the SSSP queries
    b->bp.dmin = b->dmin;
    b->bp.defer_deg = t.defer_deg;
    b->bp.defer_delta = t.defer_delta;
  }
  b->aps.clear();
  for (const Wave& wv : b->waves) {
    AdmitParams ap{};
    ap.qn = b->qnew + wv.q0;
    ap.nnew = wv.q1 - wv.q0;
    ap.total = static_cast<uint32_t>(wv.n);
    ap.srcs = b->srcs;
    ap.state = b->state;
    ap.ds = b->ds;
    ap.qlast = b->qlast;
    ap.qfirst = b->qfirst;
    ap.blim = b->blim;
    ap.delta = b->bp.delta;
    ap.items[0] = b->items[0];
    ap.items[1] = b->items[1];
    ap.cap = static_cast<uint32_t>(b->wl_cap);
    ap.cont = b->cont;
    ap.st = b->st;
    ap.id_step = b->id_step;
    b->aps.push_back(ap);
  }
  b->admit_grid = static_cast<uint32_t>(ctx->sm_count) * 4;
  b->graph_ok = false;
  if (use_cuda_graph) {
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(b);
      cudaGraph_t gr = nullptr;
      e = cudaStreamEndCapture(b->stream, &gr);
      if (e2 == cudaSuccess && e == cudaSuccess && gr) {
        e = cudaGraphInstantiate(&b->exec, gr, 0);
        if (e == cudaSuccess) {
          b->graph = gr;
          b->graph_ok = true;
        } else {
          cudaGraphDestroy(gr);
        }
      } else if (gr) {
        cudaGraphDestroy(gr);
      }
    }
    cudaGetLastError();  // a failed capture falls back to direct launches
  }
  b->prepared = true;
  return IRGL_OK;
}

irgl_status irgl_batch_set_wave_bytes(irgl_batch* b, uint64_t bytes) {
  if (!b) return fail(IRGL_ERR_INVALID_ARG, "batch is NULL");
  b->wave_bytes = bytes;
  return IRGL_OK;
}

irgl_status irgl_batch_waves(irgl_batch* b, uint32_t* waves) {
  if (!b || !waves) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  *waves = static_cast<uint32_t>(b->waves.size());
  return IRGL_OK;
}

irgl_status irgl_batch_launch(irgl_batch* b) {
  if (!b || !b->prepared) return fail(IRGL_ERR_INVALID_ARG, "batch not prepared");
  DeviceGuard guard(b->ctx->device);
  cudaError_t e = cudaEventRecord(b->ev[0], b->stream);
  if (e == cudaSuccess) e = b->graph_ok ? cudaGraphLaunch(b->exec, b->stream) : enqueue(b);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev[1], b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return IRGL_OK;
}

irgl_status irgl_batch_sync(irgl_batch* b, irgl_stats* stats) {
  if (!b || !b->prepared) return fail(IRGL_ERR_INVALID_ARG, "batch not prepared");
  DeviceGuard guard(b->ctx->device);
  const uint32_t Q = static_cast<uint32_t>(b->qs.size());
  cudaError_t e = cudaMemcpyAsync(b->st_host, b->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->qlast_host, b->qlast, sizeof(uint32_t) * Q, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->qfirst_host, b->qfirst, sizeof(uint32_t) * Q, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch sync");
  const DevStatus st = *b->st_host;
  b->ctx->st_host->rounds = st.rounds;  // lets irgl_trace_read size a batch trace (the last wave's)
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->rounds = (st.epoch - b->epoch_prev) / b->id_step;  // every wave's rounds
    stats->grid = b->grid;
    stats->cta_size = b->t.cta_size;
    // per wave: fill, sources, iterate; then the result extraction
    stats->launches = 3u * static_cast<uint32_t>(b->waves.size()) + (b->ds ? 1u : 0u);
    stats->edges_scanned = st.edges;
    stats->last_out = st.last_out;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) stats->device_ms = ms;
  }
  if (st.err != DERR_NONE) {
    irgl_status s = IRGL_ERR_CUDA;
    switch (st.err) {
      case DERR_WL_OVERFLOW: s = fail(IRGL_ERR_WL_OVERFLOW, "a push found the batch worklist full"); break;
      case DERR_BARRIER_TIMEOUT: s = fail(IRGL_ERR_BARRIER_TIMEOUT, "grid barrier wait exceeded its time limit"); break;
      case DERR_MAX_ROUNDS: s = fail(IRGL_ERR_MAX_ROUNDS, "batch reached max_rounds with work left"); break;
      case DERR_BAD_ITEM: s = fail(IRGL_ERR_INVALID_ARG, "a worklist item is not a vertex of its graph"); break;
      case DERR_TIME_LIMIT: s = fail(IRGL_ERR_TIME_LIMIT, "batched launch ran past its time limit"); break;
      default: s = fail(IRGL_ERR_CUDA, "unknown device error %u", st.err); break;
    }
    batch_reset_status(b);
    return s;
  }
  // per-instance rounds from the termination flags and the round its wave began at
  for (uint32_t i = 0; i < Q; ++i)
    b->qs[i].rounds = static_cast<uint32_t>(static_cast<int32_t>(b->qlast_host[i] - b->qfirst_host[i]) /
                                            static_cast<int32_t>(b->id_step) + 2);
  b->epoch_prev = st.epoch;
  cudaMemsetAsync(&b->st->edges, 0, sizeof(unsigned long long), b->stream);
  if (st.epoch > 0xF0000000u) batch_reset_status(b);
  return IRGL_OK;
}

irgl_status irgl_batch_run(irgl_batch* b, irgl_stats* stats) {
  irgl_status s = irgl_batch_launch(b);
  if (s != IRGL_OK) return s;
  return irgl_batch_sync(b, stats);
}

irgl_status irgl_batch_autotune(irgl_batch* b, uint32_t reps, irgl_tuning* best, float* best_ms) {
  if (!b || !b->prepared || !best) return fail(IRGL_ERR_INVALID_ARG, "NULL argument or batch not prepared");
  const int use_graph = b->graph_ok ? 1 : 0;
  reps = std::max<uint32_t>(reps, 1);
  auto measure = [&](const irgl_tuning& t) -> float {
    if (irgl_batch_prepare(b, &t, use_graph) != IRGL_OK) return -1.f;
    std::vector<float> ms;
    for (uint32_t r = 0; r <= reps; ++r) {
      irgl_stats st;
      if (irgl_batch_run(b, &st) != IRGL_OK) return -1.f;
      if (r) ms.push_back(st.device_ms);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };
  bool has_sssp = false;  // near-far delta is searched when the batch holds SSSP queries
  for (const BQuery& q : b->qs) has_sssp |= q.op == IRGL_SSSP;
  irgl_status s = tune_descend(measure, best, best_ms, has_sssp, true, false, 0, has_sssp);
  if (s != IRGL_OK) return s;
  // then the wave budget: a quarter, half (the default) and all of the L2, and one wave
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->ctx->device);
  const uint64_t keep = b->wave_bytes;
  uint64_t best_w = keep;
  float w_ms = best_ms ? *best_ms : measure(*best);
  const uint64_t l2b = static_cast<uint64_t>(l2);
  const uint64_t budgets[4] = {l2b / 4, l2b / 2, l2b, ~uint64_t{0}};
  for (uint64_t w : budgets) {
    b->wave_bytes = w;
    const float ms = measure(*best);
    if (ms >= 0 && ms < w_ms * 0.98f) {
      w_ms = ms;
      best_w = w;
    }
  }
  b->wave_bytes = best_w;
  if (best_ms) *best_ms = w_ms;
  return irgl_batch_prepare(b, best, use_graph);
}

irgl_status irgl_batch_info(irgl_batch* b, uint32_t* nqueries, uint32_t* grid, uint32_t* cta_size,
                            int* graph_captured, uint64_t* arena_entries) {
  if (!b) return fail(IRGL_ERR_INVALID_ARG, "batch is NULL");
  if (nqueries) *nqueries = static_cast<uint32_t>(b->qs.size());
  if (grid) *grid = b->grid;
  if (cta_size) *cta_size = b->t.cta_size;
  if (graph_captured) *graph_captured = b->graph_ok ? 1 : 0;
  if (arena_entries) *arena_entries = b->arena_n;
  return IRGL_OK;
}

irgl_status irgl_batch_result(irgl_batch* b, uint32_t query_id, uint32_t** state_dev, uint32_t* n, uint32_t* rounds) {
  if (!b || !b->prepared) return fail(IRGL_ERR_INVALID_ARG, "batch not prepared");
  if (query_id >= b->qs.size()) return fail(IRGL_ERR_INVALID_ARG, "query id out of range");
  const BQuery& q = b->qs[query_id];
  if (state_dev) *state_dev = b->state + q.base;
  if (n) *n = q.n;
  if (rounds) *rounds = q.rounds;
  return IRGL_OK;
}

irgl_status irgl_batch_copy_result(irgl_batch* b, uint32_t query_id, uint32_t* host_out) {
  if (!b || !b->prepared || !host_out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument or batch not prepared");
  if (query_id >= b->qs.size()) return fail(IRGL_ERR_INVALID_ARG, "query id out of range");
  DeviceGuard guard(b->ctx->device);
  const BQuery& q = b->qs[query_id];
  cudaError_t e = cudaMemcpyAsync(host_out, b->state + q.base, sizeof(uint32_t) * (size_t)q.n,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch result copy");
  return IRGL_OK;
}

irgl_status irgl_batch_copy_results(irgl_batch* b, uint32_t* host_out) {
  if (!b || !b->prepared || !host_out) return fail(IRGL_ERR_INVALID_ARG, "NULL argument or batch not prepared");
  DeviceGuard guard(b->ctx->device);
  uint64_t total = 0;
  for (const BQuery& q : b->qs) total += q.n;  // bases are the running sums of n
  cudaError_t e = cudaMemcpyAsync(host_out, b->state, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch results copy");
  return IRGL_OK;
}

}  // extern "C"
