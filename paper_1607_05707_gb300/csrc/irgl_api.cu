// C-ABI of libirgl.so: contexts, CSR graphs, worklists, Invoke and Iterate.
//
// Host runtime around the sm_103a kernels. Every entry point returns a status
// code; CUDA errors, bad arguments and device-reported errors (worklist
// overflow, barrier timeout, max rounds) are turned into irgl_status values
// with a thread-local message. Nothing here computes a traversal on the CPU.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

using namespace irgl;

namespace irgl {

thread_local std::string g_last_error;

irgl_status fail(irgl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

irgl_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(IRGL_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(IRGL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

DeviceGuard::DeviceGuard(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
  dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
  if (prev_ != dev_) cudaSetDevice(prev_);
}

unsigned long long run_time_limit_ns(const irgl_ctx* ctx) {
  return ctx->dbg_time_limit_ms ? ctx->dbg_time_limit_ms * 1000000ull : kRunTimeLimitNs;
}

uint32_t thread_bin(const irgl_tuning& t) { return (t.flags & IRGL_TUNE_THREAD_BIN) ? kThreadBin : 0u; }

irgl_tuning default_tuning() {
  irgl_tuning t;
  t.cta_size = 128;
  t.warp_thresh = 32;
  t.cta_thresh = 32;
  t.chunk = 1;
  t.blocks_per_sm = 0;
  t.max_blocks = 0;
  t.flags = 0;
  t.delta = 0;
  t.defer_deg = 128;
  t.defer_delta = 2;
  return t;
}

irgl_status resolve_tuning(const irgl_tuning* in, irgl_tuning* out) {
  irgl_tuning d = default_tuning();
  if (in) {
    if (in->cta_size) d.cta_size = in->cta_size;
    if (in->warp_thresh) d.warp_thresh = in->warp_thresh;
    if (in->cta_thresh) d.cta_thresh = in->cta_thresh;
    if (in->chunk) d.chunk = in->chunk;
    d.blocks_per_sm = in->blocks_per_sm;
    d.max_blocks = in->max_blocks;
    d.flags = in->flags;
    d.delta = in->delta;
    if (in->defer_deg) d.defer_deg = in->defer_deg;
    if (in->defer_delta) d.defer_delta = in->defer_delta;
  }
  if (!valid_cta(d.cta_size)) return fail(IRGL_ERR_INVALID_ARG, "cta_size must be 128, 256, 512 or 1024");
  if (d.chunk > 64) return fail(IRGL_ERR_INVALID_ARG, "chunk must be <= 64");
  if (d.warp_thresh < 1) d.warp_thresh = 1;
  if (d.cta_thresh < d.warp_thresh) d.cta_thresh = d.warp_thresh;
  *out = d;
  return IRGL_OK;
}

irgl_status status_from_device(const DevStatus& s) {
  switch (s.err) {
    case DERR_NONE: return IRGL_OK;
    case DERR_WL_OVERFLOW: return fail(IRGL_ERR_WL_OVERFLOW, "a push found the out-worklist full");
    case DERR_BARRIER_TIMEOUT:
      return fail(IRGL_ERR_BARRIER_TIMEOUT, "grid barrier wait exceeded its time limit");
    case DERR_MAX_ROUNDS: return fail(IRGL_ERR_MAX_ROUNDS, "Iterate reached max_rounds with work left");
    case DERR_BAD_ITEM: return fail(IRGL_ERR_INVALID_ARG, "a worklist item is not a vertex of the graph");
    case DERR_LOCK_TIMEOUT: return fail(IRGL_ERR_LOCK_TIMEOUT, "an Atomic section's lock wait exceeded its time limit");
    case DERR_MSF_ITERS: return fail(IRGL_ERR_CUDA, "Boruvka's algorithm did not converge");
    case DERR_TIME_LIMIT: return fail(IRGL_ERR_TIME_LIMIT, "persistent launch ran past its time limit");
  }
  return fail(IRGL_ERR_CUDA, "unknown device error %u", s.err);
}

// Copy the status block back and synchronise; clear it after a device error.
irgl_status read_status(irgl_ctx* ctx, DevStatus* out) {
  cudaError_t e = cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status readback");
  if (out) *out = *ctx->st_host;
  if (ctx->st_host->err != DERR_NONE) {
    const irgl_status s = status_from_device(*ctx->st_host);
    reset_status(ctx);
    return s;
  }
  if (ctx->st_host->epoch > 0xF0000000u) {
    // stamp epoch close to wrapping: clear the stamps and restart at 1
    if (ctx->ws_stamp) cudaMemsetAsync(ctx->ws_stamp, 0, sizeof(uint32_t) * (size_t)ctx->ws_stamp_n, ctx->stream);
    reset_status(ctx);
  }
  return IRGL_OK;
}

void reset_status(irgl_ctx* ctx) {
  // Clear counters and errors. Stamps may hold any epoch used so far, so they
  // are cleared too and the epoch restarts at 1.
  DevStatus z;
  std::memset(&z, 0, sizeof(z));
  z.epoch = 1;
  *ctx->st_host = z;
  cudaMemcpyAsync(ctx->st, ctx->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, ctx->stream);
  if (ctx->ws_stamp) cudaMemsetAsync(ctx->ws_stamp, 0, sizeof(uint32_t) * (size_t)ctx->ws_stamp_n, ctx->stream);
  if (ctx->ws_far_stamp) cudaMemsetAsync(ctx->ws_far_stamp, 0, sizeof(uint32_t) * (size_t)ctx->ws_far_n, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
}

// Big-list entries: at most one per popped vertex of a round, capped (a full
// list sends further long lists to the warp bin, which is still correct).
uint32_t big_capacity(uint64_t n) { return static_cast<uint32_t>(std::min<uint64_t>(std::max<uint64_t>(n, 1), 1u << 22)); }

cudaError_t alloc_big(uint32_t cap, uint4** e, unsigned long long** off) {
  cudaError_t r = cudaMalloc(e, sizeof(uint4) * (size_t)cap);
  if (r == cudaSuccess) r = cudaMalloc(off, sizeof(unsigned long long) * (size_t)cap);
  return r;
}

irgl_status ensure_workspace(irgl_ctx* ctx, uint32_t n, bool need_stamp, bool need_far, bool need_vis, bool need_ds,
                             uint32_t wl_mult) {
  if (need_far && n > ctx->ws_far_n) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws_far[0]);
    cudaFree(ctx->ws_far[1]);
    cudaFree(ctx->ws_far_stamp);
    ctx->ws_far[0] = ctx->ws_far[1] = ctx->ws_far_stamp = nullptr;
    ctx->ws_far_n = 0;
    cudaError_t e = cudaMalloc(&ctx->ws_far[0], sizeof(uint32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws_far[1], sizeof(uint32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws_far_stamp, sizeof(uint32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws_far_stamp, 0, sizeof(uint32_t) * (size_t)n, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "near-far allocation");
    ctx->ws_far_n = n;
  }
  const uint32_t bcap = big_capacity(n);
  if (bcap > ctx->big_cap) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->big_e);
    cudaFree(ctx->big_off);
    ctx->big_e = nullptr;
    ctx->big_off = nullptr;
    ctx->big_cap = 0;
    cudaError_t e = alloc_big(bcap, &ctx->big_e, &ctx->big_off);
    if (e != cudaSuccess) return cuda_fail(e, "big-list allocation");
    ctx->big_cap = bcap;
  }
  const uint64_t want = std::max<uint64_t>(static_cast<uint64_t>(n) * std::max<uint32_t>(wl_mult, 1u), 1);
  uint32_t cap = ctx->dbg_cap ? ctx->dbg_cap : static_cast<uint32_t>(std::min<uint64_t>(want, 0xFFFFFFF0ull));
  if (cap > ctx->ws_cap || ctx->dbg_cap) {
    if (ctx->ws_items[0] || ctx->ws_items[1]) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws_items[0]);
      cudaFree(ctx->ws_items[1]);
      ctx->ws_items[0] = ctx->ws_items[1] = nullptr;
      ctx->ws_cap = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws_items[0], sizeof(uint32_t) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws_items[1], sizeof(uint32_t) * (size_t)cap);
    if (e != cudaSuccess) return cuda_fail(e, "worklist allocation");
    ctx->ws_cap = cap;
  }
  if (need_vis && (n + 31u) / 32u > ctx->ws_vis_words) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws_vis);
    ctx->ws_vis = nullptr;
    ctx->ws_vis_words = 0;
    const uint32_t words = (n + 31u) / 32u;
    cudaError_t e = cudaMalloc(&ctx->ws_vis, sizeof(uint32_t) * (size_t)words);
    if (e != cudaSuccess) return cuda_fail(e, "visited bitmap allocation");
    ctx->ws_vis_words = words;
  }
  if (need_ds && n > ctx->ws_ds_n) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws_ds);
    ctx->ws_ds = nullptr;
    ctx->ws_ds_n = 0;
    cudaError_t e = cudaMalloc(&ctx->ws_ds, sizeof(unsigned long long) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "packed distance allocation");
    ctx->ws_ds_n = n;
  }
  if (need_stamp && n > ctx->ws_stamp_n) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws_stamp);
    ctx->ws_stamp = nullptr;
    ctx->ws_stamp_n = 0;
    cudaError_t e = cudaMalloc(&ctx->ws_stamp, sizeof(uint32_t) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "stamp allocation");
    e = cudaMemsetAsync(ctx->ws_stamp, 0, sizeof(uint32_t) * (size_t)n, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stamp clear");
    ctx->ws_stamp_n = n;
  }
  return IRGL_OK;
}

int occupancy(irgl_ctx* ctx, int kind, uint32_t op, uint32_t cta, int red) {
  const int key = ((kind * 8 + static_cast<int>(op)) * 5 + (static_cast<int>(cta) >> 8)) * 3 + red;
  auto it = ctx->occ.find(key);
  if (it != ctx->occ.end()) return it->second;
  int nb = 0;
  cudaError_t e = kind == 0 ? occupancy_iterate(op, cta, &nb) : occupancy_round(op, cta, red, &nb);
  if (e != cudaSuccess) nb = 0;
  ctx->occ[key] = nb;
  return nb;
}

uint32_t persistent_grid(irgl_ctx* ctx, uint32_t op, const irgl_tuning& t) {
  int nb = occupancy(ctx, 0, op, t.cta_size, 0);
  if (nb <= 0) return 0;
  if (t.blocks_per_sm && static_cast<int>(t.blocks_per_sm) < nb) nb = static_cast<int>(t.blocks_per_sm);
  uint32_t grid = static_cast<uint32_t>(nb) * static_cast<uint32_t>(ctx->sm_count);
  if (t.max_blocks && t.max_blocks < grid) grid = t.max_blocks;
  grid = std::min<uint32_t>(grid, kMaxGrid);  // one barrier arrival slot per CTA
  return std::max<uint32_t>(grid, 1);
}

uint32_t op_of(irgl_kernel k) { return k == IRGL_CC_JUMP ? OP_CCJ : static_cast<uint32_t>(k); }

irgl_status check_kernel_graph(irgl_kernel k, const irgl_graph* g) {
  if (k == IRGL_SSSP) {
    if (!g->w) return fail(IRGL_ERR_INVALID_ARG, "SSSP needs edge weights");
    if (g->n > 1 && static_cast<uint64_t>(g->max_w) * (g->n - 1) >= 0xFFFFFFFFull)
      return fail(IRGL_ERR_INVALID_ARG, "max(w) * (n-1) does not fit below INF: uint32 distances could wrap");
  } else if (k == IRGL_CC || k == IRGL_CC_JUMP) {
    if (!(g->flags & IRGL_SYMMETRIC)) return fail(IRGL_ERR_NOT_SYMMETRIC, "CC needs a graph loaded with IRGL_SYMMETRIC");
  } else if (k != IRGL_BFS) {
    return fail(IRGL_ERR_INVALID_ARG, "unknown kernel %d", static_cast<int>(k));
  }
  return IRGL_OK;
}

KParams make_params(irgl_ctx* ctx, irgl_graph* g, uint32_t* state, const irgl_tuning& t) {
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.row_ptr = g->row_ptr;
  p.col = g->col;
  p.w = g->w;
  p.n = g->n;
  p.state = state;
  p.stamp = ctx->ws_stamp;
  p.items[0] = ctx->ws_items[0];
  p.items[1] = ctx->ws_items[1];
  p.cap = ctx->ws_cap;
  p.st = ctx->st;
  p.tn.warp_thresh = t.warp_thresh;
  p.tn.cta_thresh = t.cta_thresh;
  p.tn.chunk = t.chunk;
  p.tn.thread_max = thread_bin(t);
  p.max_rounds = 0xFFFFFFFFu;
  p.timeout_ns = ctx->dbg_timeout_us ? ctx->dbg_timeout_us * 1000ull : 2000000000ull;
  p.time_limit_ns = run_time_limit_ns(ctx);
  p.skip_cta = -1;
  p.init_state = 1;
  p.trace = ctx->trace;
  p.trace_cap = ctx->trace_cap;
  p.trace_ph = ctx->trace ? ctx->trace + 2 * (size_t)ctx->trace_cap : nullptr;
  p.big = (t.flags & IRGL_TUNE_NO_SPLIT) ? BigList{nullptr, nullptr, 0} : BigList{ctx->big_e, ctx->big_off, ctx->big_cap};
  if (ctx->dbg_big_cap && p.big.cap > ctx->dbg_big_cap) p.big.cap = ctx->dbg_big_cap;
  // small-frontier rounds pay for their broadcast reads by skipping the big
  // list: only graphs with lists long enough to go there use them
  p.bcast = (!(t.flags & IRGL_TUNE_NO_BCAST) && g->max_deg >= std::min(t.warp_thresh, t.cta_thresh)) ? 1u : 0u;
  p.dense_div = (t.flags & IRGL_TUNE_DENSE) ? 8u : 0u;
  p.spread = ctx->dbg_no_spread ? 0u : 1u;
  if ((t.flags & IRGL_TUNE_DIROPT) && (g->in_row_ptr || (g->flags & IRGL_SYMMETRIC))) {
    p.in_row_ptr = g->in_row_ptr ? g->in_row_ptr : g->row_ptr;
    p.in_col = g->in_row_ptr ? g->in_col : g->col;
    p.diropt = ctx->dbg_force_bottom_up ? 2u : 1u;
    p.m_total = g->m;
  }
  if (t.delta && ctx->ws_far_stamp && ctx->ws_far_n >= g->n) {
    p.far[0] = ctx->ws_far[0];
    p.far[1] = ctx->ws_far[1];
    p.far_cap = g->n;
    p.far_stamp = ctx->ws_far_stamp;
    p.delta = t.delta;
  }
  return p;
}

}  // namespace irgl

// ============================================================================ C ABI

extern "C" {

const char* irgl_last_error(void) { return g_last_error.c_str(); }

const char* irgl_status_string(irgl_status s) {
  switch (s) {
    case IRGL_OK: return "ok";
    case IRGL_ERR_INVALID_ARG: return "invalid argument";
    case IRGL_ERR_OOM: return "out of memory";
    case IRGL_ERR_WL_OVERFLOW: return "worklist overflow";
    case IRGL_ERR_BARRIER_TIMEOUT: return "grid barrier timeout";
    case IRGL_ERR_CUDA: return "CUDA error";
    case IRGL_ERR_NOT_SYMMETRIC: return "graph not symmetric";
    case IRGL_ERR_ADMISSION: return "admission rejected";
    case IRGL_ERR_MAX_ROUNDS: return "max rounds reached";
    case IRGL_ERR_NOT_READY: return "not ready";
    case IRGL_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

irgl_status irgl_ctx_create(int device, void* cuda_stream, irgl_ctx** out) {
  if (!out) return fail(IRGL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(IRGL_ERR_INVALID_ARG, "device %d out of range", device);
  DeviceGuard guard(device);
  irgl_ctx* ctx = new (std::nothrow) irgl_ctx();
  if (!ctx) return fail(IRGL_ERR_OOM, "context allocation");
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->st, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->st_host, sizeof(DevStatus));
  if (e != cudaSuccess) {
    irgl_ctx_destroy(ctx);
    return cuda_fail(e, "context setup");
  }
  reset_status(ctx);
  *out = ctx;
  return IRGL_OK;
}

irgl_status irgl_ctx_destroy(irgl_ctx* ctx) {
  if (!ctx) return IRGL_OK;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->run_wl) irgl_worklist_destroy(ctx->run_wl);
  delete ctx->run_src_wl;
  cudaFree(ctx->run_src);
  if (ctx->run_src_host) cudaFreeHost(ctx->run_src_host);
  cudaFree(ctx->ws_items[0]);
  cudaFree(ctx->ws_items[1]);
  cudaFree(ctx->ws_stamp);
  cudaFree(ctx->ws_vis);
  cudaFree(ctx->ws_bu[0]);
  cudaFree(ctx->ws_bu[1]);
  cudaFree(ctx->ws_ds);
  cudaFree(ctx->msf_buf);
  if (ctx->msf_host) cudaFreeHost(ctx->msf_host);
  cudaFree(ctx->ws_far[0]);
  cudaFree(ctx->ws_far[1]);
  cudaFree(ctx->ws_far_stamp);
  cudaFree(ctx->ws_state);
  cudaFree(ctx->trace);
  cudaFree(ctx->big_e);
  cudaFree(ctx->big_off);
  cudaFree(ctx->st);
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  delete ctx;
  return IRGL_OK;
}

irgl_status irgl_ctx_set_stream(irgl_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(IRGL_ERR_INVALID_ARG, "ctx is NULL");
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return IRGL_OK;
}

irgl_status irgl_ctx_info(irgl_ctx* ctx, uint32_t* sm_count, irgl_tuning* defaults) {
  if (!ctx) return fail(IRGL_ERR_INVALID_ARG, "ctx is NULL");
  if (sm_count) *sm_count = static_cast<uint32_t>(ctx->sm_count);
  if (defaults) *defaults = default_tuning();
  return IRGL_OK;
}

irgl_status irgl_trace_enable(irgl_ctx* ctx, uint32_t max_rounds) {
  if (!ctx) return fail(IRGL_ERR_INVALID_ARG, "ctx is NULL");
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->trace);
  ctx->trace = nullptr;
  ctx->trace_cap = 0;
  if (max_rounds == 0) return IRGL_OK;
  // round records (2 words each), then the phase records (kPhaseWords each)
  const size_t bytes = sizeof(unsigned long long) * (2 + kPhaseWords) * ((size_t)max_rounds + 1);
  cudaError_t e = cudaMalloc(&ctx->trace, bytes);
  if (e == cudaSuccess) e = cudaMemset(ctx->trace, 0, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "trace allocation");
  ctx->trace_cap = max_rounds + 1;
  return IRGL_OK;
}

irgl_status irgl_trace_read(irgl_ctx* ctx, uint64_t* t_ns, uint32_t* in_n, uint32_t* out_n, uint32_t cap,
                            uint32_t* nrec) {
  if (!ctx || !nrec) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  *nrec = 0;
  if (!ctx->trace) return IRGL_OK;
  DeviceGuard guard(ctx->device);
  const uint32_t k = std::min(std::min(cap, ctx->trace_cap), ctx->st_host->rounds + 2);
  std::vector<unsigned long long> buf(2 * (size_t)k);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && k)
    e = cudaMemcpy(buf.data(), ctx->trace, sizeof(unsigned long long) * buf.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "trace read");
  for (uint32_t i = 0; i < k; ++i) {
    if (t_ns) t_ns[i] = buf[2 * i];
    if (in_n) in_n[i] = static_cast<uint32_t>(buf[2 * i + 1] >> 32);
    if (out_n) out_n[i] = static_cast<uint32_t>(buf[2 * i + 1]);
  }
  *nrec = k;
  return IRGL_OK;
}

irgl_status irgl_trace_phases(irgl_ctx* ctx, uint64_t* words, uint32_t cap, uint32_t* nrec) {
  if (!ctx || !nrec || (cap && !words)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  *nrec = 0;
  if (!ctx->trace) return IRGL_OK;
  DeviceGuard guard(ctx->device);
  const uint32_t k = std::min(std::min(cap, ctx->trace_cap), ctx->st_host->rounds);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && k)
    e = cudaMemcpy(words, ctx->trace + 2 * (size_t)ctx->trace_cap, sizeof(unsigned long long) * kPhaseWords * k,
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "trace phases read");
  *nrec = k;
  return IRGL_OK;
}

irgl_status irgl_debug_set(irgl_ctx* ctx, int key, int64_t value) {
  if (!ctx) return fail(IRGL_ERR_INVALID_ARG, "ctx is NULL");
  switch (key) {
    case 1: ctx->dbg_timeout_us = value > 0 ? static_cast<uint64_t>(value) : 0; return IRGL_OK;
    case 2: ctx->dbg_skip_cta = static_cast<int>(value); return IRGL_OK;
    case 3: ctx->dbg_cap = value > 0 ? static_cast<uint32_t>(value) : 0; return IRGL_OK;
    case 4: ctx->dbg_big_cap = value > 0 ? static_cast<uint32_t>(value) : 0; return IRGL_OK;
    case 7: ctx->dbg_time_limit_ms = value > 0 ? static_cast<uint64_t>(value) : 0; return IRGL_OK;
    case 8: ctx->dbg_no_spread = value > 0 ? 1u : 0u; return IRGL_OK;
    case 5: ctx->dbg_force_bottom_up = value > 0 ? 1u : 0u; return IRGL_OK;
    case 6: ctx->dbg_held_lock = value >= 0 ? static_cast<uint32_t>(value) : 0xFFFFFFFFu; return IRGL_OK;
  }
  return fail(IRGL_ERR_INVALID_ARG, "unknown debug key %d", key);
}

// ---------------------------------------------------------------------------- graphs

irgl_status irgl_csr_validate(uint32_t n, uint64_t m, const uint32_t* row_ptr, const uint32_t* col,
                              const int32_t* w, int flags) {
  if (!row_ptr || (m > 0 && !col)) return fail(IRGL_ERR_INVALID_ARG, "row_ptr/col is NULL");
  if (m >= 0xFFFFFFFFull) return fail(IRGL_ERR_INVALID_ARG, "m must be < 2^32");
  if (n == 0xFFFFFFFFu) return fail(IRGL_ERR_INVALID_ARG, "n must be < 2^32 - 1");
  if (row_ptr[0] != 0) return fail(IRGL_ERR_INVALID_ARG, "row_ptr[0] must be 0");
  for (uint32_t u = 0; u < n; ++u)
    if (row_ptr[u + 1] < row_ptr[u]) return fail(IRGL_ERR_INVALID_ARG, "row_ptr not monotone at %u", u);
  if (row_ptr[n] != m) return fail(IRGL_ERR_INVALID_ARG, "row_ptr[n] != m");
  for (uint64_t e = 0; e < m; ++e)
    if (col[e] >= n) return fail(IRGL_ERR_INVALID_ARG, "col[%llu] = %u >= n", (unsigned long long)e, col[e]);
  if (w)
    for (uint64_t e = 0; e < m; ++e)
      if (w[e] < 0) return fail(IRGL_ERR_INVALID_ARG, "negative weight at edge %llu", (unsigned long long)e);
  if (flags & IRGL_SYMMETRIC) {
    // every (u, v) needs a (v, u): compare sorted copies of both directions
    std::vector<uint64_t> fwd, rev;
    try {
      fwd.resize(m);
      rev.resize(m);
    } catch (const std::bad_alloc&) {
      return fail(IRGL_ERR_OOM, "symmetry check");
    }
    for (uint32_t u = 0; u < n; ++u)
      for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        fwd[e] = (static_cast<uint64_t>(u) << 32) | col[e];
        rev[e] = (static_cast<uint64_t>(col[e]) << 32) | u;
      }
    std::sort(fwd.begin(), fwd.end());
    std::sort(rev.begin(), rev.end());
    if (fwd != rev) return fail(IRGL_ERR_NOT_SYMMETRIC, "graph flagged IRGL_SYMMETRIC is not symmetric");
  }
  return IRGL_OK;
}

irgl_status irgl_csr_load(irgl_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* row_ptr, const uint32_t* col,
                          const int32_t* w, int flags, irgl_graph** out) {
  if (!ctx || !out) return fail(IRGL_ERR_INVALID_ARG, "ctx/out is NULL");
  *out = nullptr;
  if (flags & ~(IRGL_DEVICE_PTRS | IRGL_SYMMETRIC | IRGL_VALIDATE | IRGL_IN_EDGES))
    return fail(IRGL_ERR_INVALID_ARG, "unknown flags");
  if ((flags & IRGL_IN_EDGES) && (flags & IRGL_DEVICE_PTRS))
    return fail(IRGL_ERR_UNSUPPORTED, "IRGL_IN_EDGES needs host pointers");
  if (m >= 0xFFFFFFFFull) return fail(IRGL_ERR_INVALID_ARG, "m must be < 2^32");
  DeviceGuard guard(ctx->device);
  const bool dev = (flags & IRGL_DEVICE_PTRS) != 0;
  int32_t max_w = 0;
  uint32_t max_deg = 0xFFFFFFFFu;  // unknown unless the offsets are read on the host
  if (!dev) {
    irgl_status s = irgl_csr_validate(n, m, row_ptr, col, w, flags);
    if (s != IRGL_OK) return s;
    if (w)
      for (uint64_t e = 0; e < m; ++e) max_w = std::max(max_w, w[e]);
    max_deg = 0;
    for (uint32_t v = 0; v < n; ++v) max_deg = std::max(max_deg, row_ptr[v + 1] - row_ptr[v]);
  } else {
    if (!row_ptr || (m > 0 && !col)) return fail(IRGL_ERR_INVALID_ARG, "row_ptr/col is NULL");
    if ((reinterpret_cast<uintptr_t>(col) & 15u) || (w && (reinterpret_cast<uintptr_t>(w) & 15u)))
      return fail(IRGL_ERR_INVALID_ARG, "device col/w must be 16-byte aligned");
    // Copy back for validation (IRGL_VALIDATE) and for the weight bound.
    if ((flags & IRGL_VALIDATE) || w) {
      std::vector<uint32_t> hr, hc;
      std::vector<int32_t> hw;
      try {
        if (flags & IRGL_VALIDATE) {
          hr.resize((size_t)n + 1);
          hc.resize(m);
        }
        if (w) hw.resize(m);
      } catch (const std::bad_alloc&) {
        return fail(IRGL_ERR_OOM, "validation copy");
      }
      cudaError_t e = cudaSuccess;
      if (flags & IRGL_VALIDATE) {
        e = cudaMemcpy(hr.data(), row_ptr, sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && m) e = cudaMemcpy(hc.data(), col, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost);
      }
      if (e == cudaSuccess && w && m) e = cudaMemcpy(hw.data(), w, sizeof(int32_t) * m, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "validation copy");
      if (flags & IRGL_VALIDATE) {
        irgl_status s = irgl_csr_validate(n, m, hr.data(), hc.data(), w ? hw.data() : nullptr, flags);
        if (s != IRGL_OK) return s;
        max_deg = 0;
        for (uint32_t v = 0; v < n; ++v) max_deg = std::max(max_deg, hr[v + 1] - hr[v]);
      }
      for (uint64_t e2 = 0; e2 < m && w; ++e2) {
        if (hw[e2] < 0) return fail(IRGL_ERR_INVALID_ARG, "negative weight at edge %llu", (unsigned long long)e2);
        max_w = std::max(max_w, hw[e2]);
      }
    }
  }
  irgl_graph* g = new (std::nothrow) irgl_graph();
  if (!g) return fail(IRGL_ERR_OOM, "graph allocation");
  g->ctx = ctx;
  g->n = n;
  g->m = m;
  g->flags = flags;
  g->max_w = max_w;
  g->max_deg = max_deg;
  if (dev) {
    g->row_ptr = const_cast<uint32_t*>(row_ptr);
    g->col = const_cast<uint32_t*>(col);
    g->w = const_cast<int32_t*>(w);
    g->owns = false;
  } else {
    g->owns = true;
    cudaError_t e = cudaMalloc(&g->row_ptr, sizeof(uint32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(uint32_t) * std::max<uint64_t>(m, 4));
    if (e == cudaSuccess && w) e = cudaMalloc(&g->w, sizeof(int32_t) * std::max<uint64_t>(m, 4));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && m)
      e = cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && w && m)
      e = cudaMemcpyAsync(g->w, w, sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && (flags & IRGL_IN_EDGES) && !(flags & IRGL_SYMMETRIC)) {
      // transpose by counting sort over destinations (rows of the result are in source order)
      std::vector<uint32_t> irp, icol;
      try {
        irp.assign((size_t)n + 1, 0);
        icol.resize(m);
      } catch (const std::bad_alloc&) {
        irgl_graph_destroy(g);
        return fail(IRGL_ERR_OOM, "in-edge build");
      }
      for (uint64_t k = 0; k < m; ++k) ++irp[(size_t)col[k] + 1];
      for (uint32_t v = 0; v < n; ++v) irp[(size_t)v + 1] += irp[v];
      std::vector<uint32_t> fillp(irp.begin(), irp.end() - 1);
      for (uint32_t u = 0; u < n; ++u)
        for (uint32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) icol[fillp[col[k]]++] = u;
      e = cudaMalloc(&g->in_row_ptr, sizeof(uint32_t) * ((size_t)n + 1));
      if (e == cudaSuccess) e = cudaMalloc(&g->in_col, sizeof(uint32_t) * std::max<uint64_t>(m, 4));
      if (e == cudaSuccess)
        e = cudaMemcpy(g->in_row_ptr, irp.data(), sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && m) e = cudaMemcpy(g->in_col, icol.data(), sizeof(uint32_t) * m, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      irgl_graph_destroy(g);
      return cuda_fail(e, "graph upload");
    }
  }
  *out = g;
  return IRGL_OK;
}

irgl_status irgl_graph_destroy(irgl_graph* g) {
  if (!g) return IRGL_OK;
  DeviceGuard guard(g->ctx->device);
  if (g->owns) {
    cudaStreamSynchronize(g->ctx->stream);
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->w);
  }
  cudaFree(g->in_row_ptr);
  cudaFree(g->in_col);
  delete g;
  return IRGL_OK;
}

irgl_status irgl_graph_info(const irgl_graph* g, uint32_t* n, uint64_t* m, int* flags) {
  if (!g) return fail(IRGL_ERR_INVALID_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (flags) *flags = g->flags;
  return IRGL_OK;
}

// ---------------------------------------------------------------------------- worklists

irgl_status irgl_worklist_create(irgl_ctx* ctx, uint32_t capacity, irgl_worklist** out) {
  if (!ctx || !out) return fail(IRGL_ERR_INVALID_ARG, "ctx/out is NULL");
  *out = nullptr;
  if (capacity == 0) return fail(IRGL_ERR_INVALID_ARG, "capacity must be > 0");
  DeviceGuard guard(ctx->device);
  irgl_worklist* wl = new (std::nothrow) irgl_worklist();
  if (!wl) return fail(IRGL_ERR_OOM, "worklist allocation");
  wl->ctx = ctx;
  wl->cap = capacity;
  cudaError_t e = cudaMalloc(&wl->items, sizeof(uint32_t) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&wl->tail, 128);
  if (e == cudaSuccess) e = cudaMemsetAsync(wl->tail, 0, 128, ctx->stream);
  if (e != cudaSuccess) {
    irgl_worklist_destroy(wl);
    return cuda_fail(e, "worklist allocation");
  }
  *out = wl;
  return IRGL_OK;
}

irgl_status irgl_worklist_destroy(irgl_worklist* wl) {
  if (!wl) return IRGL_OK;
  DeviceGuard guard(wl->ctx->device);
  cudaStreamSynchronize(wl->ctx->stream);
  cudaFree(wl->items);
  cudaFree(wl->tail);
  cudaFree(wl->staging);
  delete wl;
  return IRGL_OK;
}

irgl_status irgl_worklist_push(irgl_worklist* wl, const uint32_t* items_host, uint32_t k) {
  if (!wl || (k && !items_host)) return fail(IRGL_ERR_INVALID_ARG, "worklist/items is NULL");
  if (k == 0) return IRGL_OK;
  if (k > wl->cap) return fail(IRGL_ERR_WL_OVERFLOW, "push of %u items exceeds capacity %u", k, wl->cap);
  irgl_ctx* ctx = wl->ctx;
  DeviceGuard guard(ctx->device);
  if (k > wl->staging_n) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(wl->staging);
    wl->staging = nullptr;
    wl->staging_n = 0;
    cudaError_t e = cudaMalloc(&wl->staging, sizeof(uint32_t) * (size_t)k);
    if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
    wl->staging_n = k;
  }
  cudaError_t e = cudaMemcpyAsync(wl->staging, items_host, sizeof(uint32_t) * (size_t)k, cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess) e = launch_wl_append(wl->items, wl->tail, wl->cap, wl->staging, k, &ctx->st->err, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "worklist push");
  return IRGL_OK;
}

irgl_status irgl_worklist_push_range(irgl_worklist* wl, uint32_t k) {
  if (!wl) return fail(IRGL_ERR_INVALID_ARG, "worklist is NULL");
  if (k > wl->cap) return fail(IRGL_ERR_WL_OVERFLOW, "push of %u items exceeds capacity %u", k, wl->cap);
  DeviceGuard guard(wl->ctx->device);
  cudaError_t e = launch_wl_append(wl->items, wl->tail, wl->cap, nullptr, k, &wl->ctx->st->err, wl->ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "worklist push_range");
  return IRGL_OK;
}

irgl_status irgl_worklist_clear(irgl_worklist* wl) {
  if (!wl) return fail(IRGL_ERR_INVALID_ARG, "worklist is NULL");
  DeviceGuard guard(wl->ctx->device);
  cudaError_t e = cudaMemsetAsync(wl->tail, 0, sizeof(uint32_t), wl->ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "worklist clear");
  return IRGL_OK;
}

irgl_status irgl_worklist_size(irgl_worklist* wl, uint32_t* out) {
  if (!wl || !out) return fail(IRGL_ERR_INVALID_ARG, "worklist/out is NULL");
  irgl_ctx* ctx = wl->ctx;
  DeviceGuard guard(ctx->device);
  uint32_t* h = &ctx->st_host->pad3[0];
  cudaError_t e = cudaMemcpyAsync(h, wl->tail, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "worklist size");
  *out = std::min(*h, wl->cap);
  // surface a push overflow recorded by an append
  return read_status(ctx, nullptr);
}

irgl_status irgl_worklist_read(irgl_worklist* wl, uint32_t* items_host, uint32_t cap, uint32_t* n) {
  if (!wl || !n || (cap && !items_host)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  irgl_status s = irgl_worklist_size(wl, n);
  if (s != IRGL_OK) return s;
  const uint32_t k = std::min(*n, cap);
  if (k) {
    cudaError_t e = cudaMemcpy(items_host, wl->items, sizeof(uint32_t) * (size_t)k, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "worklist read");
  }
  return IRGL_OK;
}

// ---------------------------------------------------------------------------- kernels

irgl_status irgl_init_state(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial,
                            uint32_t* state_dev) {
  if (!ctx || !g || !state_dev) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  irgl_status s = check_kernel_graph(k, g);
  if (s != IRGL_OK) return s;
  DeviceGuard guard(ctx->device);
  irgl_tuning t = default_tuning();
  KParams p = make_params(ctx, g, state_dev, t);
  p.init_items = initial ? initial->items : nullptr;
  p.init_count = initial ? initial->tail : nullptr;
  p.init_cap = initial ? initial->cap : 0;
  const uint32_t grid = static_cast<uint32_t>(ctx->sm_count) * 4;
  cudaError_t e = launch_init_state(k == IRGL_CC_JUMP ? OP_CC : static_cast<uint32_t>(k), p, grid, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init_state launch");
  return IRGL_OK;
}

irgl_status irgl_invoke(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* in, irgl_worklist* out,
                        uint32_t* state_dev, uint32_t level, irgl_reduce r, const irgl_tuning* tin, int* result) {
  if (!ctx || !g || !in || !out || !state_dev) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (in == out) return fail(IRGL_ERR_INVALID_ARG, "in and out must be different worklists");
  if (r != IRGL_REDUCE_ANY && r != IRGL_REDUCE_ALL) return fail(IRGL_ERR_INVALID_ARG, "unknown reduction");
  if (k == IRGL_CC_JUMP) return fail(IRGL_ERR_UNSUPPORTED, "pointer-jumping CC runs only as a persistent Iterate");
  irgl_status s = check_kernel_graph(k, g);
  if (s != IRGL_OK) return s;
  irgl_tuning t;
  s = resolve_tuning(tin, &t);
  if (s != IRGL_OK) return s;
  DeviceGuard guard(ctx->device);
  s = ensure_workspace(ctx, g->n, k != IRGL_BFS);
  if (s != IRGL_OK) return s;
  KParams p = make_params(ctx, g, state_dev, t);
  RoundArgs a;
  a.in_items = in->items;
  a.in_count = in->tail;
  a.in_cap = in->cap;
  a.in_consume = in->tail;
  a.out_items = out->items;
  a.out_tail = out->tail;
  a.out_cap = out->cap;
  a.level = level;
  const int red = r == IRGL_REDUCE_ANY ? RED_ANY : RED_ALL;
  const int nb = occupancy(ctx, 1, static_cast<uint32_t>(k), t.cta_size, red);
  const uint32_t grid = std::max(1, nb) * static_cast<uint32_t>(ctx->sm_count);
  cudaError_t e = launch_round(static_cast<uint32_t>(k), t.cta_size, red, grid, p, a, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "invoke launch");
  DevStatus st;
  s = read_status(ctx, &st);
  if (s != IRGL_OK) return s;
  if (result) *result = static_cast<int>(st.result);
  return IRGL_OK;
}

}  // extern "C"

irgl_status iterate_impl(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial, uint32_t* state_dev,
                         irgl_mode mode, const irgl_tuning* tin, uint32_t max_rounds, irgl_stats* stats,
                         bool sync) {
  if (!ctx || !g || !state_dev) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (mode != IRGL_PER_LAUNCH && mode != IRGL_PERSISTENT) return fail(IRGL_ERR_INVALID_ARG, "unknown mode");
  irgl_status s = check_kernel_graph(k, g);
  if (s != IRGL_OK) return s;
  irgl_tuning t;
  s = resolve_tuning(tin, &t);
  if (s != IRGL_OK) return s;
  DeviceGuard guard(ctx->device);
  // CTA-local sub-rounds (persistent BFS and SSSP on packed words, plain rounds)
  const uint32_t sub_rounds = (t.flags >> 8) & 15u;
  const bool use_local = mode == IRGL_PERSISTENT && sub_rounds != 0 && !(t.flags & IRGL_TUNE_NO_PACKED) &&
                         ((k == IRGL_SSSP && t.delta == 0) ||
                          (k == IRGL_BFS && !(t.flags & (IRGL_TUNE_DIROPT | IRGL_TUNE_BITMAP))));
  const bool vis = k == IRGL_BFS && mode == IRGL_PERSISTENT && (t.flags & IRGL_TUNE_BITMAP) && !use_local;
  const bool packed = (k == IRGL_SSSP || (k == IRGL_BFS && use_local)) && mode == IRGL_PERSISTENT &&
                      !(t.flags & IRGL_TUNE_NO_PACKED);
  const bool far = (k == IRGL_SSSP || k == IRGL_CC) && mode == IRGL_PERSISTENT && t.delta != 0;
  // a vertex can be pushed once per sub-round: worklists of n * (sub-rounds + 1)
  s = ensure_workspace(ctx, g->n, k != IRGL_BFS, far, vis, packed, use_local ? sub_rounds + 1u : 1u);
  if (s != IRGL_OK) return s;
  const uint32_t op = (use_local && k == IRGL_BFS) ? OP_BFSR : op_of(k);
  if (k == IRGL_CC_JUMP && mode != IRGL_PERSISTENT)
    return fail(IRGL_ERR_UNSUPPORTED, "pointer-jumping CC runs only as a persistent Iterate");
  KParams p = make_params(ctx, g, state_dev, t);
  p.init_items = initial ? initial->items : nullptr;
  p.init_count = initial ? initial->tail : nullptr;
  p.init_cap = initial ? initial->cap : 0;
  p.max_rounds = max_rounds ? max_rounds : 0xFFFFFFFFu;
  if (vis) p.vis = ctx->ws_vis;
  if (packed) p.ds = ctx->ws_ds;
  if (mode == IRGL_PERSISTENT && k == IRGL_SSSP && packed && !far && !use_local &&
      !(t.flags & (IRGL_TUNE_NO_DEFER | IRGL_TUNE_DENSE))) {
    p.defer_deg = t.defer_deg;
    p.defer_delta = t.defer_delta;
  }
  if (mode == IRGL_PERSISTENT && p.diropt != 0 && !use_local) {
    // lists of the vertices each bottom-up round leaves open (the next one looks at those only)
    if (g->n > ctx->ws_bu_n) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws_bu[0]);
      cudaFree(ctx->ws_bu[1]);
      ctx->ws_bu[0] = ctx->ws_bu[1] = nullptr;
      ctx->ws_bu_n = 0;
      cudaError_t e = cudaMalloc(&ctx->ws_bu[0], sizeof(uint32_t) * (size_t)g->n);
      if (e == cudaSuccess) e = cudaMalloc(&ctx->ws_bu[1], sizeof(uint32_t) * (size_t)g->n);
      if (e != cudaSuccess) return cuda_fail(e, "bottom-up list allocation");
      ctx->ws_bu_n = g->n;
    }
    p.bu_list[0] = ctx->ws_bu[0];
    p.bu_list[1] = ctx->ws_bu[1];
  }
  if (use_local) {
    p.local_rounds = sub_rounds;
    p.diropt = 0;
    // round r stamps with ids r * (sub-rounds + 1) + 1 .. (r + 1) * (sub-rounds + 1):
    // stop before they would wrap to 0, the "on no worklist" stamp
    p.max_rounds = std::min(p.max_rounds, 0xFFFFFFFFu / (sub_rounds + 1u) - 1u);
  }
  irgl_stats local;
  std::memset(&local, 0, sizeof(local));
  local.cta_size = t.cta_size;

  if (mode == IRGL_PERSISTENT && !(t.flags & IRGL_TUNE_NO_SMEM) && k != IRGL_CC_JUMP &&
      ctx->smem_optin > static_cast<int>(kSmemStaticReserve) &&
      smem_iterate_fits(op_of(k), g->n, g->m, static_cast<size_t>(ctx->smem_optin) - kSmemStaticReserve)) {
    // the whole Iterate in one CTA, the graph in shared memory (schedule choices
    // such as sub-rounds, near-far or bottom-up rounds do not apply to it)
    p.skip_cta = -1;
    cudaError_t e = launch_smem_iterate(op_of(k), p, g->m, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory Iterate launch");
    local.grid = 1;
    local.cta_size = 1024;
    local.launches = 1;
    if (!sync) {
      if (stats) *stats = local;
      return IRGL_OK;
    }
    DevStatus st;
    s = read_status(ctx, &st);
    local.rounds = ctx->st_host->rounds;
    local.last_out = ctx->st_host->last_out;
    local.edges_scanned = ctx->st_host->edges;
    if (s == IRGL_OK) cudaMemsetAsync(&ctx->st->edges, 0, sizeof(unsigned long long), ctx->stream);
    if (stats) *stats = local;
    return s;
  }

  if (mode == IRGL_PERSISTENT) {
    const uint32_t grid = persistent_grid(ctx, op, t);
    if (grid == 0) return fail(IRGL_ERR_CUDA, "persistent kernel cannot be made resident");
    p.skip_cta = ctx->dbg_skip_cta;
    if (p.trace_ph != nullptr) {
      // phase records gather with atomicMax: cleared before each traced launch
      cudaError_t e = cudaMemsetAsync(p.trace_ph, 0, sizeof(unsigned long long) * kPhaseWords * p.trace_cap, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "trace phase clear");
    }
    cudaError_t e = launch_iterate(op, t.cta_size, grid, p, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "persistent launch");
    local.grid = grid;
    local.launches = 1;
    if (!sync) {
      if (stats) *stats = local;
      return IRGL_OK;
    }
    DevStatus st;
    s = read_status(ctx, &st);
    local.rounds = ctx->st_host->rounds;
    local.last_out = ctx->st_host->last_out;
    local.edges_scanned = ctx->st_host->edges;
    if (s == IRGL_OK) {
      // edges accumulate across calls: clear for the next one
      cudaMemsetAsync(&ctx->st->edges, 0, sizeof(unsigned long long), ctx->stream);
    }
    if (stats) *stats = local;
    return s;
  }

  // Per-launch: init, then one launch per round; the host reads the out size.
  const uint32_t init_grid = static_cast<uint32_t>(ctx->sm_count) * 4;
  cudaError_t e = launch_init_state(op, p, init_grid, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init launch");
  local.launches = 1 + (op != OP_CC ? 1 : 0);
  uint32_t n_in = g->n;
  if (initial) {
    e = cudaMemcpyAsync(&ctx->st_host->pad3[0], initial->tail, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "initial size");
    n_in = std::min(ctx->st_host->pad3[0], initial->cap);
  }
  const int nb = occupancy(ctx, 1, op, t.cta_size, RED_NONE);
  const uint32_t max_grid = std::max(1, nb) * static_cast<uint32_t>(ctx->sm_count);
  const uint32_t rmax = max_rounds ? max_rounds : 0xFFFFFFFFu;
  uint32_t r = 0;
  for (; n_in > 0; ++r) {
    if (r >= rmax) {
      local.rounds = r;
      local.last_out = n_in;
      if (stats) *stats = local;
      // leave the scratch tails clean
      cudaMemsetAsync(ctx->st->tail, 0, sizeof(uint32_t) * 4, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      return fail(IRGL_ERR_MAX_ROUNDS, "Iterate reached max_rounds with work left");
    }
    RoundArgs a;
    if (r == 0) {
      a.in_items = p.init_items;
      a.in_count = p.init_count;
      a.in_cap = p.init_cap;
      a.in_consume = nullptr;
    } else {
      a.in_items = ctx->ws_items[r & 1];
      a.in_count = &ctx->st->tail[r & 1];
      a.in_cap = ctx->ws_cap;
      a.in_consume = &ctx->st->tail[r & 1];
    }
    a.out_items = ctx->ws_items[(r + 1) & 1];
    a.out_tail = &ctx->st->tail[(r + 1) & 1];
    a.out_cap = ctx->ws_cap;
    a.level = r;
    const uint64_t tiles = (static_cast<uint64_t>(n_in) + t.cta_size * t.chunk - 1) / (t.cta_size * t.chunk);
    const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>(std::max<uint64_t>(tiles, 1), max_grid));
    local.grid = std::max(local.grid, grid);
    e = launch_round(op, t.cta_size, RED_NONE, grid, p, a, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "round launch");
    ++local.launches;
    DevStatus st;
    s = read_status(ctx, &st);
    if (s != IRGL_OK) {
      local.rounds = r + 1;
      if (stats) *stats = local;
      return s;
    }
    n_in = std::min(st.tail[(r + 1) & 1], ctx->ws_cap);
  }
  local.rounds = r;
  local.edges_scanned = ctx->st_host->edges;
  cudaMemsetAsync(&ctx->st->edges, 0, sizeof(unsigned long long), ctx->stream);
  if (sync) cudaStreamSynchronize(ctx->stream);
  if (stats) *stats = local;
  return IRGL_OK;
}

extern "C" {

irgl_status irgl_iterate(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial, uint32_t* state_dev,
                         irgl_mode mode, const irgl_tuning* t, uint32_t max_rounds, irgl_stats* stats) {
  return iterate_impl(ctx, k, g, initial, state_dev, mode, t, max_rounds, stats, true);
}

irgl_status irgl_iterate_async(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial,
                               uint32_t* state_dev, const irgl_tuning* t, uint32_t max_rounds) {
  return iterate_impl(ctx, k, g, initial, state_dev, IRGL_PERSISTENT, t, max_rounds, nullptr, false);
}

irgl_status irgl_ctx_sync(irgl_ctx* ctx, irgl_stats* stats) {
  if (!ctx) return fail(IRGL_ERR_INVALID_ARG, "ctx is NULL");
  DeviceGuard guard(ctx->device);
  DevStatus st;
  irgl_status s = read_status(ctx, &st);
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->rounds = st.rounds;
    stats->last_out = st.last_out;
    stats->edges_scanned = st.edges;
  }
  if (s == IRGL_OK) cudaMemsetAsync(&ctx->st->edges, 0, sizeof(unsigned long long), ctx->stream);
  return s;
}

irgl_status irgl_run(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, const uint32_t* srcs_host, uint32_t nsrc,
                     uint32_t* state, int state_on_host, irgl_mode mode, const irgl_tuning* t, uint32_t max_rounds,
                     irgl_stats* stats) {
  if (!ctx || !g || !state || (nsrc && !srcs_host)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(ctx->device);
  for (uint32_t i = 0; i < nsrc; ++i)
    if (srcs_host[i] >= g->n) return fail(IRGL_ERR_INVALID_ARG, "source %u out of range", srcs_host[i]);
  irgl_worklist* init = nullptr;
  if (nsrc > 0 && nsrc <= kRunSrcMax) {
    // count and sources in one copy (no clear, push kernel or staging copy)
    if (!ctx->run_src) {
      cudaError_t e = cudaMalloc(&ctx->run_src, sizeof(uint32_t) * kRunSrcWords);
      if (e == cudaSuccess) e = cudaMallocHost(&ctx->run_src_host, sizeof(uint32_t) * kRunSrcWords);
      if (e != cudaSuccess) return cuda_fail(e, "run source buffer");
      ctx->run_src_wl = new (std::nothrow) irgl_worklist();
      if (!ctx->run_src_wl) return fail(IRGL_ERR_OOM, "run source worklist");
      ctx->run_src_wl->ctx = ctx;
      ctx->run_src_wl->cap = kRunSrcMax;
      ctx->run_src_wl->tail = ctx->run_src;
      ctx->run_src_wl->items = ctx->run_src + 32;
      std::memset(ctx->run_src_host, 0, sizeof(uint32_t) * 32);
    }
    // the mirror is free again: every irgl_run waits for its stream before returning
    ctx->run_src_host[0] = nsrc;
    std::memcpy(ctx->run_src_host + 32, srcs_host, sizeof(uint32_t) * nsrc);
    cudaError_t e = cudaMemcpyAsync(ctx->run_src, ctx->run_src_host, sizeof(uint32_t) * (32 + (size_t)nsrc),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "run sources");
    init = ctx->run_src_wl;
  } else if (nsrc > 0) {
    if (!ctx->run_wl || ctx->run_wl->cap < nsrc) {
      if (ctx->run_wl) irgl_worklist_destroy(ctx->run_wl);
      ctx->run_wl = nullptr;
      irgl_status s = irgl_worklist_create(ctx, std::max<uint32_t>(nsrc, 64), &ctx->run_wl);
      if (s != IRGL_OK) return s;
    }
    irgl_status s = irgl_worklist_clear(ctx->run_wl);
    if (s == IRGL_OK) s = irgl_worklist_push(ctx->run_wl, srcs_host, nsrc);
    if (s != IRGL_OK) return s;
    init = ctx->run_wl;
  } else if (k != IRGL_CC && k != IRGL_CC_JUMP) {
    return fail(IRGL_ERR_INVALID_ARG, "BFS/SSSP need at least one source");
  }
  uint32_t* dst = state;
  if (state_on_host) {
    if (g->n > ctx->ws_state_n) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws_state);
      ctx->ws_state = nullptr;
      ctx->ws_state_n = 0;
      cudaError_t e = cudaMalloc(&ctx->ws_state, sizeof(uint32_t) * std::max<size_t>(g->n, 4));
      if (e != cudaSuccess) return cuda_fail(e, "result buffer");
      ctx->ws_state_n = g->n;
    }
    dst = ctx->ws_state;
  }
  irgl_status s = iterate_impl(ctx, k, g, init, dst, mode, t, max_rounds, stats, !state_on_host);
  if (s != IRGL_OK) return s;
  if (state_on_host) {
    cudaError_t e = cudaMemcpyAsync(state, dst, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    if (mode == IRGL_PERSISTENT) {
      // one wait for the launch, the result copy and the status read
      DevStatus st;
      s = read_status(ctx, &st);
      if (stats) {
        stats->rounds = ctx->st_host->rounds;
        stats->last_out = ctx->st_host->last_out;
        stats->edges_scanned = ctx->st_host->edges;
      }
      if (s != IRGL_OK) return s;
      // cleared for the next call; later work on the stream runs after it
      cudaMemsetAsync(&ctx->st->edges, 0, sizeof(unsigned long long), ctx->stream);
      return IRGL_OK;
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
  }
  return IRGL_OK;
}

}  // extern "C"
