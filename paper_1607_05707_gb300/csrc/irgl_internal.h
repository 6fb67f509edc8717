// Host-side object layouts shared by the translation units of libirgl.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <unordered_map>

#include "irgl.h"
#include "irgl_device.cuh"

struct irgl_worklist;

struct irgl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int smem_optin = 0;  // opt-in shared memory per block (bytes)
  irgl::DevStatus* st = nullptr;       // device status block
  irgl::DevStatus* st_host = nullptr;  // pinned mirror
  uint32_t* run_src = nullptr;       // irgl_run sources (kRunSrcWords words, device)
  uint32_t* run_src_host = nullptr;  //   and their pinned mirror
  irgl_worklist* run_src_wl = nullptr;  // worklist view of run_src (owns nothing)
  uint32_t* ws_items[2] = {nullptr, nullptr};  // Iterate scratch worklists
  uint32_t ws_cap = 0;
  uint4* big_e = nullptr;               // big list of long adjacency lists (persistent kernels)
  unsigned long long* big_off = nullptr;
  uint32_t big_cap = 0;
  uint32_t* ws_far[2] = {nullptr, nullptr};  // SSSP near-far lists
  uint32_t* ws_far_stamp = nullptr;
  uint32_t ws_far_n = 0;
  uint32_t* ws_stamp = nullptr;  // SSSP/CC push dedup stamps
  uint32_t ws_stamp_n = 0;
  uint32_t* msf_buf = nullptr;   // minimum spanning forest workspace (status block + 14 arrays of msf_n)
  uint32_t msf_n = 0;
  void* msf_host = nullptr;      // pinned copy of its status block
  uint32_t* ws_bu[2] = {nullptr, nullptr};  // direction-optimising BFS: open-vertex lists
  uint32_t ws_bu_n = 0;
  uint32_t* ws_vis = nullptr;    // persistent BFS visited bitmap
  uint32_t ws_vis_words = 0;
  unsigned long long* ws_ds = nullptr;  // persistent SSSP packed (dist, round id) words
  uint32_t ws_ds_n = 0;
  uint32_t* ws_state = nullptr;  // result buffer of irgl_run with a host output
  uint32_t ws_state_n = 0;
  irgl_worklist* run_wl = nullptr;  // sources of irgl_run
  std::unordered_map<int, int> occ;  // occupancy cache
  unsigned long long* trace = nullptr;  // per-round trace (2 words per round)
  uint32_t trace_cap = 0;
  // test hooks
  uint64_t dbg_timeout_us = 0;
  uint64_t dbg_time_limit_ms = 0;  // wall-time limit of persistent launches (0: the default)
  uint32_t dbg_no_spread = 0;      // 1: sub-grid frontiers stay in static per-CTA spans
  int dbg_skip_cta = -1;
  uint32_t dbg_cap = 0;
  uint32_t dbg_big_cap = 0;
  uint32_t dbg_force_bottom_up = 0;
  uint32_t dbg_held_lock = 0xFFFFFFFFu;  // MSF: this component's lock starts held (never released)
};

struct irgl_graph {
  irgl_ctx* ctx = nullptr;
  uint32_t n = 0;
  uint64_t m = 0;
  uint32_t* row_ptr = nullptr;
  uint32_t* col = nullptr;
  int32_t* w = nullptr;
  bool owns = false;
  int flags = 0;
  int32_t max_w = 0;
  uint32_t max_deg = 0xFFFFFFFFu;  // largest out-degree (0xFFFFFFFF: not known)
  uint32_t* in_row_ptr = nullptr;  // in-edge CSR (IRGL_IN_EDGES), owned
  uint32_t* in_col = nullptr;
};

struct irgl_worklist {
  irgl_ctx* ctx = nullptr;
  uint32_t cap = 0;
  uint32_t* items = nullptr;
  uint32_t* tail = nullptr;     // device counter (own 128-byte line)
  uint32_t* staging = nullptr;  // device copy of host items being pushed
  uint32_t staging_n = 0;
};

// irgl_run's sources: one device block [count, 31 words of padding, items...]
// written by a single copy from a pinned mirror, viewed as a worklist.
constexpr uint32_t kRunSrcWords = 1024;
constexpr uint32_t kRunSrcMax = kRunSrcWords - 32;

namespace irgl {

struct DeviceGuard {
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
  int prev_ = 0;
  int dev_ = 0;
};

extern thread_local std::string g_last_error;
irgl_status fail(irgl_status s, const char* fmt, ...);
irgl_status cuda_fail(cudaError_t e, const char* what);
irgl_tuning default_tuning();
uint32_t thread_bin(const irgl_tuning& t);  // Tune::thread_max of a tuning
constexpr unsigned long long kRunTimeLimitNs = 60ull * 1000000000ull;  // persistent launches: 60 s
unsigned long long run_time_limit_ns(const irgl_ctx* ctx);
irgl_status resolve_tuning(const irgl_tuning* in, irgl_tuning* out);
irgl_status read_status(irgl_ctx* ctx, DevStatus* out);
irgl_status status_from_device(const DevStatus& s);
irgl_status control_cta(const uint32_t* masks, uint32_t count, uint32_t preferred, uint32_t* out);
void reset_status(irgl_ctx* ctx);
irgl_status ensure_workspace(irgl_ctx* ctx, uint32_t n, bool need_stamp, bool need_far = false,
                             bool need_vis = false, bool need_ds = false, uint32_t wl_mult = 1);
uint32_t big_capacity(uint64_t n);
cudaError_t alloc_big(uint32_t cap, uint4** e, unsigned long long** off);
int occupancy(irgl_ctx* ctx, int kind, uint32_t op, uint32_t cta, int red);
uint32_t persistent_grid(irgl_ctx* ctx, uint32_t op, const irgl_tuning& t);
irgl_status check_kernel_graph(irgl_kernel k, const irgl_graph* g);
uint32_t op_of(irgl_kernel k);
KParams make_params(irgl_ctx* ctx, irgl_graph* g, uint32_t* state, const irgl_tuning& t);
irgl_status tune_descend(const std::function<float(const irgl_tuning&)>& measure, irgl_tuning* best, float* best_ms,
                         bool with_delta = false, bool with_local = false, bool with_diropt = false,
                         uint32_t sms = 0, bool with_defer = false);

}  // namespace irgl

irgl_status iterate_impl(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, irgl_worklist* initial, uint32_t* state_dev,
                         irgl_mode mode, const irgl_tuning* tin, uint32_t max_rounds, irgl_stats* stats, bool sync);
