// Autotuner for the block-level launch choices (the paper mentions auto-tuning
// over block-level optimisation choices in its conclusion; the search itself is
// this library's): coordinate descent over CTA size, warp and CTA degree
// thresholds, worklist chunk and CTAs per SM. Each candidate is timed as the
// median CUDA-event time of `reps` persistent runs on the caller's workload.
#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

using namespace irgl;

namespace {

struct Axis {
  uint32_t irgl_tuning::*field;
  std::vector<uint32_t> values;
};

std::vector<Axis> axes(bool with_delta, bool with_local, bool with_diropt, uint32_t sms, bool with_defer) {
  std::vector<Axis> a = {
      {&irgl_tuning::cta_size, {128, 256, 512, 1024}},
      {&irgl_tuning::cta_thresh, {32, 64, 128, 256, 512, 1024, 4096}},
      {&irgl_tuning::warp_thresh, {4, 8, 16, 32, 64}},
      {&irgl_tuning::chunk, {1, 2, 4}},
      {&irgl_tuning::blocks_per_sm, {0, 1, 2, 4}},
  };
  // total grid below one CTA per SM (blocks_per_sm cannot go there): a small
  // graph's rounds then synchronise a few CTAs, or one CTA with no grid barrier
  // at all (the barrier's occupancy bound of Sec. 3.4 is an upper bound only)
  if (sms) a.push_back({&irgl_tuning::max_blocks, {0, 1, 2, 8, 32, sms}});
  if (with_delta) a.push_back({&irgl_tuning::delta, {0, 16, 32, 64, 128, 256, 512, 1024}});
  // deferred expansion of long lists (single-query SSSP): degree bound and margin
  if (with_defer) {
    a.push_back({&irgl_tuning::defer_deg, {32, 64, 128, 256, 1024, 1u << 30}});
    a.push_back({&irgl_tuning::defer_delta, {1, 2, 4, 8, 16}});
  }
  // the flags the search sets (the defaults have none): CTA-local sub-rounds
  // and, when the graph has in-edges, direction-optimising BFS
  std::vector<uint32_t> fl = {0};
  if (with_local) {
    fl.push_back(IRGL_TUNE_LOCAL(4));
    fl.push_back(IRGL_TUNE_LOCAL(15));
  }
  if (with_diropt) fl.push_back(IRGL_TUNE_DIROPT);
  if (fl.size() > 1) a.push_back({&irgl_tuning::flags, fl});
  return a;
}

}  // namespace

// Coordinate descent; `measure` returns the median ms of one candidate (< 0: invalid).
irgl_status irgl::tune_descend(const std::function<float(const irgl_tuning&)>& measure, irgl_tuning* best, float* best_ms,
                                bool with_delta, bool with_local, bool with_diropt, uint32_t sms, bool with_defer) {
  irgl_tuning cur = default_tuning();
  float cur_ms = measure(cur);
  if (cur_ms < 0) return fail(IRGL_ERR_CUDA, "autotune: default tuning failed: %s", g_last_error.c_str());
  for (int pass = 0; pass < 2; ++pass) {
    bool moved = false;
    for (const Axis& ax : axes(with_delta, with_local, with_diropt, sms, with_defer)) {
      for (uint32_t v : ax.values) {
        if (cur.*(ax.field) == v) continue;
        irgl_tuning cand = cur;
        cand.*(ax.field) = v;
        if (cand.cta_thresh < cand.warp_thresh) continue;
        const float ms = measure(cand);
        if (ms >= 0 && ms < cur_ms * 0.98f) {
          cur = cand;
          cur_ms = ms;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return IRGL_OK;
}

namespace {

float median(std::vector<float>& v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? -1.f : v[v.size() / 2];
}

}  // namespace

extern "C" {

irgl_status irgl_autotune(irgl_ctx* ctx, irgl_kernel k, irgl_graph* g, const uint32_t* srcs_host, uint32_t nsrc,
                          uint32_t reps, irgl_tuning* best, float* best_ms) {
  if (!ctx || !g || !best || (nsrc && !srcs_host)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (k != IRGL_CC && k != IRGL_CC_JUMP && nsrc == 0) return fail(IRGL_ERR_INVALID_ARG, "BFS/SSSP need at least one source");
  irgl_status s = check_kernel_graph(k, g);
  if (s != IRGL_OK) return s;
  DeviceGuard guard(ctx->device);
  reps = std::max<uint32_t>(reps, 1);
  // sources on the context's run worklist, result into its scratch state
  if (nsrc) {
    if (!ctx->run_wl || ctx->run_wl->cap < nsrc) {
      if (ctx->run_wl) irgl_worklist_destroy(ctx->run_wl);
      ctx->run_wl = nullptr;
      s = irgl_worklist_create(ctx, std::max<uint32_t>(nsrc, 64), &ctx->run_wl);
      if (s != IRGL_OK) return s;
    }
    s = irgl_worklist_clear(ctx->run_wl);
    if (s == IRGL_OK) s = irgl_worklist_push(ctx->run_wl, srcs_host, nsrc);
    if (s != IRGL_OK) return s;
  }
  if (g->n > ctx->ws_state_n) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws_state);
    ctx->ws_state = nullptr;
    ctx->ws_state_n = 0;
    cudaError_t e = cudaMalloc(&ctx->ws_state, sizeof(uint32_t) * std::max<size_t>(g->n, 4));
    if (e != cudaSuccess) return cuda_fail(e, "autotune state");
    ctx->ws_state_n = g->n;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  irgl_worklist* init = nsrc ? ctx->run_wl : nullptr;
  auto measure = [&](const irgl_tuning& t) -> float {
    std::vector<float> ms;
    for (uint32_t r = 0; r <= reps; ++r) {  // first run warms up
      cudaEventRecord(e0, ctx->stream);
      if (iterate_impl(ctx, k, g, init, ctx->ws_state, IRGL_PERSISTENT, &t, 0, nullptr, false) != IRGL_OK)
        return -1.f;
      cudaEventRecord(e1, ctx->stream);
      if (read_status(ctx, nullptr) != IRGL_OK) return -1.f;
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r) ms.push_back(x);
    }
    return median(ms);
  };
  const bool diropt = k == IRGL_BFS && (g->in_row_ptr != nullptr || (g->flags & IRGL_SYMMETRIC));
  s = tune_descend(measure, best, best_ms, k == IRGL_SSSP, k == IRGL_BFS || k == IRGL_SSSP, diropt,
                   static_cast<uint32_t>(ctx->sm_count), k == IRGL_SSSP);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // extern "C"
