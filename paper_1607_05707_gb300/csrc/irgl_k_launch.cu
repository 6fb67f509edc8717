// One-invocation kernels (Invoke, per-launch Iterate rounds) and small helpers.
#include "irgl_launch.h"

namespace irgl {

template <uint32_t OP, int CTA, int RED>
__global__ void __launch_bounds__(CTA, MinBlocks<CTA>::value) k_round(KParams p, RoundArgs a) {
  __shared__ Smem<CTA> sm;
  invoke_round<OP, CTA, RED>(p, a, sm);
}

template <uint32_t OP>
__global__ void k_fill(KParams p) {
  fill_state<OP>(p.state, p.n, nullptr, 0, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void k_set_sources(KParams p) {
  const uint32_t cnt = p.init_count ? min(__ldcg(p.init_count), p.init_cap) : p.n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint32_t s = p.init_items ? __ldcg(p.init_items + i) : i;
    if (s < p.n) __stcg(p.state + s, 0u);
  }
}

__global__ void k_wl_append(uint32_t* items, uint32_t* tail, uint32_t cap, const uint32_t* src, uint32_t k,
                            uint32_t* err) {
  __shared__ uint32_t base;
  // one CTA reserves for the whole append, so the items stay in order
  if (threadIdx.x == 0) base = atomicAdd(tail, k);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    const uint32_t idx = base + i;
    if (idx < cap) items[idx] = src ? src[i] : i;
    else set_err(err, DERR_WL_OVERFLOW);
  }
}

namespace {

template <uint32_t OP, int CTA>
cudaError_t launch_red(int red, uint32_t grid, const KParams& p, const RoundArgs& a, cudaStream_t s) {
  switch (red) {
    case RED_NONE: k_round<OP, CTA, RED_NONE><<<grid, CTA, 0, s>>>(p, a); break;
    case RED_ANY: k_round<OP, CTA, RED_ANY><<<grid, CTA, 0, s>>>(p, a); break;
    case RED_ALL: k_round<OP, CTA, RED_ALL><<<grid, CTA, 0, s>>>(p, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <uint32_t OP, int CTA>
cudaError_t occ_red(int red, int* nb) {
  switch (red) {
    case RED_NONE: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_round<OP, CTA, RED_NONE>, CTA, 0);
    case RED_ANY: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_round<OP, CTA, RED_ANY>, CTA, 0);
    case RED_ALL: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_round<OP, CTA, RED_ALL>, CTA, 0);
  }
  return cudaErrorInvalidValue;
}

template <uint32_t OP>
cudaError_t launch_cta(uint32_t cta, int red, uint32_t grid, const KParams& p, const RoundArgs& a, cudaStream_t s) {
  switch (cta) {
    case 128: return launch_red<OP, 128>(red, grid, p, a, s);
    case 256: return launch_red<OP, 256>(red, grid, p, a, s);
    case 512: return launch_red<OP, 512>(red, grid, p, a, s);
    case 1024: return launch_red<OP, 1024>(red, grid, p, a, s);
  }
  return cudaErrorInvalidValue;
}

template <uint32_t OP>
cudaError_t occ_cta(uint32_t cta, int red, int* nb) {
  switch (cta) {
    case 128: return occ_red<OP, 128>(red, nb);
    case 256: return occ_red<OP, 256>(red, nb);
    case 512: return occ_red<OP, 512>(red, nb);
    case 1024: return occ_red<OP, 1024>(red, nb);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_round(uint32_t op, uint32_t cta, int red, uint32_t grid, const KParams& p, const RoundArgs& a,
                         cudaStream_t s) {
  switch (op) {
    case OP_BFS: return launch_cta<OP_BFS>(cta, red, grid, p, a, s);
    case OP_SSSP: return launch_cta<OP_SSSP>(cta, red, grid, p, a, s);
    case OP_CC: return launch_cta<OP_CC>(cta, red, grid, p, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_round(uint32_t op, uint32_t cta, int red, int* nb) {
  switch (op) {
    case OP_BFS: return occ_cta<OP_BFS>(cta, red, nb);
    case OP_SSSP: return occ_cta<OP_SSSP>(cta, red, nb);
    case OP_CC: return occ_cta<OP_CC>(cta, red, nb);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init_state(uint32_t op, const KParams& p, uint32_t grid, cudaStream_t s) {
  switch (op) {
    case OP_BFS: k_fill<OP_BFS><<<grid, 256, 0, s>>>(p); break;
    case OP_SSSP: k_fill<OP_SSSP><<<grid, 256, 0, s>>>(p); break;
    case OP_CC: k_fill<OP_CC><<<grid, 256, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  if (op != OP_CC) k_set_sources<<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_wl_append(uint32_t* items, uint32_t* tail, uint32_t cap, const uint32_t* src, uint32_t k,
                             uint32_t* err, cudaStream_t s) {
  if (k == 0) return cudaSuccess;
  k_wl_append<<<1, 1024, 0, s>>>(items, tail, cap, src, k, err);
  return cudaGetLastError();
}

}  // namespace irgl
