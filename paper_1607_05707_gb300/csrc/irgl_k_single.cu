// Persistent cooperative Iterate kernels: BFS / SSSP / CC / pointer-jumping CC x CTA size.
#include "irgl_launch.h"

namespace irgl {

template <uint32_t OP, int CTA>
__global__ void __launch_bounds__(CTA, MinBlocks<CTA>::value) k_iterate(KParams p) {
  __shared__ Smem<CTA> sm;
  if constexpr (OP == OP_CCJ) cc_jump_persistent<CTA>(p, sm);
  else iterate_persistent<OP, CTA>(p, sm);
}

namespace {

template <uint32_t OP, int CTA>
cudaError_t launch_one(uint32_t grid, const KParams& p, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(CTA);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_iterate<OP, CTA>, p);
}

template <uint32_t OP>
cudaError_t launch_op(uint32_t cta, uint32_t grid, const KParams& p, cudaStream_t s) {
  switch (cta) {
    case 128: return launch_one<OP, 128>(grid, p, s);
    case 256: return launch_one<OP, 256>(grid, p, s);
    case 512: return launch_one<OP, 512>(grid, p, s);
    case 1024: return launch_one<OP, 1024>(grid, p, s);
  }
  return cudaErrorInvalidValue;
}

template <uint32_t OP>
cudaError_t occ_op(uint32_t cta, int* nb) {
  switch (cta) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_iterate<OP, 128>, 128, 0);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_iterate<OP, 256>, 256, 0);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_iterate<OP, 512>, 512, 0);
    case 1024: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_iterate<OP, 1024>, 1024, 0);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_iterate(uint32_t op, uint32_t cta, uint32_t grid, const KParams& p, cudaStream_t s) {
  switch (op) {
    case OP_BFS: return launch_op<OP_BFS>(cta, grid, p, s);
    case OP_SSSP: return launch_op<OP_SSSP>(cta, grid, p, s);
    case OP_CC: return launch_op<OP_CC>(cta, grid, p, s);
    case OP_CCJ: return launch_op<OP_CCJ>(cta, grid, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_iterate(uint32_t op, uint32_t cta, int* nb) {
  switch (op) {
    case OP_BFS: return occ_op<OP_BFS>(cta, nb);
    case OP_SSSP: return occ_op<OP_SSSP>(cta, nb);
    case OP_CC: return occ_op<OP_CC>(cta, nb);
    case OP_CCJ: return occ_op<OP_CCJ>(cta, nb);
  }
  return cudaErrorInvalidValue;
}

}  // namespace irgl
