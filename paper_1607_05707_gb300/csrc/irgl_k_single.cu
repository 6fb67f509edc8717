// Persistent cooperative Iterate kernels: BFS / SSSP / CC / pointer-jumping CC / BFS by relaxation x CTA size.
#include <algorithm>

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

// Resident CTAs per SM, after asking for the smallest shared-memory carveout
// that keeps them all resident: the rest of the SM's 256 KB stays L1, which
// caches the row offsets and (with the BFS bitmap) the visited bits. The
// carveout is kept only if the occupancy calculator still gives the same
// number of CTAs (the persistent grid is sized from it).
template <class K>
cudaError_t occ_prefer_l1(K kern, int cta, int* nb) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, cta, 0);
  if (e != cudaSuccess || *nb <= 0) return e;
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, reserved = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess || smem_sm <= 0)
    return cudaSuccess;  // keep the default carveout
  const long long need = static_cast<long long>(*nb) * (static_cast<long long>(fa.sharedSizeBytes) + reserved);
  const int pct = static_cast<int>(std::min<long long>(100, (need * 100 + smem_sm - 1) / smem_sm));
  if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess) {
    cudaGetLastError();  // the refused hint's own error, not a sticky one
    return cudaSuccess;
  }
  int nb2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, kern, cta, 0) != cudaSuccess || nb2 != *nb) {
    cudaGetLastError();
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, cta, 0);
}

template <uint32_t OP>
cudaError_t occ_op(uint32_t cta, int* nb) {
  switch (cta) {
    case 128: return occ_prefer_l1(k_iterate<OP, 128>, 128, nb);
    case 256: return occ_prefer_l1(k_iterate<OP, 256>, 256, nb);
    case 512: return occ_prefer_l1(k_iterate<OP, 512>, 512, nb);
    case 1024: return occ_prefer_l1(k_iterate<OP, 1024>, 1024, nb);
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
    case OP_BFSR: return launch_op<OP_BFSR>(cta, grid, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_iterate(uint32_t op, uint32_t cta, int* nb) {
  switch (op) {
    case OP_BFS: return occ_op<OP_BFS>(cta, nb);
    case OP_SSSP: return occ_op<OP_SSSP>(cta, nb);
    case OP_CC: return occ_op<OP_CC>(cta, nb);
    case OP_CCJ: return occ_op<OP_CCJ>(cta, nb);
    case OP_BFSR: return occ_op<OP_BFSR>(cta, nb);
  }
  return cudaErrorInvalidValue;
}

}  // namespace irgl
