// Batched kernels: admission (initial values + pending sources) and the
// persistent multi-query Iterate (one cooperative launch for all instances).
#include "irgl_launch.h"

namespace irgl {

template <int CTA>
__global__ void __launch_bounds__(CTA, MinBlocks<CTA>::value) k_batch_iterate(BParams p) {
  __shared__ BatchSmem<CTA> bs;
  iterate_batch<CTA>(p, bs);
}

__global__ void __launch_bounds__(256) k_batch_fill(AdmitParams a) { admit_fill(a); }
__global__ void __launch_bounds__(256) k_batch_sources(AdmitParams a) { admit_sources(a); }

// Results out of the packed arena: out[i] = ds[i] >> 32 (the value half),
// two entries per thread per step.
__global__ void __launch_bounds__(256) k_extract_values(const unsigned long long* __restrict__ ds,
                                                        uint32_t* __restrict__ out, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    __stcs(out + i, static_cast<uint32_t>(__ldcs(ds + i) >> 32));
}

namespace {

template <int CTA>
cudaError_t launch_b(uint32_t grid, const BParams& p, cudaStream_t s) {
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
  return cudaLaunchKernelEx(&cfg, k_batch_iterate<CTA>, p);
}

}  // namespace

cudaError_t launch_batch_iterate(uint32_t cta, uint32_t grid, const BParams& p, cudaStream_t s) {
  switch (cta) {
    case 128: return launch_b<128>(grid, p, s);
    case 256: return launch_b<256>(grid, p, s);
    case 512: return launch_b<512>(grid, p, s);
    case 1024: return launch_b<1024>(grid, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_batch(uint32_t cta, int* nb) {
  switch (cta) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_batch_iterate<128>, 128, 0);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_batch_iterate<256>, 256, 0);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_batch_iterate<512>, 512, 0);
    case 1024: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_batch_iterate<1024>, 1024, 0);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_extract_values(const unsigned long long* ds, uint32_t* out, uint64_t n, uint32_t grid,
                                  cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_extract_values<<<grid, 256, 0, s>>>(ds, out, n);
  return cudaGetLastError();
}

cudaError_t launch_admit(const AdmitParams& a, uint32_t grid, cudaStream_t s) {
  if (a.nnew == 0) return cudaSuccess;
  k_batch_fill<<<grid, 256, 0, s>>>(a);
  k_batch_sources<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace irgl
