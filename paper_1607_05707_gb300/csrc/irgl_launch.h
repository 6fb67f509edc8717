// Host-side launchers of the sm_103a kernels (one set per translation unit).
#pragma once

#include <cuda_runtime.h>

#include "irgl_device.cuh"

namespace irgl {

// Persistent (iteration-outlined) Iterate: one cooperative launch.
cudaError_t launch_iterate(uint32_t op, uint32_t cta, uint32_t grid, const KParams& p, cudaStream_t s);
cudaError_t occupancy_iterate(uint32_t op, uint32_t cta, int* blocks_per_sm);

// One invocation (Invoke / a round of a per-launch Iterate).
cudaError_t launch_round(uint32_t op, uint32_t cta, int red, uint32_t grid, const KParams& p, const RoundArgs& a,
                         cudaStream_t s);
cudaError_t occupancy_round(uint32_t op, uint32_t cta, int red, int* blocks_per_sm);

// Initial values of an Iterate (state fill, then sources = 0).
cudaError_t launch_init_state(uint32_t op, const KParams& p, uint32_t grid, cudaStream_t s);

// Worklist append helpers: items[tail..] = src[0..k) (src == nullptr: 0..k-1).
cudaError_t launch_wl_append(uint32_t* items, uint32_t* tail, uint32_t cap, const uint32_t* src, uint32_t k,
                             uint32_t* err, cudaStream_t s);

// Batched multi-query Iterate (cooperative) and query admission.
cudaError_t launch_batch_iterate(uint32_t cta, uint32_t grid, const BParams& p, cudaStream_t s);
cudaError_t occupancy_batch(uint32_t cta, int* blocks_per_sm);
cudaError_t launch_admit(const AdmitParams& a, uint32_t grid, cudaStream_t s);
// out[i] = value half of the packed arena word ds[i], i < n.
cudaError_t launch_extract_values(const unsigned long long* ds, uint32_t* out, uint64_t n, uint32_t grid,
                                  cudaStream_t s);

inline bool valid_cta(uint32_t cta) { return cta == 128 || cta == 256 || cta == 512 || cta == 1024; }

}  // namespace irgl
