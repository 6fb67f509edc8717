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

// Iterate in one CTA with the graph in shared memory (BFS, SSSP, min-label CC):
// bytes of dynamic shared memory it needs, whether that fits `limit` (the
// device's opt-in per-block maximum less the kernel's static shared memory),
// and the launch (one CTA of 1024 threads; the status block gets rounds,
// out size, edges and errors like a persistent launch).
size_t smem_iterate_bytes(uint32_t op, uint32_t n, uint64_t m);
bool smem_iterate_fits(uint32_t op, uint32_t n, uint64_t m, size_t limit);
cudaError_t launch_smem_iterate(uint32_t op, const KParams& p, uint64_t m, cudaStream_t s);
constexpr size_t kSmemStaticReserve = 256;  // the kernel's own __shared__ counters, rounded up

inline bool valid_cta(uint32_t cta) { return cta == 128 || cta == 256 || cta == 512 || cta == 1024; }

}  // namespace irgl
