// irgl_bfs_noalloc: the persistent BFS Iterate for callers that cannot allocate
// device memory.
//
// Who needs it: code that must not call cudaMalloc at all, for example a
// plugin inside a host application whose own allocator reserves the whole
// device at start-up, or a latency-critical loop that cannot afford the
// implicit device synchronisation an allocation can bring. Such callers still
// own their inputs and outputs (CSR arrays and the level array); everything
// else the kernel needs (status block, the two worklists, the big list) lives
// in the file-scope array below, which every GPU that loads this library keeps
// until the process exits.
//
// Limits and sharing: at most kNoAllocMaxN vertices per graph (a larger graph
// is rejected with IRGL_ERR_INVALID_ARG before any GPU work). Every call on a
// device uses the same array and it keeps the previous call's contents, so each
// call clears the counters that must start at zero; calls whose GPU work
// overlaps (other streams or threads) race on the array and give wrong results.
// A non-null stream must belong to `device` (checked: IRGL_ERR_INVALID_ARG).
// The first call on a device looks up the array's device address (with that
// device current) and caches it. Every call copies its source from host
// memory, reads the status block back and synchronises the stream before it
// returns, so no call can be captured into a CUDA graph.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "irgl.h"
#include "irgl_internal.h"
#include "irgl_launch.h"

namespace irgl {
namespace {

constexpr uint32_t kNoAllocMaxN = 1u << 20;    // vertices
constexpr uint32_t kNoAllocBigCap = 1u << 16;  // big-list entries; long lists beyond it go to the warp bin
constexpr int kNoAllocCta = 256;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  DevStatus st;
  uint32_t init[32];  // the source and its count (round-0 worklist)
  uint32_t items[2][kNoAllocMaxN];
  uint4 big_e[kNoAllocBigCap];
  unsigned long long big_off[kNoAllocBigCap];
};

// about 1 KiB status + 128 B + 8 MiB worklists + 1.5 MiB big list: about 9.6 MiB per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

__global__ void __launch_bounds__(kNoAllocCta, MinBlocks<kNoAllocCta>::value) k_bfs_noalloc(KParams p) {
  __shared__ Smem<kNoAllocCta> sm;
  iterate_persistent<OP_BFS, kNoAllocCta>(p, sm);
}

struct DeviceSetup {
  bool ready = false;
  NoAllocScratch* scratch = nullptr;
  uint32_t grid = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

irgl_status setup_device(int device, DeviceSetup* out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup& d = g_setup[device];
  if (!d.ready) {
    DeviceGuard guard(device);  // the address is looked up with this device current
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc scratch address");
    int nb = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bfs_noalloc, kNoAllocCta, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc launch set-up");
    if (nb <= 0) return fail(IRGL_ERR_CUDA, "no-alloc kernel cannot be made resident");
    d.scratch = static_cast<NoAllocScratch*>(ptr);
    d.grid = std::min<uint32_t>(static_cast<uint32_t>(nb) * static_cast<uint32_t>(sms), kMaxGrid);
    d.ready = true;
  }
  *out = d;
  return IRGL_OK;
}

}  // namespace
}  // namespace irgl

using namespace irgl;

extern "C" irgl_status irgl_bfs_noalloc(int device, void* cuda_stream, uint32_t n, uint64_t m, const uint32_t* row_ptr,
                                        const uint32_t* col, uint32_t src, uint32_t* level, uint32_t* rounds) {
  if (!row_ptr || !level || (m > 0 && !col)) return fail(IRGL_ERR_INVALID_ARG, "NULL argument");
  if (n == 0 || n > kNoAllocMaxN)
    return fail(IRGL_ERR_INVALID_ARG, "irgl_bfs_noalloc handles 1..%u vertices, got %u", kNoAllocMaxN, n);
  if (m >= 0xFFFFFFFFull) return fail(IRGL_ERR_INVALID_ARG, "m must be < 2^32");
  if (src >= n) return fail(IRGL_ERR_INVALID_ARG, "source %u out of range", src);
  if (reinterpret_cast<uintptr_t>(col) & 15u) return fail(IRGL_ERR_INVALID_ARG, "col must be 16-byte aligned");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev || device >= kMaxDevices)
    return fail(IRGL_ERR_INVALID_ARG, "device %d out of range", device);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (stream != nullptr) {
    // the scratch address below is the one on `device`: a stream of another GPU would
    // send the launch to that GPU's copy of the array through the wrong address
    int sdev = -1;
    e = cudaStreamGetDevice(stream, &sdev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetDevice");
    if (sdev != device) return fail(IRGL_ERR_INVALID_ARG, "cuda_stream belongs to device %d, not %d", sdev, device);
  }
  DeviceSetup d;
  irgl_status s = setup_device(device, &d);
  if (s != IRGL_OK) return s;
  DeviceGuard guard(device);
  NoAllocScratch* sc = d.scratch;

  // what must start at zero: the whole status block (barrier, tails, grabs, big list, error)
  e = cudaMemsetAsync(&sc->st, 0, sizeof(DevStatus), stream);
  const uint32_t init_host[2] = {src, 1u};  // source and count, copied before the call returns
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc->init, init_host, sizeof(init_host), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc set-up copies");

  irgl_tuning t = default_tuning();
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.row_ptr = row_ptr;
  p.col = col;
  p.w = nullptr;
  p.n = n;
  p.state = level;
  p.stamp = nullptr;  // BFS pushes each vertex once (CAS), no stamps
  p.init_items = sc->init;
  p.init_count = sc->init + 1;
  p.init_cap = 1;
  p.items[0] = sc->items[0];
  p.items[1] = sc->items[1];
  p.cap = kNoAllocMaxN;
  p.st = &sc->st;
  p.tn = Tune{t.warp_thresh, t.cta_thresh, t.chunk};
  p.max_rounds = 0xFFFFFFFFu;
  p.timeout_ns = 2000000000ull;
  p.skip_cta = -1;
  p.init_state = 1;
  p.trace = nullptr;
  p.trace_cap = 0;
  p.big = BigList{sc->big_e, sc->big_off, kNoAllocBigCap};

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.grid);
  cfg.blockDim = dim3(kNoAllocCta);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_bfs_noalloc, p);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc launch");

  DevStatus st_host;
  e = cudaMemcpyAsync(&st_host, &sc->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc status");
  if (rounds) *rounds = st_host.rounds;
  switch (st_host.err) {
    case DERR_NONE: return IRGL_OK;
    case DERR_WL_OVERFLOW: return fail(IRGL_ERR_WL_OVERFLOW, "a push found the worklist full");
    case DERR_BARRIER_TIMEOUT: return fail(IRGL_ERR_BARRIER_TIMEOUT, "grid barrier wait exceeded its time limit");
    case DERR_BAD_ITEM: return fail(IRGL_ERR_INVALID_ARG, "a worklist item is not a vertex of the graph");
  }
  return fail(IRGL_ERR_CUDA, "device error %u", st_host.err);
}
