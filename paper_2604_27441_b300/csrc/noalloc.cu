// revo_op_depth_stats_noalloc: the depth-statistics step for callers that
// cannot allocate device memory themselves.
//
// The statistics kernels need a few KB of global scratch for their per-block
// partial sums.  revo_op_depth_stats takes that scratch from the caller; this
// variant keeps it in a fixed array of this file instead, so nothing is
// allocated at call time.  Every GPU that loads the library holds the array
// (kNoAllocScratchBytes) until the process exits.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "revo.h"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr size_t kNoAllocScratchBytes = 8192;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_depth_stats_scratch[kNoAllocScratchBytes];

// The array's device address is a property of the context the module was
// loaded into: a cudaDeviceReset (or a caller switching to a context of its
// own) loads the module again, possibly elsewhere.  So the address kept for a
// device is tagged with the unique id of the context it was taken in
// (cuCtxGetId: unique for the life of the process, unlike the handle, which a
// re-created primary context can reuse) and looked up again when it differs.
struct Cached {
  unsigned long long ctx_id = 0;
  void* addr = nullptr;
};

std::mutex g_mu;
Cached g_cache[kMaxDevices];
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
std::once_flag g_once;

void resolve_driver() {
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
}

// Id of the calling thread's current context; 0 if there is none yet.
revo_status current_ctx_id(unsigned long long* id) {
  *id = 0;
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) {
    set_last_error("revo_op_depth_stats_noalloc: cuCtxGetCurrent failed");
    return REVO_ECUDA;
  }
  if (ctx && g_ctx_id(ctx, id) != CUDA_SUCCESS) {
    set_last_error("revo_op_depth_stats_noalloc: cuCtxGetId failed");
    return REVO_ECUDA;
  }
  return REVO_OK;
}

// Device address of the array in the current context of the current device
// (the host-side name is only a stand-in for it).
revo_status scratch_address(void** out) {
  std::call_once(g_once, resolve_driver);
  if (!g_ctx_current || !g_ctx_id) {
    set_last_error("revo_op_depth_stats_noalloc: the driver lacks cuCtxGetCurrent / cuCtxGetId");
    return REVO_ENOTSUP;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "revo_op_depth_stats_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("revo_op_depth_stats_noalloc: device ordinal %d beyond %d", dev, kMaxDevices - 1);
    return REVO_ENOTSUP;
  }
  unsigned long long id = 0;
  revo_status s = current_ctx_id(&id);
  if (s != REVO_OK) return s;
  std::lock_guard<std::mutex> lk(g_mu);
  Cached& c = g_cache[dev];
  if (id == 0 || c.ctx_id != id || !c.addr) {
    // Also makes the runtime's context current when the thread has none yet.
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_depth_stats_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e, "revo_op_depth_stats_noalloc: cudaGetSymbolAddress");
    if (id == 0 && (s = current_ctx_id(&id)) != REVO_OK) return s;
    c.ctx_id = id;
    c.addr = p;
  }
  *out = c.addr;
  return REVO_OK;
}

}  // namespace

}  // namespace revo

using namespace revo;

extern "C" revo_status revo_op_depth_stats_noalloc(const uint16_t* depth, int height, int width, size_t pitch_bytes,
                                                   float* mu_sigma, void* stream) {
  if (!depth || !mu_sigma || height < 0 || width < 0 || pitch_bytes < 2ull * static_cast<size_t>(width)) {
    set_last_error("revo_op_depth_stats_noalloc: bad argument");
    return REVO_EINVAL;
  }
  if (static_cast<long long>(height) * width > kDepthStatsMaxPixels) {
    set_last_error("revo_op_depth_stats_noalloc: frame of %d x %d pixels exceeds the maximum of %lld pixels", height,
                   width, kDepthStatsMaxPixels);
    return REVO_EINVAL;
  }
  if (depth_stats_scratch_bytes() > kNoAllocScratchBytes) {
    set_last_error("revo_op_depth_stats_noalloc: statistics scratch (%zu B) exceeds the fixed %zu B array",
                   depth_stats_scratch_bytes(), kNoAllocScratchBytes);
    return REVO_ENOTSUP;
  }
  void* scratch = nullptr;
  revo_status s = scratch_address(&scratch);
  if (s != REVO_OK) return s;
  // The launcher clears the scratch's arrival counters on the stream before the
  // kernels run; the partial sums are overwritten by every call.
  return cuda_status(
      launch_depth_stats(depth, height, width, pitch_bytes, mu_sigma, scratch, static_cast<cudaStream_t>(stream)),
      "revo_op_depth_stats_noalloc");
}
