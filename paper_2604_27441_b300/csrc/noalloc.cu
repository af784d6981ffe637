// revo_op_depth_stats_noalloc: the depth-statistics step for callers that
// cannot allocate device memory themselves.
//
// The statistics kernels need a few KB of global scratch for their per-block
// partial sums.  revo_op_depth_stats takes that scratch from the caller; this
// variant keeps it in a fixed array of this file instead, so nothing is
// allocated at call time.  Every GPU that loads the library holds the array
// (kNoAllocScratchBytes) until the process exits.
#include <mutex>

#include "common.cuh"
#include "revo.h"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr size_t kNoAllocScratchBytes = 8192;
// The exact float32 division by the pixel count in the statistics needs
// count < 2^24, which bounds the frames this variant accepts.
constexpr long long kNoAllocMaxPixels = 1LL << 24;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_depth_stats_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device (looked up once per device;
// the host-side name is only a stand-in for it).
revo_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "revo_op_depth_stats_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("revo_op_depth_stats_noalloc: device ordinal %d beyond %d", dev, kMaxDevices - 1);
    return REVO_ENOTSUP;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_depth_stats_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e, "revo_op_depth_stats_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
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
  if (static_cast<long long>(height) * width > kNoAllocMaxPixels) {
    set_last_error("revo_op_depth_stats_noalloc: frame of %d x %d pixels exceeds the maximum of %lld pixels", height,
                   width, kNoAllocMaxPixels);
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
