// Step-level entry points of the C ABI: each runs one stage of the recovery
// forward on caller-owned device buffers.
#include <stdarg.h>
#include <string.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "revo.h"
#include <vector>

#include "revo_internal.h"

namespace revo {

namespace {
thread_local std::string g_last_error;
std::mutex g_err_mu;
int* g_err_word[64] = {nullptr};
}  // namespace

void set_last_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

revo_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return REVO_OK;
  set_last_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorInvalidValue ? REVO_EINVAL : REVO_ECUDA;
}

// The device error word the step-level tensor-core kernels report timeouts in
// (one per device, allocated on first use).
int* op_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_word[dev]) {
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
    g_err_word[dev] = p;
  }
  return g_err_word[dev];
}

// Device scratch of the step-level entry points, one buffer per kind and
// device, grown on demand (a grown buffer replaces the old one after the
// device is idle: earlier launches may still use it); calls on one device run
// in stream order.
enum OpScratch { kScratchAttnPartial = 0, kScratchLnCounters = 1, kScratchPePositions = 2, kScratchKinds = 3 };
void* op_scratch(int kind, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  static void* bufs[kScratchKinds][64] = {};
  static size_t sizes[kScratchKinds][64] = {};
  std::lock_guard<std::mutex> lk(g_err_mu);
  void*& buf = bufs[kind][dev];
  if (!buf || sizes[kind][dev] < bytes) {
    if (buf) {
      if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
      cudaFree(buf);
      buf = nullptr;
      sizes[kind][dev] = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes < 256 ? 256 : bytes) != cudaSuccess) return nullptr;
    buf = p;
    sizes[kind][dev] = bytes;
  }
  return buf;
}

// The frequencies of the position embedding's parts at width D, one copy per
// device and width (built on first use).
const float* op_pe_omega(int D) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || D % 192 || D > 1024) return nullptr;
  static float* oms[64][6] = {};
  const int w = D / 192 - 1;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!oms[dev][w]) {
    float host[128] = {};
    float* p = nullptr;
    if (!pe_omega(D, host) || cudaMalloc(&p, sizeof(host)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(p, host, sizeof(host), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    oms[dev][w] = p;
  }
  return oms[dev][w];
}

// The position embedding's column-part table of the step-level entry point,
// one per device and width (built on first use).
float* op_pe_table(int D, int rows) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || D % 192 || D > 1024) return nullptr;
  static float* tabs[64][6] = {};
  const int w = D / 192 - 1;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!tabs[dev][w]) {
    float* p = nullptr;
    if (cudaMalloc(&p, static_cast<size_t>(rows) * (D / 3) * sizeof(float)) != cudaSuccess) return nullptr;
    if (launch_pe_table(p, rows, D, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    tabs[dev][w] = p;
  }
  return tabs[dev][w];
}

// The argument table of the step-level batched launches (one per device,
// grown on demand; calls on one device run in stream order).  The host bytes
// are uploaded on `st` unless the table already holds exactly them (a repeated
// call with the same jobs launches without a copy).  Returns the device table.
void* op_arg_table(const void* host, size_t bytes, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  static void* bufs[64] = {};
  static size_t sizes[64] = {};
  static std::vector<uint8_t> held[64];
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!bufs[dev] || sizes[dev] < bytes) {
    if (bufs[dev]) {
      if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
      cudaFree(bufs[dev]);
      bufs[dev] = nullptr;
    }
    held[dev].clear();
    if (cudaMalloc(&bufs[dev], bytes) != cudaSuccess) return nullptr;
    sizes[dev] = bytes;
  }
  const uint8_t* h = static_cast<const uint8_t*>(host);
  if (held[dev].size() != bytes || memcmp(held[dev].data(), h, bytes) != 0) {
    // From pageable memory: the call returns once the bytes are staged.
    if (cudaMemcpyAsync(bufs[dev], h, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    held[dev].assign(h, h + bytes);
  }
  return bufs[dev];
}

}  // namespace revo

using namespace revo;

extern "C" {

const char* revo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace revo {
namespace {
// One thread waits on an mbarrier that nothing completes: the bounded wait
// every pipeline kernel uses gives up after `limit` clocks, records its code
// in the error word and returns.
__global__ void wait_selftest_kernel(int* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbarrier_init();
  mbar_wait(&bar, 0, err, kDevTimeoutSelftest, limit);
}
}  // namespace
}  // namespace revo

extern "C" {

revo_status revo_op_wait_selftest(long long limit_cycles, void* stream) {
  if (limit_cycles < 1000 || limit_cycles > kWaitLimitCycles) {
    set_last_error("revo_op_wait_selftest: limit_cycles outside [1000, %lld]", kWaitLimitCycles);
    return REVO_EINVAL;
  }
  int* err = op_error_word();
  if (!err) {
    set_last_error("revo_op_wait_selftest: no device error word");
    return REVO_ECUDA;
  }
  wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err, limit_cycles);
  return cuda_status(cudaGetLastError(), "revo_op_wait_selftest");
}

int revo_op_take_device_error(void) {
  int* w = op_error_word();
  if (!w) return -1;
  int v = 0;
  if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (v) cudaMemset(w, 0, sizeof(int));
  return v;
}

revo_status revo_op_assemble(int channels, int k, int T, int p, int height, int width, const void* const* refs,
                             const void* current, size_t pitch_bytes, const float* mu_sigma, void* out, int out_bf16,
                             void* stream) {
  if (!current || !out || (k > 0 && !refs) || k < 0 || k > kMaxRefs || (channels == 1 && !mu_sigma)) {
    set_last_error("revo_op_assemble: null pointer or k out of range");
    return REVO_EINVAL;
  }
  AssembleArgs a{};
  for (int i = 0; i < k; ++i) {
    if (!refs[i]) {
      set_last_error("revo_op_assemble: null reference frame");
      return REVO_EINVAL;
    }
    a.frames[i] = refs[i];
    a.pitch[i] = pitch_bytes;
  }
  a.frames[k] = current;
  a.pitch[k] = pitch_bytes;
  a.mu_sigma = mu_sigma;
  a.out = out;
  a.C = channels;
  a.F = k + 1;
  a.T = T;
  a.p = p;
  a.H = height;
  a.W = width;
  a.out_bf16 = out_bf16;
  return cuda_status(launch_assemble(a, static_cast<cudaStream_t>(stream)), "revo_op_assemble");
}

size_t revo_depth_stats_scratch_bytes(void) { return depth_stats_scratch_bytes(); }

revo_status revo_op_depth_stats(const uint16_t* depth, int height, int width, size_t pitch_bytes, float* mu_sigma,
                                void* scratch, void* stream) {
  if (!depth || !mu_sigma || !scratch || height < 0 || width < 0 || pitch_bytes < 2ull * width) {
    set_last_error("revo_op_depth_stats: bad argument");
    return REVO_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(scratch) % depth_stats_scratch_align()) {
    set_last_error("revo_op_depth_stats: scratch must be %zu-byte aligned", depth_stats_scratch_align());
    return REVO_EINVAL;
  }
  if (static_cast<long long>(height) * width > kDepthStatsMaxPixels) {
    set_last_error("revo_op_depth_stats: frame of %d x %d pixels exceeds the maximum of %lld pixels", height, width,
                   kDepthStatsMaxPixels);
    return REVO_EINVAL;
  }
  return cuda_status(
      launch_depth_stats(depth, height, width, pitch_bytes, mu_sigma, scratch, static_cast<cudaStream_t>(stream)),
      "revo_op_depth_stats");
}

revo_status revo_op_linear(revo_precision precision, int epilogue, const void* A, const void* W, const float* bias,
                           void* out, int M, int N, int K, int tile_n, void* stream) {
  if (!A || !W || !out || M < 0 || N <= 0 || K <= 0 || epilogue < 0 || epilogue > 3) {
    set_last_error("revo_op_linear: bad argument");
    return REVO_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == REVO_FP32) {
    if (K % 8) {
      set_last_error("revo_op_linear: FP32 path needs K %% 8 == 0");
      return REVO_EINVAL;
    }
    return cuda_status(launch_gemm_simt(epilogue, static_cast<const float*>(A), static_cast<const float*>(W), bias,
                                        out, N, M, N, K, st),
                       "revo_op_linear");
  }
  if (precision != REVO_BF16) {
    set_last_error("revo_op_linear: precision not supported by this entry point");
    return REVO_ENOTSUP;
  }
  const bool f32_out = epilogue == 0 || epilogue == 3;
  if (K % 64 || N % (f32_out ? 32 : 64)) {
    set_last_error("revo_op_linear: BF16 path needs K %% 64 == 0 and N %% 32 == 0 (N %% 64 == 0 for bf16 outputs)");
    return REVO_EINVAL;
  }
  const bool pair = (tile_n & REVO_TILE_PAIR) != 0;
  const int req = tile_n & ~REVO_TILE_PAIR;
  // 192: single tiles with float32 outputs only (other uses fall back to 128).
  const int width = req == 256 ? 256 : (req == 192 && f32_out && !pair) ? 192 : 128;
  const int bn = pair ? (width | kTilePair) : width;
  CUtensorMap ma, mb, mc;
  const uint64_t rows = M > 0 ? M : 1;
  if (!encode_tmap_bf16_2d(&ma, A, rows, K, K, 128, 64) ||
      !encode_tmap_bf16_2d(&mb, W, N, K, K, pair ? width / 2 : width, 64) ||
      !encode_tmap_out_2d(&mc, out, f32_out, rows, N, N)) {
    set_last_error("revo_op_linear: tensor map encoding failed (alignment?)");
    return REVO_EINVAL;
  }
  int* err = op_error_word();
  if (!err) {
    set_last_error("revo_op_linear: no device error word");
    return REVO_ECUDA;
  }
  return cuda_status(launch_gemm_tc(ma, mb, mc, bn, epilogue, bias, M, N, K, err, device_sm_count(), st),
                     "revo_op_linear");
}

revo_status revo_op_linear_pe(const void* A, const void* W, const float* bias, float* out, int slots, int grid_h,
                              int grid_w, int N, int K, const int* taus, int tile_n, void* stream) {
  if (!A || !W || !out || !taus || slots < 0 || slots > 8 || grid_h < 0 || grid_w < 0 || grid_h > 0xFFFF ||
      grid_w > 0xFFFF || N % 192 || N <= 0 || N > 1024 || K <= 0) {
    set_last_error("revo_op_linear_pe: bad argument");
    return REVO_EINVAL;
  }
  if (K % 64) {
    set_last_error("revo_op_linear_pe: needs K %% 64 == 0");
    return REVO_EINVAL;
  }
  const long long Mll = static_cast<long long>(slots) * grid_h * grid_w;
  if (Mll > (1LL << 30)) {
    set_last_error("revo_op_linear_pe: too many tokens");
    return REVO_EINVAL;
  }
  const int M = static_cast<int>(Mll);
  if (M == 0) return REVO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool pair = (tile_n & REVO_TILE_PAIR) != 0;
  const int req = tile_n & ~REVO_TILE_PAIR;
  const int width = req == 256 ? 256 : (req == 192 && !pair) ? 192 : 128;
  const int bn = pair ? (width | kTilePair) : width;
  CUtensorMap ma, mb, mc;
  if (!encode_tmap_bf16_2d(&ma, A, M, K, K, 128, 64) ||
      !encode_tmap_bf16_2d(&mb, W, N, K, K, pair ? width / 2 : width, 64) ||
      !encode_tmap_out_2d(&mc, out, true, M, N, N)) {
    set_last_error("revo_op_linear_pe: tensor map encoding failed (alignment?)");
    return REVO_EINVAL;
  }
  constexpr int kTabRows = 256;  // the table of revo_op_add_position
  int* err = op_error_word();
  auto* pos = static_cast<int2*>(op_scratch(kScratchPePositions, static_cast<size_t>(M) * sizeof(int2)));
  const float* tab = op_pe_table(N, kTabRows);
  const float* om = op_pe_omega(N);
  if (!err || !pos || !tab || !om) {
    set_last_error("revo_op_linear_pe: no device scratch");
    return REVO_ECUDA;
  }
  cudaError_t e = launch_pe_positions(pos, grid_h, grid_w, slots, taus, st);
  if (e != cudaSuccess) return cuda_status(e, "revo_op_linear_pe");
  EpiAux aux{};
  aux.pe_pos = pos;
  aux.pe_tab = tab;
  aux.pe_omega = om;
  aux.pe_rows = kTabRows;
  aux.pe_part = N / 3;
  return cuda_status(launch_gemm_tc(ma, mb, mc, bn, kEpiF32Pe, bias, M, N, K, err, device_sm_count(), st, &aux),
                     "revo_op_linear_pe");
}

revo_status revo_op_linear_resid_ln(const void* A, const void* W, const float* bias, float* x, int M, int N, int K,
                                    const float* gamma, const float* beta, void* ln_out, float* ln_row_scale,
                                    int ln_fp8, int tile_n, void* stream) {
  if (!A || !W || !x || !gamma || !beta || !ln_out || (ln_fp8 && !ln_row_scale) || M < 0 || N <= 0 || K <= 0) {
    set_last_error("revo_op_linear_resid_ln: bad argument");
    return REVO_EINVAL;
  }
  if (K % 64 || N % 32 || N > 1024 || (tile_n & ~REVO_TILE_PAIR) == 192) {
    set_last_error("revo_op_linear_resid_ln: needs K %% 64 == 0, N %% 32 == 0, N <= 1024 and a 128 or 256 tile");
    return REVO_EINVAL;
  }
  if (M == 0) return REVO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool pair = (tile_n & REVO_TILE_PAIR) != 0;
  const int width = (tile_n & ~REVO_TILE_PAIR) == 256 ? 256 : 128;
  const int bn = pair ? (width | kTilePair) : width;
  CUtensorMap ma, mb, mc;
  if (!encode_tmap_bf16_2d(&ma, A, M, K, K, 128, 64) ||
      !encode_tmap_bf16_2d(&mb, W, N, K, K, pair ? width / 2 : width, 64) ||
      !encode_tmap_out_2d(&mc, x, true, M, N, N)) {
    set_last_error("revo_op_linear_resid_ln: tensor map encoding failed (alignment?)");
    return REVO_EINVAL;
  }
  int* err = op_error_word();
  const size_t blocks = static_cast<size_t>(M + 127) / 128;
  int* counters = static_cast<int*>(op_scratch(kScratchLnCounters, blocks * sizeof(int)));
  if (!err || !counters) {
    set_last_error("revo_op_linear_resid_ln: no device scratch");
    return REVO_ECUDA;
  }
  cudaError_t e = cudaMemsetAsync(counters, 0, blocks * sizeof(int), st);
  if (e != cudaSuccess) return cuda_status(e, "revo_op_linear_resid_ln");
  EpiAux ln{};
  ln.x = x;
  ln.g = gamma;
  ln.b = beta;
  ln.out = ln_out;
  ln.row_scale = ln_row_scale;
  ln.counters = counters;
  ln.mode = ln_fp8 ? 2 : 1;
  return cuda_status(launch_gemm_tc(ma, mb, mc, bn, kEpiResidLn, bias, M, N, K, err, device_sm_count(), st, &ln),
                     "revo_op_linear_resid_ln");
}

revo_status revo_op_layernorm(const float* x, const float* gamma, const float* beta, void* out, int M, int D,
                              int out_bf16, void* stream) {
  if (!x || !gamma || !beta || !out || M < 0 || D <= 0) {
    set_last_error("revo_op_layernorm: bad argument");
    return REVO_EINVAL;
  }
  return cuda_status(launch_layernorm(x, gamma, beta, out, M, D, out_bf16, static_cast<cudaStream_t>(stream)),
                     "revo_op_layernorm");
}

revo_status revo_op_quantize_rows_e4m3(const float* x, int rows, int cols, uint8_t* q, float* scale, void* stream) {
  if (!x || !q || !scale || rows < 0 || cols <= 0 || cols % 4) {
    set_last_error("revo_op_quantize_rows_e4m3: bad argument (cols must be a positive multiple of 4)");
    return REVO_EINVAL;
  }
  return cuda_status(launch_quantize_rows_e4m3(x, rows, cols, q, scale, static_cast<cudaStream_t>(stream)),
                     "revo_op_quantize_rows_e4m3");
}

revo_status revo_op_layernorm_e4m3(const float* x, const float* gamma, const float* beta, uint8_t* out,
                                   float* row_scale, int M, int D, void* stream) {
  if (!x || !gamma || !beta || !out || !row_scale || M < 0 || D <= 0) {
    set_last_error("revo_op_layernorm_e4m3: bad argument");
    return REVO_EINVAL;
  }
  return cuda_status(launch_layernorm_e4m3(x, gamma, beta, out, row_scale, M, D, static_cast<cudaStream_t>(stream)),
                     "revo_op_layernorm_e4m3");
}

revo_status revo_op_linear_fp8(int epilogue, const uint8_t* A, const float* a_scale, const uint8_t* W,
                               const float* w_scale, const float* bias, void* out, int M, int N, int K, int tile_n,
                               void* stream) {
  if (!A || !a_scale || !W || !w_scale || !out || M < 0 || N <= 0 || K <= 0 ||
      (epilogue != kEpiBf16 && epilogue != kEpiGeluBf16)) {
    set_last_error("revo_op_linear_fp8: bad argument (epilogue must be 1 or 2)");
    return REVO_EINVAL;
  }
  if (K % 128 || N % 64) {
    set_last_error("revo_op_linear_fp8: needs K %% 128 == 0 and N %% 64 == 0");
    return REVO_EINVAL;
  }
  const bool pair = (tile_n & REVO_TILE_PAIR) != 0;
  const int width = (tile_n & ~REVO_TILE_PAIR) == 256 && N >= 256 ? 256 : 128;
  const int bn = pair ? (width | kTilePair) : width;
  CUtensorMap ma, mb, mc;
  const uint64_t rows = M > 0 ? M : 1;
  if (!encode_tmap_u8_2d(&ma, A, rows, K, K, 128) || !encode_tmap_u8_2d(&mb, W, N, K, K, pair ? width / 2 : width) ||
      !encode_tmap_out_2d(&mc, out, false, rows, N, N)) {
    set_last_error("revo_op_linear_fp8: tensor map encoding failed (alignment?)");
    return REVO_EINVAL;
  }
  int* err = op_error_word();
  if (!err) {
    set_last_error("revo_op_linear_fp8: no device error word");
    return REVO_ECUDA;
  }
  return cuda_status(launch_gemm_tc_fp8(ma, mb, mc, bn, epilogue, bias, a_scale, w_scale, M, N, K, err,
                                        device_sm_count(), static_cast<cudaStream_t>(stream)),
                     "revo_op_linear_fp8");
}

revo_status revo_fec_encode(int n, int r, size_t packet_bytes, const uint8_t* data, size_t data_pitch,
                            uint8_t* parity, size_t parity_pitch, void* stream) {
  if (!data || (r > 0 && !parity) || n < 1 || r < 0 || n + r > 256 || packet_bytes == 0 || packet_bytes % 4 ||
      data_pitch < packet_bytes || (r > 0 && parity_pitch < packet_bytes) || data_pitch % 4 || parity_pitch % 4) {
    set_last_error("revo_fec_encode: bad argument (1 <= n, n + r <= 256, packet_bytes and pitches multiples of 4)");
    return REVO_EINVAL;
  }
  return cuda_status(fec_encode(n, r, packet_bytes, data, data_pitch, parity, parity_pitch,
                                static_cast<cudaStream_t>(stream)),
                     "revo_fec_encode");
}

size_t revo_fec_decode_scratch_bytes(int n) { return fec_decode_scratch_bytes(n); }

revo_status revo_fec_decode(int n, int r, size_t packet_bytes, const int* present, const uint8_t* received,
                            size_t received_pitch, uint8_t* data_out, size_t out_pitch, void* scratch, void* stream) {
  if (!present || !received || !data_out || n < 1 || r < 0 || n + r > 256 || packet_bytes == 0 || packet_bytes % 4 ||
      received_pitch < packet_bytes || out_pitch < packet_bytes || received_pitch % 4 || out_pitch % 4) {
    set_last_error("revo_fec_decode: bad argument");
    return REVO_EINVAL;
  }
  std::vector<char> seen(static_cast<size_t>(n + r), 0);
  int missing = 0;
  for (int a = 0; a < n; ++a) {
    if (present[a] < 0 || present[a] >= n + r || seen[present[a]]) {
      set_last_error("revo_fec_decode: present[] must hold n distinct packet indices in [0, n + r)");
      return REVO_EINVAL;
    }
    seen[present[a]] = 1;
  }
  for (int d = 0; d < n; ++d) missing += !seen[d];
  if (missing > 0 && !scratch) {
    set_last_error("revo_fec_decode: scratch (revo_fec_decode_scratch_bytes(n) bytes) needed");
    return REVO_EINVAL;
  }
  return cuda_status(fec_decode(n, r, packet_bytes, present, received, received_pitch, data_out, out_pitch, scratch,
                                static_cast<cudaStream_t>(stream)),
                     "revo_fec_decode");
}

size_t revo_render_scratch_bytes(int out_h, int out_w) { return render_scratch_bytes(out_h, out_w); }

revo_status revo_render_rgbd(const uint8_t* rgb, int rgb_h, int rgb_w, size_t rgb_pitch, const uint16_t* depth, int h,
                             int w, size_t depth_pitch, const revo_intrinsics* src, const revo_pose* pose,
                             const revo_intrinsics* dst, int out_h, int out_w, int splat_radius, void* scratch,
                             uint8_t* out_rgb, size_t out_rgb_pitch, uint16_t* out_depth, size_t out_depth_pitch,
                             void* stream) {
  if (!rgb || !depth || !src || !pose || !dst || !scratch || !out_rgb || !out_depth || h <= 0 || w <= 0 ||
      rgb_h <= 0 || rgb_w <= 0 || out_h <= 0 || out_w <= 0 || splat_radius < 0 || splat_radius > 16 ||
      rgb_pitch < static_cast<size_t>(rgb_w) * 3 || depth_pitch < static_cast<size_t>(w) * 2 ||
      out_rgb_pitch < static_cast<size_t>(out_w) * 3 || out_depth_pitch < static_cast<size_t>(out_w) * 2 ||
      depth_pitch % 2 || out_depth_pitch % 2 || static_cast<long long>(h) * w > 0xFFFFFFFFll) {
    set_last_error("revo_render_rgbd: bad argument");
    return REVO_EINVAL;
  }
  RenderCall c{};
  c.rgb = rgb;
  c.rgb_pitch = rgb_pitch;
  c.rgb_h = rgb_h;
  c.rgb_w = rgb_w;
  c.depth = depth;
  c.depth_pitch = depth_pitch;
  c.h = h;
  c.w = w;
  c.src[0] = src->fx;
  c.src[1] = src->fy;
  c.src[2] = src->cx;
  c.src[3] = src->cy;
  for (int i = 0; i < 9; ++i) c.r[i] = pose->r[i];
  for (int i = 0; i < 3; ++i) c.t[i] = pose->t[i];
  c.dst[0] = dst->fx;
  c.dst[1] = dst->fy;
  c.dst[2] = dst->cx;
  c.dst[3] = dst->cy;
  c.out_h = out_h;
  c.out_w = out_w;
  c.splat = splat_radius;
  c.scratch = scratch;
  c.out_rgb = out_rgb;
  c.out_rgb_pitch = out_rgb_pitch;
  c.out_depth = out_depth;
  c.out_depth_pitch = out_depth_pitch;
  return cuda_status(launch_render(c, static_cast<cudaStream_t>(stream)), "revo_render_rgbd");
}

size_t revo_frame_metrics_scratch_bytes(int height, int width, int channels) {
  return frame_metrics_scratch_bytes(height, width, channels);
}

revo_status revo_op_frame_metrics(const void* a, size_t pitch_a, const void* b, size_t pitch_b, int height, int width,
                                  int channels, int sample_bytes, float data_range, void* scratch, float* out,
                                  void* stream) {
  if (!a || !b || !scratch || !out || height <= 10 || width <= 10 || (channels != 1 && channels != 3) ||
      (sample_bytes != 1 && sample_bytes != 2) || !(data_range > 0.f) ||
      pitch_a < static_cast<size_t>(width) * channels * sample_bytes ||
      pitch_b < static_cast<size_t>(width) * channels * sample_bytes) {
    set_last_error("revo_op_frame_metrics: bad argument");
    return REVO_EINVAL;
  }
  return cuda_status(launch_frame_metrics(a, pitch_a, b, pitch_b, height, width, channels, sample_bytes, data_range, out,
                                          scratch, static_cast<cudaStream_t>(stream)),
                     "revo_op_frame_metrics");
}

revo_status revo_op_attention(revo_precision precision, const void* qkv, void* out, int M, int D, int heads,
                              const int* seg_start, const int* q_begin, const int* q_end, int n_seg, int flags,
                              void* stream) {
  if (!qkv || !out || !seg_start || n_seg <= 0 || n_seg > kMaxSegments || heads <= 0 || D != 64 * heads) {
    set_last_error("revo_op_attention: bad argument (head width must be 64, n_seg <= 64)");
    return REVO_EINVAL;
  }
  Segments seg{};
  seg.n = n_seg;
  for (int i = 0; i <= n_seg; ++i) {
    seg.start[i] = seg_start[i];
    if (seg.start[i] < 0 || seg.start[i] > M || (i && seg.start[i] < seg.start[i - 1])) {
      set_last_error("revo_op_attention: segment bounds not increasing within [0, M]");
      return REVO_EINVAL;
    }
  }
  if ((q_begin != nullptr) != (q_end != nullptr)) {
    set_last_error("revo_op_attention: q_begin and q_end go together");
    return REVO_EINVAL;
  }
  if (q_begin) {
    seg.queries = true;
    for (int i = 0; i < n_seg; ++i) {
      seg.q_begin[i] = q_begin[i];
      seg.q_end[i] = q_end[i];
      if (q_begin[i] < seg.start[i] || q_end[i] > seg.start[i + 1] || q_end[i] < q_begin[i]) {
        set_last_error("revo_op_attention: query rows outside their segment");
        return REVO_EINVAL;
      }
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == REVO_FP32)
    return cuda_status(
        launch_attention_simt(static_cast<const float*>(qkv), static_cast<float*>(out), M, D, heads, seg, st),
        "revo_op_attention");
  if (precision != REVO_BF16) {
    set_last_error("revo_op_attention: precision not supported");
    return REVO_ENOTSUP;
  }
  CUtensorMap m;
  if (!encode_attention_tmap(&m, qkv, M > 0 ? M : 1, D)) {
    set_last_error("revo_op_attention: tensor map encoding failed");
    return REVO_EINVAL;
  }
  int* err = op_error_word();
  if (!err) return REVO_ECUDA;
  float* part = nullptr;
  if (flags & REVO_ATTN_SPLIT_TAIL) {
    const size_t need = attention_partial_bytes(M, heads, seg, device_sm_count());
    if (!(part = static_cast<float*>(op_scratch(kScratchAttnPartial, need)))) {
      set_last_error("revo_op_attention: partial-result buffer allocation failed");
      return REVO_ENOMEM;
    }
  }
  return cuda_status(launch_attention_tc(m, out, M, D, heads, seg, err, st, part, device_sm_count()),
                     "revo_op_attention");
}

revo_status revo_op_add_position(float* x, int slots, int grid_h, int grid_w, int D, const int* taus, void* stream) {
  if (!x || !taus || slots < 0 || slots > 8 || grid_h < 0 || grid_w < 0 || D % 192 || D > 1024) {
    set_last_error("revo_op_add_position: bad argument");
    return REVO_EINVAL;
  }
  // Up to 256 patch rows and columns the row and column parts come from a
  // table (as in the recovery forward); larger grids compute them per element
  // (the same values).
  constexpr int kTabRows = 256;
  const float* tab = nullptr;
  if (grid_w <= kTabRows && grid_h <= kTabRows) {
    float* t = op_pe_table(D, kTabRows);
    if (!t) {
      set_last_error("revo_op_add_position: table allocation failed");
      return REVO_ENOMEM;
    }
    tab = t;
  }
  return cuda_status(launch_add_pe(x, grid_h, grid_w, slots, taus, D, static_cast<cudaStream_t>(stream), nullptr, tab,
                                   kTabRows),
                     "revo_op_add_position");
}

revo_status revo_op_blend(int channels, int p, int height, int width, const float* head, const void* decoded,
                          size_t pitch_bytes, const uint32_t* mask, size_t mask_pitch_words, const float* mu_sigma,
                          void* out, size_t out_pitch, float* values, void* stream) {
  if (!head || !decoded || !mask || !out || (channels == 1 && !mu_sigma) ||
      mask_pitch_words < static_cast<size_t>((width + 31) / 32)) {
    set_last_error("revo_op_blend: bad argument");
    return REVO_EINVAL;
  }
  BlendArgs a{};
  a.C = channels;
  a.p = p;
  a.H = height;
  a.W = width;
  a.head = head;
  a.decoded = decoded;
  a.pitch = pitch_bytes;
  a.mask = mask;
  a.mask_pitch = mask_pitch_words;
  a.mu_sigma = mu_sigma;
  a.out = out;
  a.out_pitch = out_pitch;
  a.values = values;
  return cuda_status(launch_blend(a, static_cast<cudaStream_t>(stream)), "revo_op_blend");
}

}  // extern "C"

revo_status revo_op_assemble_batch(int channels, int k, int T, int n, const revo_assemble_job* jobs, int out_bf16,
                                   void* stream) {
  if (!jobs || n <= 0 || n > kMaxSegments || k < 1 || k > kMaxRefs || (channels != 1 && channels != 3)) {
    set_last_error("revo_op_assemble_batch: bad argument");
    return REVO_EINVAL;
  }
  std::vector<AssembleArgs> a(n);
  for (int i = 0; i < n; ++i) {
    const revo_assemble_job& j = jobs[i];
    if (!j.out || (channels == 1 && !j.mu_sigma)) {
      set_last_error("revo_op_assemble_batch: bad job %d", i);
      return REVO_EINVAL;
    }
    a[i] = AssembleArgs{};
    for (int f = 0; f <= k; ++f) {
      if (!j.frames[f]) {
        set_last_error("revo_op_assemble_batch: job %d lacks frame %d", i, f);
        return REVO_EINVAL;
      }
      a[i].frames[f] = j.frames[f];
      a[i].pitch[f] = j.pitch_bytes;
    }
    a[i].mu_sigma = j.mu_sigma;
    a[i].out = j.out;
    a[i].C = channels;
    a[i].F = k + 1;
    a[i].T = T;
    a[i].p = 16;
    a[i].H = j.height;
    a[i].W = j.width;
    a[i].out_bf16 = out_bf16;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* dev = op_arg_table(a.data(), n * sizeof(AssembleArgs), st);
  if (!dev) {
    set_last_error("revo_op_assemble_batch: argument table allocation or upload failed");
    return REVO_ENOMEM;
  }
  return cuda_status(launch_assemble_batch(a.data(), n, static_cast<const AssembleArgs*>(dev), sizeof(AssembleArgs), st),
                     "revo_op_assemble_batch");
}

revo_status revo_op_embed_batch(int channels, int k, int T, int n, const revo_assemble_job* jobs, const int* taus,
                                const void* W, const float* bias, float* out, int N, void* stream) {
  if (!jobs || !taus || !W || !out || n <= 0 || n > kMaxSegments || k < 1 || k > kMaxRefs ||
      (channels != 1 && channels != 3) || T < 1 || T > 2 || (k + 1) % T != 0 || N <= 0 || N % 192 || N > 1024) {
    set_last_error("revo_op_embed_batch: bad argument");
    return REVO_EINVAL;
  }
  const int slots = (k + 1) / T;
  if (slots > 8) {
    set_last_error("revo_op_embed_batch: more than 8 slots");
    return REVO_EINVAL;
  }
  std::vector<AssembleArgs> a(n);
  EmbedParams ep{};
  ep.n = n;
  ep.C = channels;
  ep.T = T;
  long long M = 0;
  for (int i = 0; i < n; ++i) {
    const revo_assemble_job& j = jobs[i];
    if (j.height <= 0 || j.width <= 0 || j.height % 16 || j.width % 16 || j.height / 16 > 0xFFFF ||
        j.width / 16 > 0xFFFF || (channels == 1 && !j.mu_sigma)) {
      set_last_error("revo_op_embed_batch: bad job %d", i);
      return REVO_EINVAL;
    }
    a[i] = AssembleArgs{};
    for (int f = 0; f <= k; ++f) {
      if (!j.frames[f]) {
        set_last_error("revo_op_embed_batch: job %d lacks frame %d", i, f);
        return REVO_EINVAL;
      }
      a[i].frames[f] = j.frames[f];
      a[i].pitch[f] = j.pitch_bytes;
    }
    a[i].mu_sigma = j.mu_sigma;
    a[i].C = channels;
    a[i].F = k + 1;
    a[i].T = T;
    a[i].p = 16;
    a[i].H = j.height;
    a[i].W = j.width;
    a[i].out_bf16 = 1;
    for (int s = 0; s < slots; ++s) a[i].taus[s] = taus[i * 8 + s];
    ep.seg_start[i] = static_cast<int>(M);
    ep.hp[i] = j.height / 16;
    ep.wp[i] = j.width / 16;
    M += static_cast<long long>(slots) * ep.hp[i] * ep.wp[i];
    if (M > (1LL << 30)) {
      set_last_error("revo_op_embed_batch: too many tokens");
      return REVO_EINVAL;
    }
  }
  ep.seg_start[n] = static_cast<int>(M);
  const int K = T * channels * 256;
  const int bn = N % 256 == 0 ? 256 : 128;
  CUtensorMap mb, mc;
  if (!encode_tmap_bf16_2d(&mb, W, N, K, K, bn, 64) || !encode_tmap_out_2d(&mc, out, true, M, N, N)) {
    set_last_error("revo_op_embed_batch: tensor map encoding failed (alignment?)");
    return REVO_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  constexpr int kTabRows = 256;  // the table of revo_op_add_position
  int* err = op_error_word();
  auto* pos = static_cast<int2*>(op_scratch(kScratchPePositions, static_cast<size_t>(M) * sizeof(int2)));
  const float* tab = op_pe_table(N, kTabRows);
  const float* om = op_pe_omega(N);
  void* dev = op_arg_table(a.data(), n * sizeof(AssembleArgs), st);
  if (!err || !pos || !tab || !om || !dev) {
    set_last_error("revo_op_embed_batch: no device scratch");
    return REVO_ECUDA;
  }
  ep.jobs = static_cast<const uint8_t*>(dev);
  ep.stride = sizeof(AssembleArgs);
  ep.pe_pos = pos;
  EpiAux aux{};
  aux.pe_tab = tab;
  aux.pe_omega = om;
  aux.pe_rows = kTabRows;
  aux.pe_part = N / 3;
  return cuda_status(launch_embed_tc(mb, mc, bn, bias, static_cast<int>(M), N, K, err, device_sm_count(), st, aux, ep),
                     "revo_op_embed_batch");
}

revo_status revo_op_blend_batch(int channels, int n, const revo_blend_job* jobs, void* stream) {
  if (!jobs || n <= 0 || n > kMaxSegments || (channels != 1 && channels != 3)) {
    set_last_error("revo_op_blend_batch: bad argument");
    return REVO_EINVAL;
  }
  std::vector<BlendArgs> a(n);
  for (int i = 0; i < n; ++i) {
    const revo_blend_job& j = jobs[i];
    if (!j.head || !j.decoded || !j.mask || !j.out || (channels == 1 && !j.mu_sigma) ||
        j.mask_pitch_words < static_cast<size_t>((j.width + 31) / 32)) {
      set_last_error("revo_op_blend_batch: bad job %d", i);
      return REVO_EINVAL;
    }
    a[i] = BlendArgs{channels, 16, j.height, j.width, j.head, j.decoded, j.pitch_bytes, j.mask, j.mask_pitch_words,
                     j.mu_sigma, j.out, j.out_pitch, j.values};
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* dev = op_arg_table(a.data(), n * sizeof(BlendArgs), st);
  if (!dev) {
    set_last_error("revo_op_blend_batch: argument table allocation or upload failed");
    return REVO_ENOMEM;
  }
  return cuda_status(launch_blend_batch(a.data(), n, static_cast<const BlendArgs*>(dev), sizeof(BlendArgs), st),
                     "revo_op_blend_batch");
}
