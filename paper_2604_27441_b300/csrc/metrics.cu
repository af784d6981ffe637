// Frame-quality metrics the paper evaluates recovered frames with (Section 5,
// Metrics): SSIM and PSNR of a frame against its original.  Both are
// HBM-bound passes over two frames.
//
// SSIM: local means, variances and covariance under a normalised 11 x 11
// Gaussian window (sigma 1.5, separable), C1 = (0.01 L)^2, C2 = (0.03 L)^2, the
// SSIM map over the positions where the window lies inside the frame, averaged
// per channel and over channels.  One CTA computes a 32 x 32 tile of the map
// for one channel: the 42 x 42 input tile of both frames goes to shared
// memory, a horizontal pass filters the five products (x, y, x^2, y^2, xy)
// into shared memory, a vertical pass gives each output; the second moments
// are taken about the tile's first sample (variances and covariance do not
// depend on the offset; it keeps float32 sums of squares well conditioned for
// uint16 depth).  Each CTA writes its partial sum; a one-block pass adds them
// in a fixed order in double precision, so the result is deterministic.
//
// PSNR: a grid-stride sum of squared differences over every sample, per-CTA
// partials, the same fixed-order final pass.
#include <math.h>

#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kWin = 11;
constexpr int kHalo = kWin - 1;
constexpr int kTile = 32;
constexpr int kIn = kTile + kHalo;  // 42
constexpr int kSsimThreads = 256;
constexpr int kPsnrBlocks = 296;
constexpr int kPsnrThreads = 256;

struct SsimArgs {
  const uint8_t* a;
  const uint8_t* b;
  size_t pitch_a, pitch_b;
  int H, W, C, sample_bytes;
  float c1, c2;
  float g[kWin];
  float* partial;  // [tiles_x * tiles_y * C]
};

REVO_DEVI float load_sample(const uint8_t* base, size_t pitch, int row, int col, int C, int c, int sb) {
  const uint8_t* p = base + static_cast<size_t>(row) * pitch;
  if (sb == 1) return static_cast<float>(p[col * C + c]);
  return static_cast<float>(reinterpret_cast<const uint16_t*>(p)[col * C + c]);
}

__global__ void __launch_bounds__(kSsimThreads) ssim_tile_kernel(const __grid_constant__ SsimArgs a) {
  __shared__ float sx[kIn][kIn + 1], sy[kIn][kIn + 1];
  __shared__ float hx[kIn][kTile], hy[kIn][kTile], hxx[kIn][kTile], hyy[kIn][kTile], hxy[kIn][kTile];
  __shared__ float red[kSsimThreads / 32];
  const int c = blockIdx.z;
  const int oy0 = blockIdx.y * kTile, ox0 = blockIdx.x * kTile;  // output (valid-map) origin = input origin
  const int Hv = a.H - kHalo, Wv = a.W - kHalo;
  const float base = load_sample(a.a, a.pitch_a, oy0, ox0, a.C, c, a.sample_bytes);
  for (int i = threadIdx.x; i < kIn * kIn; i += kSsimThreads) {
    const int r = i / kIn, q = i % kIn;
    const int row = oy0 + r, col = ox0 + q;
    float vx = 0.f, vy = 0.f;
    if (row < a.H && col < a.W) {
      vx = load_sample(a.a, a.pitch_a, row, col, a.C, c, a.sample_bytes) - base;
      vy = load_sample(a.b, a.pitch_b, row, col, a.C, c, a.sample_bytes) - base;
    }
    sx[r][q] = vx;
    sy[r][q] = vy;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kIn * kTile; i += kSsimThreads) {
    const int r = i / kTile, q = i % kTile;
    float m1 = 0.f, m2 = 0.f, m11 = 0.f, m22 = 0.f, m12 = 0.f;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const float w = a.g[k], x = sx[r][q + k], y = sy[r][q + k];
      m1 = fmaf(w, x, m1);
      m2 = fmaf(w, y, m2);
      m11 = fmaf(w * x, x, m11);
      m22 = fmaf(w * y, y, m22);
      m12 = fmaf(w * x, y, m12);
    }
    hx[r][q] = m1;
    hy[r][q] = m2;
    hxx[r][q] = m11;
    hyy[r][q] = m22;
    hxy[r][q] = m12;
  }
  __syncthreads();
  float acc = 0.f;
  for (int i = threadIdx.x; i < kTile * kTile; i += kSsimThreads) {
    const int r = i / kTile, q = i % kTile;
    if (oy0 + r >= Hv || ox0 + q >= Wv) continue;
    float m1 = 0.f, m2 = 0.f, m11 = 0.f, m22 = 0.f, m12 = 0.f;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const float w = a.g[k];
      m1 = fmaf(w, hx[r + k][q], m1);
      m2 = fmaf(w, hy[r + k][q], m2);
      m11 = fmaf(w, hxx[r + k][q], m11);
      m22 = fmaf(w, hyy[r + k][q], m22);
      m12 = fmaf(w, hxy[r + k][q], m12);
    }
    const float vx = m11 - m1 * m1, vy = m22 - m2 * m2, cxy = m12 - m1 * m2;
    const float mx = m1 + base, my = m2 + base;
    const float num = (2.f * mx * my + a.c1) * (2.f * cxy + a.c2);
    const float den = (mx * mx + my * my + a.c1) * (vx + vy + a.c2);
    acc += num / den;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < kSsimThreads / 32; ++w) s += red[w];
    a.partial[(static_cast<size_t>(c) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void psnr_partial_kernel(const uint8_t* __restrict__ pa, const uint8_t* __restrict__ pb, size_t pitch_a,
                                    size_t pitch_b, int H, int rowlen, int sb, float* __restrict__ partial) {
  __shared__ float red[kPsnrThreads / 32];
  const long long total = static_cast<long long>(H) * rowlen;
  float acc = 0.f;
  for (long long i = blockIdx.x * static_cast<long long>(kPsnrThreads) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * kPsnrThreads) {
    const int r = static_cast<int>(i / rowlen), q = static_cast<int>(i % rowlen);
    float d;
    if (sb == 1)
      d = static_cast<float>(pa[r * pitch_a + q]) - static_cast<float>(pb[r * pitch_b + q]);
    else
      d = static_cast<float>(reinterpret_cast<const uint16_t*>(pa + r * pitch_a)[q]) -
          static_cast<float>(reinterpret_cast<const uint16_t*>(pb + r * pitch_b)[q]);
    acc = fmaf(d, d, acc);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < kPsnrThreads / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

// out[0] = mean SSIM over channels, out[1] = MSE, out[2] = PSNR (dB); one warp,
// fixed summation order (lane-strided partial sums, then lane 0 in order).
__global__ void metrics_final_kernel(const float* __restrict__ ssim_part, int tiles_per_channel, int C, double ssim_count,
                                     const float* __restrict__ mse_part, int mse_parts, double samples, float peak,
                                     float* __restrict__ out) {
  __shared__ double sh[32];
  const int lane = threadIdx.x;
  double s_all = 0.0;
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int i = lane; i < tiles_per_channel; i += 32) s += ssim_part[static_cast<size_t>(c) * tiles_per_channel + i];
    sh[lane] = s;
    __syncwarp();
    if (lane == 0) {
      double t = 0.0;
      for (int i = 0; i < 32; ++i) t += sh[i];
      s_all += t / ssim_count;
    }
    __syncwarp();
  }
  double m = 0.0;
  for (int i = lane; i < mse_parts; i += 32) m += mse_part[i];
  sh[lane] = m;
  __syncwarp();
  if (lane == 0) {
    double t = 0.0;
    for (int i = 0; i < 32; ++i) t += sh[i];
    const double mse = t / samples;
    out[0] = static_cast<float>(s_all / C);
    out[1] = static_cast<float>(mse);
    out[2] = mse > 0.0 ? static_cast<float>(10.0 * log10(static_cast<double>(peak) * peak / mse)) : INFINITY;
  }
}

}  // namespace

size_t frame_metrics_scratch_bytes(int H, int W, int C) {
  if (H <= kHalo || W <= kHalo || C <= 0) return 0;
  const size_t tiles = static_cast<size_t>((W - kHalo + kTile - 1) / kTile) * ((H - kHalo + kTile - 1) / kTile);
  return (tiles * C + kPsnrBlocks) * sizeof(float);
}

cudaError_t launch_frame_metrics(const void* a, size_t pitch_a, const void* b, size_t pitch_b, int H, int W, int C,
                                 int sample_bytes, float data_range, float* out, void* scratch, cudaStream_t st) {
  if (H <= kHalo || W <= kHalo || (C != 1 && C != 3) || (sample_bytes != 1 && sample_bytes != 2) ||
      !(data_range > 0.f))
    return cudaErrorInvalidValue;
  SsimArgs s{};
  s.a = static_cast<const uint8_t*>(a);
  s.b = static_cast<const uint8_t*>(b);
  s.pitch_a = pitch_a;
  s.pitch_b = pitch_b;
  s.H = H;
  s.W = W;
  s.C = C;
  s.sample_bytes = sample_bytes;
  s.c1 = static_cast<float>((0.01 * data_range) * (0.01 * data_range));
  s.c2 = static_cast<float>((0.03 * data_range) * (0.03 * data_range));
  double g[kWin], gs = 0.0;
  for (int i = 0; i < kWin; ++i) {
    const double x = i - (kWin - 1) / 2.0;
    g[i] = exp(-(x * x) / (2.0 * 1.5 * 1.5));
    gs += g[i];
  }
  for (int i = 0; i < kWin; ++i) s.g[i] = static_cast<float>(g[i] / gs);
  const int Hv = H - kHalo, Wv = W - kHalo;
  const dim3 grid((Wv + kTile - 1) / kTile, (Hv + kTile - 1) / kTile, C);
  s.partial = static_cast<float*>(scratch);
  float* mse_part = s.partial + static_cast<size_t>(grid.x) * grid.y * C;
  ssim_tile_kernel<<<grid, kSsimThreads, 0, st>>>(s);
  psnr_partial_kernel<<<kPsnrBlocks, kPsnrThreads, 0, st>>>(s.a, s.b, pitch_a, pitch_b, H, W * C, sample_bytes,
                                                            mse_part);
  metrics_final_kernel<<<1, 32, 0, st>>>(s.partial, grid.x * grid.y, C, static_cast<double>(Hv) * Wv, mse_part,
                                         kPsnrBlocks, static_cast<double>(H) * W * C, data_range, out);
  return cudaGetLastError();
}

}  // namespace revo
