// RGB-D unprojection and point splatting: the receiver renders a recovered
// RGB-D frame from the viewer's pose (the pipeline's rendering step; an
// RGB-D frame is a 2-D projection of the scene, Section 2).  No graphics API:
// two CUDA passes over a 64-bit z-buffer.
//
//   pass 1, one thread per depth sample: unproject with the source pinhole
//     (x = (u - cx) d / fx, y = (v - cy) d / fy, z = d at pixel centre u = i,
//     v = j), move by x' = R x + t, project with the target pinhole, round the
//     pixel half to even, and for each pixel of the (2s+1)^2 splat take the
//     64-bit minimum of (float bits of z') << 32 | point index: the nearest
//     point wins, ties go to the lower index, independent of thread order.
//   pass 2, one thread per output pixel: resolve the winner's colour (nearest
//     RGB sample when the frames differ in size) and depth (z' rounded half to
//     even, clamped to uint16); empty pixels get 0.
// Every float step is a separately rounded IEEE operation in a fixed order
// (no contraction into FMA), so the result is reproducible bit for bit.
#include <math.h>

#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

struct RenderArgs {
  const uint8_t* rgb;
  size_t rgb_pitch;
  int rgb_h, rgb_w;
  const uint16_t* depth;
  size_t depth_pitch;
  int h, w;
  float fx, fy, cx, cy;     // source
  float r[9], t[3];         // x' = R x + t
  float fx2, fy2, cx2, cy2;  // target
  int out_h, out_w, splat;
  unsigned long long* zbuf;  // [out_h * out_w]
  uint8_t* out_rgb;
  size_t out_rgb_pitch;
  uint16_t* out_depth;
  size_t out_depth_pitch;
};

__global__ void splat_kernel(const __grid_constant__ RenderArgs a) {
  const long long n = static_cast<long long>(a.h) * a.w;
  const long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (p >= n) return;
  const int j = static_cast<int>(p / a.w), i = static_cast<int>(p % a.w);
  const uint16_t draw = reinterpret_cast<const uint16_t*>(reinterpret_cast<const uint8_t*>(a.depth) +
                                                          static_cast<size_t>(j) * a.depth_pitch)[i];
  if (draw == 0) return;
  const float d = static_cast<float>(draw);
  const float x = __fdiv_rn(__fmul_rn(__fsub_rn(static_cast<float>(i), a.cx), d), a.fx);
  const float y = __fdiv_rn(__fmul_rn(__fsub_rn(static_cast<float>(j), a.cy), d), a.fy);
  const float z = d;
  const float X = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.r[0], x), __fmul_rn(a.r[1], y)), __fmul_rn(a.r[2], z)), a.t[0]);
  const float Y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.r[3], x), __fmul_rn(a.r[4], y)), __fmul_rn(a.r[5], z)), a.t[1]);
  const float Z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.r[6], x), __fmul_rn(a.r[7], y)), __fmul_rn(a.r[8], z)), a.t[2]);
  if (!(Z > 0.f)) return;
  const float u = __fadd_rn(__fdiv_rn(__fmul_rn(a.fx2, X), Z), a.cx2);
  const float v = __fadd_rn(__fdiv_rn(__fmul_rn(a.fy2, Y), Z), a.cy2);
  if (!(fabsf(u) < 1e9f) || !(fabsf(v) < 1e9f)) return;  // also drops NaN / inf
  const int pu = static_cast<int>(rintf(u)), pv = static_cast<int>(rintf(v));
  const unsigned long long key =
      (static_cast<unsigned long long>(__float_as_uint(Z)) << 32) | static_cast<unsigned long long>(p);
  for (int dv = -a.splat; dv <= a.splat; ++dv) {
    const int row = pv + dv;
    if (row < 0 || row >= a.out_h) continue;
    for (int du = -a.splat; du <= a.splat; ++du) {
      const int col = pu + du;
      if (col < 0 || col >= a.out_w) continue;
      atomicMin(a.zbuf + static_cast<size_t>(row) * a.out_w + col, key);
    }
  }
}

__global__ void resolve_kernel(const __grid_constant__ RenderArgs a) {
  const long long n = static_cast<long long>(a.out_h) * a.out_w;
  const long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (q >= n) return;
  const int row = static_cast<int>(q / a.out_w), col = static_cast<int>(q % a.out_w);
  const unsigned long long key = a.zbuf[q];
  uint8_t* orgb = a.out_rgb + static_cast<size_t>(row) * a.out_rgb_pitch + col * 3;
  uint16_t* od = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(a.out_depth) +
                                             static_cast<size_t>(row) * a.out_depth_pitch) + col;
  if (key == ~0ull) {
    orgb[0] = orgb[1] = orgb[2] = 0;
    *od = 0;
    return;
  }
  const long long p = static_cast<long long>(key & 0xFFFFFFFFull);
  const int j = static_cast<int>(p / a.w), i = static_cast<int>(p % a.w);
  const int rj = static_cast<int>((static_cast<long long>(j) * a.rgb_h) / a.h);
  const int ri = static_cast<int>((static_cast<long long>(i) * a.rgb_w) / a.w);
  const uint8_t* src = a.rgb + static_cast<size_t>(rj) * a.rgb_pitch + ri * 3;
  orgb[0] = src[0];
  orgb[1] = src[1];
  orgb[2] = src[2];
  const float Z = __uint_as_float(static_cast<uint32_t>(key >> 32));
  *od = static_cast<uint16_t>(fminf(rintf(Z), 65535.f));
}

}  // namespace

size_t render_scratch_bytes(int out_h, int out_w) {
  return out_h > 0 && out_w > 0 ? static_cast<size_t>(out_h) * out_w * 8 : 0;
}

cudaError_t launch_render(const RenderCall& c, cudaStream_t st) {
  if (c.h <= 0 || c.w <= 0 || c.rgb_h <= 0 || c.rgb_w <= 0 || c.out_h <= 0 || c.out_w <= 0 || c.splat < 0 ||
      c.splat > 16 || static_cast<long long>(c.h) * c.w > 0xFFFFFFFFll)
    return cudaErrorInvalidValue;
  RenderArgs a{};
  a.rgb = c.rgb;
  a.rgb_pitch = c.rgb_pitch;
  a.rgb_h = c.rgb_h;
  a.rgb_w = c.rgb_w;
  a.depth = c.depth;
  a.depth_pitch = c.depth_pitch;
  a.h = c.h;
  a.w = c.w;
  a.fx = c.src[0];
  a.fy = c.src[1];
  a.cx = c.src[2];
  a.cy = c.src[3];
  for (int i = 0; i < 9; ++i) a.r[i] = c.r[i];
  for (int i = 0; i < 3; ++i) a.t[i] = c.t[i];
  a.fx2 = c.dst[0];
  a.fy2 = c.dst[1];
  a.cx2 = c.dst[2];
  a.cy2 = c.dst[3];
  a.out_h = c.out_h;
  a.out_w = c.out_w;
  a.splat = c.splat;
  a.zbuf = static_cast<unsigned long long*>(c.scratch);
  a.out_rgb = c.out_rgb;
  a.out_rgb_pitch = c.out_rgb_pitch;
  a.out_depth = c.out_depth;
  a.out_depth_pitch = c.out_depth_pitch;
  cudaError_t e = cudaMemsetAsync(c.scratch, 0xFF, render_scratch_bytes(c.out_h, c.out_w), st);
  if (e != cudaSuccess) return e;
  const long long n = static_cast<long long>(c.h) * c.w, m = static_cast<long long>(c.out_h) * c.out_w;
  splat_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(a);
  resolve_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace revo
