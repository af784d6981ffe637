// One LayerNorm row (eps 1e-6, biased variance, two passes in registers) by
// one warp, shared by the standalone LayerNorm kernel and the residual GEMM
// epilogue that fuses it: both evaluate exactly the same float32 operations
// in the same order, so a fused and a separate LayerNorm agree bit for bit.
#pragma once

#include <cuda_fp8.h>

#include "common.cuh"

namespace revo {

constexpr int kLnMaxVec = 8;  // D <= 1024

// Four floats -> four E4M3 codes (round to nearest even, saturating to +-448),
// the first value in the lowest byte.
REVO_DEVI uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

// Per-row E4M3 scale rule: s = amax / 448, inverse 448 / amax; an all-zero row
// keeps s = 1.
REVO_DEVI void e4m3_row_scale(float amax, float* s, float* inv) {
  if (amax > 0.f) {
    *s = amax / 448.0f;
    *inv = 448.0f / amax;
  } else {
    *s = 1.0f;
    *inv = 1.0f;
  }
}

// Rows row0, row0 + stride, ... (R of them, those below row_end) of x [.][D]
// -> out: OUT 0 float32, 1 bf16, 2 E4M3 codes with row_scale[row].  Each lane
// holds up to NV float4 of a row (D <= 128 NV); the R rows' loads are issued
// together so that R rows are in flight per warp.  COHERENT: read x through L2
// only (x was written by other CTAs of the running kernel), else through the
// read-only path.  The arithmetic of a row does not depend on NV or R.
template <int OUT, bool COHERENT, int NV, int R>
REVO_DEVI void ln_rows(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ b,
                       void* __restrict__ out, float* __restrict__ row_scale, int row0, int stride, int row_end,
                       int D, int lane) {
  const int nv = D / 4;
  float4 v[R][NV];
  float mean[R], rstd[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int row = row0 + j * stride;
    if (row < row_end) {
      const float4* xr = reinterpret_cast<const float4*>(x + static_cast<size_t>(row) * D);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int c = lane + 32 * i;
        if (c < nv) v[j][i] = COHERENT ? __ldcg(xr + c) : __ldg(xr + c);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int c = lane + 32 * i;
      if (c < nv && row0 + j * stride < row_end) sum += (v[j][i].x + v[j][i].y) + (v[j][i].z + v[j][i].w);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    mean[j] = sum / D;
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    float sq = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int c = lane + 32 * i;
      if (c < nv && row0 + j * stride < row_end) {
        const float a0 = v[j][i].x - mean[j], a1 = v[j][i].y - mean[j], a2 = v[j][i].z - mean[j],
                    a3 = v[j][i].w - mean[j];
        sq += (a0 * a0 + a1 * a1) + (a2 * a2 + a3 * a3);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    rstd[j] = 1.0f / sqrtf(sq / D + 1e-6f);
  }
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int row = row0 + j * stride;
    if (row >= row_end) break;  // the same in every lane
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int c = lane + 32 * i;
      if (c < nv) {
        const float4 gg = __ldg(g4 + c), bb = __ldg(b4 + c);
        const float y0 = (v[j][i].x - mean[j]) * rstd[j] * gg.x + bb.x;
        const float y1 = (v[j][i].y - mean[j]) * rstd[j] * gg.y + bb.y;
        const float y2 = (v[j][i].z - mean[j]) * rstd[j] * gg.z + bb.z;
        const float y3 = (v[j][i].w - mean[j]) * rstd[j] * gg.w + bb.w;
        if (OUT == 2) {
          v[j][i] = make_float4(y0, y1, y2, y3);
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(y0), fabsf(y1)), fmaxf(fabsf(y2), fabsf(y3))));
        } else if (OUT == 1) {
          uint2* o = reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(out) + static_cast<size_t>(row) * D) + c;
          *o = make_uint2(pack_bf16x2(y0, y1), pack_bf16x2(y2, y3));
        } else {
          float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + static_cast<size_t>(row) * D) + c;
          *o = make_float4(y0, y1, y2, y3);
        }
      }
    }
    if (OUT == 2) {
#pragma unroll
      for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      float sc, inv;
      e4m3_row_scale(amax, &sc, &inv);
      uint32_t* orow = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(out) + static_cast<size_t>(row) * D);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int c = lane + 32 * i;
        if (c < nv) orow[c] = pack_e4m3x4(v[j][i].x * inv, v[j][i].y * inv, v[j][i].z * inv, v[j][i].w * inv);
      }
      if (lane == 0) row_scale[row] = sc;
    }
  }
}

// One row, any D <= 1024.
template <int OUT, bool COHERENT>
REVO_DEVI void ln_row(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ b,
                      void* __restrict__ out, float* __restrict__ row_scale, int row, int D, int lane) {
  ln_rows<OUT, COHERENT, kLnMaxVec, 1>(x, g, b, out, row_scale, row, 0, row + 1, D, lane);
}

}  // namespace revo
