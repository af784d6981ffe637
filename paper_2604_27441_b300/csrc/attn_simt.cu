// FP32 multi-head softmax attention on the CUDA cores (the full-precision path).
// Exact scaled dot-product attention (Appendix B.1, point 4) computed
// flash-style: one CTA owns 64 queries of one head of one segment, streams the
// segment's keys/values in tiles of 64 and keeps a running max / sum (online
// softmax), so the N x N score matrix is never stored.  Head width 64.
#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kBQ = 64;
constexpr int kBKV = 64;
constexpr int kHD = 64;

struct SimtAttnParams {
  int n_seg;
  int start[kMaxSegments + 1];
  int tile_prefix[kMaxSegments + 1];
};

constexpr int kSmemFloats = kHD * kBQ + kHD * kBKV + kBKV * kHD + kBQ * (kBKV + 1) + 3 * kBQ;

__global__ void __launch_bounds__(256) attn_simt_kernel(const float* __restrict__ qkv, float* __restrict__ out, int D,
                                                        const __grid_constant__ SimtAttnParams P) {
  extern __shared__ __align__(16) float sm[];
  float* Qt = sm;                    // [d][q]
  float* Kt = Qt + kHD * kBQ;        // [d][key]
  float* Vs = Kt + kHD * kBKV;       // [key][d]
  float* Ps = Vs + kBKV * kHD;       // [q][key] (+1 pad)
  float* m_s = Ps + kBQ * (kBKV + 1);
  float* l_s = m_s + kBQ;
  float* a_s = l_s + kBQ;

  const int h = blockIdx.y;
  const int qt = blockIdx.x;
  int g = 0;
  while (g + 1 < P.n_seg && P.tile_prefix[g + 1] <= qt) ++g;
  const int s0 = P.start[g];
  const int s1 = P.start[g + 1];
  const int q0 = s0 + (qt - P.tile_prefix[g]) * kBQ;
  const int tid = threadIdx.x;
  const size_t ld = 3 * static_cast<size_t>(D);
  const float scale = 0.125f;  // 1 / sqrt(64), exact

  for (int i = tid; i < kBQ * kHD / 4; i += 256) {
    const int r = i >> 4;
    const int d4 = (i & 15) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q0 + r < s1) v = __ldg(reinterpret_cast<const float4*>(qkv + (q0 + r) * ld + h * kHD + d4));
    Qt[(d4 + 0) * kBQ + r] = v.x * scale;
    Qt[(d4 + 1) * kBQ + r] = v.y * scale;
    Qt[(d4 + 2) * kBQ + r] = v.z * scale;
    Qt[(d4 + 3) * kBQ + r] = v.w * scale;
  }
  if (tid < kBQ) {
    m_s[tid] = -INFINITY;
    l_s[tid] = 0.f;
  }

  const int ti = tid >> 4;  // rows ti*4 .. +3
  const int tj = tid & 15;  // keys / dims tj*4 .. +3
  float o[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) o[i][j] = 0.f;

  for (int kv0 = s0; kv0 < s1; kv0 += kBKV) {
    __syncthreads();
    for (int i = tid; i < kBKV * kHD / 4; i += 256) {
      const int r = i >> 4;
      const int d4 = (i & 15) * 4;
      float4 kv = make_float4(0.f, 0.f, 0.f, 0.f), vv = kv;
      if (kv0 + r < s1) {
        kv = __ldg(reinterpret_cast<const float4*>(qkv + (kv0 + r) * ld + D + h * kHD + d4));
        vv = __ldg(reinterpret_cast<const float4*>(qkv + (kv0 + r) * ld + 2 * D + h * kHD + d4));
      }
      Kt[(d4 + 0) * kBKV + r] = kv.x;
      Kt[(d4 + 1) * kBKV + r] = kv.y;
      Kt[(d4 + 2) * kBKV + r] = kv.z;
      Kt[(d4 + 3) * kBKV + r] = kv.w;
      *reinterpret_cast<float4*>(&Vs[r * kHD + d4]) = vv;
    }
    __syncthreads();

    float s[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[i][j] = 0.f;
#pragma unroll 8
    for (int d = 0; d < kHD; ++d) {
      const float4 a = *reinterpret_cast<const float4*>(&Qt[d * kBQ + ti * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Kt[d * kBKV + tj * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[i][j] = fmaf(av[i], bv[j], s[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) Ps[(ti * 4 + i) * (kBKV + 1) + tj * 4 + j] = s[i][j];
    __syncthreads();

    {
      const int r = tid >> 2;
      const int part = tid & 3;
      float* prow = Ps + r * (kBKV + 1);
      float mx = -INFINITY;
      for (int j = part * 16; j < part * 16 + 16; ++j)
        if (kv0 + j < s1) mx = fmaxf(mx, prow[j]);
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      const float m_old = m_s[r];
      const float m_new = fmaxf(m_old, mx);
      float sum = 0.f;
      for (int j = part * 16; j < part * 16 + 16; ++j) {
        const float p = (kv0 + j < s1) ? expf(prow[j] - m_new) : 0.f;
        prow[j] = p;
        sum += p;
      }
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      __syncwarp();
      if (part == 0) {
        const float a = expf(m_old - m_new);
        a_s[r] = a;
        l_s[r] = l_s[r] * a + sum;
        m_s[r] = m_new;
      }
    }
    __syncthreads();

#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float a = a_s[ti * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) o[i][j] *= a;
    }
#pragma unroll 4
    for (int j = 0; j < kBKV; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(&Vs[j * kHD + tj * 4]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float p = Ps[(ti * 4 + i) * (kBKV + 1) + j];
        o[i][0] = fmaf(p, v.x, o[i][0]);
        o[i][1] = fmaf(p, v.y, o[i][1]);
        o[i][2] = fmaf(p, v.z, o[i][2]);
        o[i][3] = fmaf(p, v.w, o[i][3]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ti * 4 + i;
    if (q0 + r >= s1) continue;
    const float inv = 1.f / l_s[r];
    *reinterpret_cast<float4*>(out + static_cast<size_t>(q0 + r) * D + h * kHD + tj * 4) =
        make_float4(o[i][0] * inv, o[i][1] * inv, o[i][2] * inv, o[i][3] * inv);
  }
}

}  // namespace

cudaError_t launch_attention_simt(const float* qkv, float* out, int M, int D, int heads, const Segments& seg,
                                  cudaStream_t st) {
  if (seg.n <= 0 || seg.n > kMaxSegments || D != heads * kHD) return cudaErrorInvalidValue;
  SimtAttnParams P{};
  P.n_seg = seg.n;
  int tiles = 0;
  for (int g = 0; g < seg.n; ++g) {
    P.start[g] = seg.start[g];
    P.tile_prefix[g] = tiles;
    const int len = seg.start[g + 1] - seg.start[g];
    if (len < 0 || seg.start[g] < 0 || seg.start[g + 1] > M) return cudaErrorInvalidValue;
    tiles += (len + kBQ - 1) / kBQ;
  }
  P.start[seg.n] = seg.start[seg.n];
  P.tile_prefix[seg.n] = tiles;
  if (tiles == 0) return cudaSuccess;
  const int smem = kSmemFloats * static_cast<int>(sizeof(float));
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = ensure_smem_attr(attn_simt_kernel, smem, attr_done);
  if (e != cudaSuccess) return e;
  attn_simt_kernel<<<dim3(tiles, heads), 256, smem, st>>>(qkv, out, D, P);
  return cudaGetLastError();
}

}  // namespace revo
