// Multi-head softmax attention on the tcgen05 tensor cores (bf16 operands,
// f32 accumulation and softmax).  Exact scaled dot-product attention over
// every token of a segment (Appendix B.1, points 4-5: flash-style attention,
// no token dropping), computed flash-style with an online softmax.
//
// One CTA owns 128 queries of one head of one segment.  TMA reads the head's
// 64-column slices of Q, K and V straight out of the qkv matrix [M][3D]
// (128-byte swizzle), so no head-split pass is needed:
//   S_j  = Q K_j^T         tcgen05.mma M=128 N=128 K=64 -> TMEM (double buffer)
//   P_j  = exp2(S_j*c - m) softmax warps, bf16, written to shared memory in
//                          the swizzled K-major operand layout
//   PV_j = P_j V_j         tcgen05.mma M=128 N=64 K=128, V read N-major -> TMEM
//   O    = alpha O + PV    in the softmax warps' registers (one row per thread)
// S_{j+1} is computed while the softmax of S_j runs, and PV_j while the softmax
// of S_{j+1} runs.
//
// Warp roles (192 threads): warp 0 TMA, warp 1 TMEM allocator + MMA issuer,
// warps 2..5 softmax/correction/epilogue (warp w owns rows 32*(w%4) .. +31).
#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kQ = 128;
constexpr int kKV = 128;
constexpr int kHD = 64;
constexpr int kKvStages = 3;
constexpr int kTileBytes = kQ * kHD * 2;        // 16 KB: 128 rows x 128 B
constexpr int kPBytes = kQ * kKV * 2;           // 32 KB: two 128 x 64 atoms
constexpr int kSmemBytes = 1024 + kTileBytes * (1 + 2 * kKvStages) + 2 * kPBytes + 512;
constexpr uint32_t kTmemCols = 512;             // S: 2 x 128, PV: 2 x 64
constexpr uint32_t kPvCol = 256;

struct TcAttnParams {
  int D, n_seg;
  float scale_log2;
  int start[kMaxSegments + 1];
  int tile_prefix[kMaxSegments + 1];
};

__global__ void __launch_bounds__(192, 1)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tm, __nv_bfloat16* __restrict__ out,
                   const __grid_constant__ TcAttnParams P, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sQ = smem;
  uint8_t* sK = sQ + kTileBytes;
  uint8_t* sV = sK + kKvStages * kTileBytes;
  uint8_t* sP = sV + kKvStages * kTileBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sP + 2 * kPBytes);
  uint64_t* q_full = bars;
  uint64_t* kv_full = bars + 1;
  uint64_t* kv_empty = kv_full + kKvStages;
  uint64_t* s_full = kv_empty + kKvStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 2;
  uint64_t* p_empty = p_full + 2;
  uint64_t* pv_full = p_empty + 2;
  uint64_t* pv_empty = pv_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pv_empty + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int h = blockIdx.y;
  const int qt = blockIdx.x;
  int g = 0;
  while (g + 1 < P.n_seg && P.tile_prefix[g + 1] <= qt) ++g;
  const int s0 = P.start[g];
  const int s1 = P.start[g + 1];
  const int q0 = s0 + (qt - P.tile_prefix[g]) * kQ;
  const int nkv = (s1 - s0 + kKV - 1) / kKV;
  const int D = P.D;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tm);
    mbar_init(q_full, 1);
    for (int s = 0; s < kKvStages; ++s) {
      mbar_init(&kv_full[s], 1);
      mbar_init(&kv_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&s_full[b], 1);
      mbar_init(&s_empty[b], 4);
      mbar_init(&p_full[b], 4);
      mbar_init(&p_empty[b], 1);
      mbar_init(&pv_full[b], 1);
      mbar_init(&pv_empty[b], 4);
    }
    fence_mbarrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      mbar_arrive_expect_tx(q_full, kTileBytes);
      tma_load_2d(sQ, &tm, h * kHD, q0, q_full);
      for (int j = 0; j < nkv; ++j) {
        const int st = j % kKvStages;
        const uint32_t ph = (j / kKvStages) & 1;
        if (!mbar_wait(&kv_empty[st], ph ^ 1u, err, kDevTimeoutProducer)) break;
        mbar_arrive_expect_tx(&kv_full[st], 2 * kTileBytes);
        tma_load_2d(sK + st * kTileBytes, &tm, D + h * kHD, s0 + j * kKV, &kv_full[st]);
        tma_load_2d(sV + st * kTileBytes, &tm, 2 * D + h * kHD, s0 + j * kKV, &kv_full[st]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t kIdS = idesc_bf16(kQ, kKV);
      constexpr uint32_t kIdPV = idesc_bf16(kQ, kHD, /*b_mn_major=*/true);
      bool ok = mbar_wait(q_full, 0, err, kDevTimeoutMma);
      const uint32_t q_addr = smem_u32(sQ);
      for (int j = 0; ok && j <= nkv; ++j) {
        if (j < nkv) {
          const int st = j % kKvStages;
          const int sb = j & 1;
          if (!mbar_wait(&kv_full[st], (j / kKvStages) & 1, err, kDevTimeoutMma)) break;
          if (!mbar_wait(&s_empty[sb], ((j >> 1) & 1) ^ 1u, err, kDevTimeoutMma)) break;
          tc_fence_after();
          const uint32_t k_addr = smem_u32(sK + st * kTileBytes);
#pragma unroll
          for (int kk = 0; kk < kHD / 16; ++kk)
            mma_f16(tmem + sb * kKV, sw128_desc(q_addr + kk * 32), sw128_desc(k_addr + kk * 32), kIdS,
                    kk > 0 ? 1u : 0u);
          mma_commit(&s_full[sb]);
        }
        if (j >= 1) {
          const int jj = j - 1;
          const int pb = jj & 1;
          const int stj = jj % kKvStages;
          if (!mbar_wait(&p_full[pb], (jj >> 1) & 1, err, kDevTimeoutMma)) break;
          if (!mbar_wait(&pv_empty[pb], ((jj >> 1) & 1) ^ 1u, err, kDevTimeoutMma)) break;
          tc_fence_after();
          const uint32_t p_addr = smem_u32(sP + pb * kPBytes);
          const uint32_t v_addr = smem_u32(sV + stj * kTileBytes);
#pragma unroll
          for (int kk = 0; kk < kKV / 16; ++kk)
            mma_f16(tmem + kPvCol + pb * kHD, sw128_desc(p_addr + (kk >> 2) * kTileBytes + (kk & 3) * 32),
                    sw128_desc(v_addr + kk * 2048), kIdPV, kk > 0 ? 1u : 0u);
          mma_commit(&pv_full[pb]);
          mma_commit(&p_empty[pb]);
          mma_commit(&kv_empty[stj]);
        }
      }
    }
  } else {
    const int q = warp & 3;
    const int r = q * 32 + lane;  // row within the tile
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const float c = P.scale_log2;
    float m = -INFINITY, l = 0.f;
    float o[kHD];
#pragma unroll
    for (int i = 0; i < kHD; ++i) o[i] = 0.f;
    bool ok = true;
    uint8_t* p_row_base = sP + r * 128;
    const int sw = r & 7;

    for (int j = 0; j < nkv && ok; ++j) {
      const int sb = j & 1;
      if (!mbar_wait(&s_full[sb], (j >> 1) & 1, err, kDevTimeoutSoftmax)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int nvalid = min(kKV, s1 - (s0 + j * kKV));
      float mx = -INFINITY;
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t v[32];
        tmem_ld32(lane_base + sb * kKV + ch * 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (ch * 32 + i < nvalid) mx = fmaxf(mx, __uint_as_float(v[i]) * c);
      }
      const float m_new = fmaxf(m, mx);
      const float alpha = ex2_approx(m - m_new);
      if (!mbar_wait(&p_empty[sb], ((j >> 1) & 1) ^ 1u, err, kDevTimeoutSoftmax)) {
        ok = false;
        break;
      }
      float sum = 0.f;
      uint8_t* prow = p_row_base + sb * kPBytes;
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t v[32];
        tmem_ld32(lane_base + sb * kKV + ch * 32, v);
        tmem_wait_ld();
        float pv[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          pv[i] = (ch * 32 + i < nvalid) ? ex2_approx(__uint_as_float(v[i]) * c - m_new) : 0.f;
          sum += pv[i];
        }
        uint8_t* atom = prow + (ch >> 1) * kTileBytes;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int chunk = (ch & 1) * 4 + u;
          const uint4 w = make_uint4(pack_bf16x2(pv[8 * u], pv[8 * u + 1]), pack_bf16x2(pv[8 * u + 2], pv[8 * u + 3]),
                                     pack_bf16x2(pv[8 * u + 4], pv[8 * u + 5]),
                                     pack_bf16x2(pv[8 * u + 6], pv[8 * u + 7]));
          *reinterpret_cast<uint4*>(atom + ((chunk ^ sw) << 4)) = w;
        }
      }
      tc_fence_before();
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&s_empty[sb]);
        mbar_arrive(&p_full[sb]);
      }
      l = l * alpha + sum;
      if (j > 0) {
        const int pp = (j - 1) & 1;
        if (!mbar_wait(&pv_full[pp], ((j - 1) >> 1) & 1, err, kDevTimeoutSoftmax)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t v[32];
          tmem_ld32(lane_base + kPvCol + pp * kHD + ch * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) o[ch * 32 + i] += __uint_as_float(v[i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&pv_empty[pp]);
      }
#pragma unroll
      for (int i = 0; i < kHD; ++i) o[i] *= alpha;
      m = m_new;
    }
    if (ok && nkv > 0) {
      const int pp = (nkv - 1) & 1;
      if (mbar_wait(&pv_full[pp], ((nkv - 1) >> 1) & 1, err, kDevTimeoutSoftmax)) {
        tc_fence_after();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t v[32];
          tmem_ld32(lane_base + kPvCol + pp * kHD + ch * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) o[ch * 32 + i] += __uint_as_float(v[i]);
        }
        const int row = q0 + r;
        if (row < s1) {
          const float inv = 1.f / l;
          uint4* dst = reinterpret_cast<uint4*>(out + static_cast<size_t>(row) * D + h * kHD);
#pragma unroll
          for (int u = 0; u < 8; ++u)
            dst[u] = make_uint4(pack_bf16x2(o[8 * u] * inv, o[8 * u + 1] * inv),
                                pack_bf16x2(o[8 * u + 2] * inv, o[8 * u + 3] * inv),
                                pack_bf16x2(o[8 * u + 4] * inv, o[8 * u + 5] * inv),
                                pack_bf16x2(o[8 * u + 6] * inv, o[8 * u + 7] * inv));
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

bool encode_attention_tmap(CUtensorMap* map, const void* qkv, int M, int D) {
  return encode_tmap_bf16_2d(map, qkv, static_cast<uint64_t>(M), 3ull * D, 3ull * D, kKV, kHD);
}

cudaError_t launch_attention_tc(const CUtensorMap& qkv_map, void* out, int M, int D, int heads, const Segments& seg,
                                int* err, cudaStream_t st) {
  if (seg.n <= 0 || seg.n > kMaxSegments || D != heads * kHD) return cudaErrorInvalidValue;
  TcAttnParams P{};
  P.D = D;
  P.n_seg = seg.n;
  P.scale_log2 = 1.4426950408889634f * 0.125f;  // log2(e) / sqrt(64)
  int tiles = 0;
  for (int g = 0; g < seg.n; ++g) {
    const int len = seg.start[g + 1] - seg.start[g];
    if (len < 0 || seg.start[g] < 0 || seg.start[g + 1] > M) return cudaErrorInvalidValue;
    P.start[g] = seg.start[g];
    P.tile_prefix[g] = tiles;
    tiles += (len + kQ - 1) / kQ;
  }
  P.start[seg.n] = seg.start[seg.n];
  P.tile_prefix[seg.n] = tiles;
  if (tiles == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(attn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  attn_tc_kernel<<<dim3(tiles, heads), 192, kSmemBytes, st>>>(qkv_map, static_cast<__nv_bfloat16*>(out), P, err);
  return cudaGetLastError();
}

}  // namespace revo
