// Multi-head softmax attention on the tcgen05 tensor cores (bf16 operands,
// f32 accumulation and softmax).  Exact scaled dot-product attention over
// every token of a segment (Appendix B.1, points 4-5: flash-style attention,
// no token dropping), computed flash-style with an online softmax.
//
// One CTA owns two 128-row query tiles (256 queries) of one head of one
// segment; both tiles share every K/V tile it streams in.  TMA reads the
// head's 64-column slices of Q, K and V straight out of the qkv matrix
// [M][3D] (128-byte swizzle), so no head-split pass is needed.  Per KV tile j
// and query tile t:
//   S_t  = Q_t K_j^T          tcgen05.mma M=128 N=128 K=64 -> TMEM
//   P_t  = exp2(S_t c - m_t)  softmax warpgroup t, bf16, written to shared
//                             memory in the swizzled K-major operand layout
//   O_t += P_t V_j            tcgen05.mma M=128 N=64 K=128 (V read N-major),
//                             accumulated in TMEM across the KV tiles
// The running row maximum m_t only moves when a row's maximum grows by more
// than 2^8 (then O_t and the row sum are rescaled in place), so P stays below
// 256 and rescaling is rare; the result is the same softmax.  The softmax
// threads read S once per tile and release it at once, so the MMA of the next
// tile overlaps their exponentials, and the two warpgroups give every SM
// sub-partition two independent softmax instruction streams.
//
// Warp roles (320 threads): warp 0 TMA, warp 1 TMEM allocator + MMA issuer,
// warps 2..5 softmax of tile 0, warps 6..9 softmax of tile 1 (warp w owns rows
// 32*(w%4) .. +31 of its tile, the TMEM lanes it may access).
#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kQ = 128;
constexpr int kTiles = 2;  // query tiles per CTA
constexpr int kKV = 128;
constexpr int kHD = 64;
constexpr int kKvStages = 3;
constexpr int kThreads = 64 + kTiles * 128;
constexpr int kTileBytes = kQ * kHD * 2;  // 16 KB: 128 rows x 128 B
constexpr int kPBytes = kQ * kKV * 2;     // 32 KB: two 128 x 64 atoms
constexpr int kSmemBytes = 1024 + kTileBytes * (kTiles + 2 * kKvStages) + kTiles * kPBytes + 512;
constexpr uint32_t kTmemCols = 512;  // per tile: S 128 + O 64 (256-column stride)
constexpr uint32_t kTileCols = 256;
constexpr uint32_t kOCol = 128;
constexpr float kRescaleLog2 = 8.0f;  // rescale once a row max grows by more than 2^8

struct TcAttnParams {
  int D, n_seg;
  float scale_log2;
  int start[kMaxSegments + 1];
  int item_prefix[kMaxSegments + 1];  // work items (256-query blocks) before each segment
};

// Keys at or beyond `nvalid` in columns [col0, col0 + 32) get a score of -inf.
REVO_DEVI void mask_chunk(uint32_t (&v)[32], int col0, int nvalid) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (col0 + i >= nvalid) v[i] = 0xff800000u;
}

REVO_DEVI float max_chunk(const uint32_t (&v)[32], float mx) {
#pragma unroll
  for (int i = 0; i < 32; ++i) mx = fmaxf(mx, __uint_as_float(v[i]));
  return mx;
}

// p = 2^(s c - m) for the 32 keys of chunk `ch` (columns 32 ch ..); writes them
// as bf16 into this thread's row of the swizzled P tile; returns their sum.
REVO_DEVI float exp_chunk(const uint32_t (&v)[32], int ch, float c, float m, uint8_t* prow, int sw) {
  float sum = 0.f;
  uint8_t* atom = prow + (ch >> 1) * kTileBytes;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      p[i] = ex2_approx(fmaf(__uint_as_float(v[8 * u + i]), c, -m));
      sum += p[i];
    }
    const int chunk = (ch & 1) * 4 + u;
    *reinterpret_cast<uint4*>(atom + ((chunk ^ sw) << 4)) =
        make_uint4(pack_bf16x2(p[0], p[1]), pack_bf16x2(p[2], p[3]), pack_bf16x2(p[4], p[5]),
                   pack_bf16x2(p[6], p[7]));
  }
  return sum;
}

REVO_DEVI void scale_chunk(uint32_t (&v)[32], float a) {
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) * a);
}

__global__ void __launch_bounds__(kThreads, 1)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tm, __nv_bfloat16* __restrict__ out,
                   const __grid_constant__ TcAttnParams P, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sQ = smem;                         // kTiles x 16 KB
  uint8_t* sK = sQ + kTiles * kTileBytes;     // kKvStages x 16 KB
  uint8_t* sV = sK + kKvStages * kTileBytes;  // kKvStages x 16 KB
  uint8_t* sP = sV + kKvStages * kTileBytes;  // kTiles x 32 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sP + kTiles * kPBytes);
  uint64_t* q_full = bars;
  uint64_t* kv_full = q_full + 1;
  uint64_t* kv_empty = kv_full + kKvStages;
  uint64_t* s_full = kv_empty + kKvStages;  // [kTiles] S ready in TMEM
  uint64_t* s_empty = s_full + kTiles;      // [kTiles] S read by the softmax
  uint64_t* p_full = s_empty + kTiles;      // [kTiles] P written, O rescaled
  uint64_t* p_done = p_full + kTiles;       // [kTiles] PV accumulated (P free, O stable)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(p_done + kTiles);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int h = blockIdx.y;
  const int item = blockIdx.x;
  int g = 0;
  while (g + 1 < P.n_seg && P.item_prefix[g + 1] <= item) ++g;
  const int s0 = P.start[g];
  const int s1 = P.start[g + 1];
  const int q0 = s0 + (item - P.item_prefix[g]) * (kTiles * kQ);
  const int nkv = (s1 - s0 + kKV - 1) / kKV;
  const int ntiles = (s1 - q0) > kQ ? kTiles : 1;  // the second tile may lie past the segment end
  const int D = P.D;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tm);
    mbar_init(q_full, 1);
    for (int s = 0; s < kKvStages; ++s) {
      mbar_init(&kv_full[s], 1);
      mbar_init(&kv_empty[s], 1);
    }
    for (int t = 0; t < kTiles; ++t) {
      mbar_init(&s_full[t], 1);
      mbar_init(&s_empty[t], 4);
      mbar_init(&p_full[t], 4);
      mbar_init(&p_done[t], 1);
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
      mbar_arrive_expect_tx(q_full, ntiles * kTileBytes);
      for (int t = 0; t < ntiles; ++t) tma_load_2d(sQ + t * kTileBytes, &tm, h * kHD, q0 + t * kQ, q_full);
      for (int j = 0; j < nkv; ++j) {
        const int st = j % kKvStages;
        if (!mbar_wait(&kv_empty[st], ((j / kKvStages) & 1) ^ 1u, err, kDevTimeoutProducer)) break;
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
      for (int j = 0; ok && j <= nkv; ++j) {
        if (j < nkv) {
          const int st = j % kKvStages;
          if (!mbar_wait(&kv_full[st], (j / kKvStages) & 1, err, kDevTimeoutMma)) break;
          const uint32_t k_addr = smem_u32(sK + st * kTileBytes);
          for (int t = 0; t < ntiles && ok; ++t) {
            if (!mbar_wait(&s_empty[t], (j & 1) ^ 1u, err, kDevTimeoutMma)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t q_addr = smem_u32(sQ + t * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < kHD / 16; ++kk)
              mma_f16(tmem + t * kTileCols, sw128_desc(q_addr + kk * 32), sw128_desc(k_addr + kk * 32), kIdS,
                      kk > 0 ? 1u : 0u);
            mma_commit(&s_full[t]);
          }
          if (!ok) break;
        }
        if (j >= 1) {
          const int jj = j - 1;
          const int stj = jj % kKvStages;
          const uint32_t v_addr = smem_u32(sV + stj * kTileBytes);
          for (int t = 0; t < ntiles && ok; ++t) {
            if (!mbar_wait(&p_full[t], jj & 1, err, kDevTimeoutMma)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t p_addr = smem_u32(sP + t * kPBytes);
#pragma unroll
            for (int kk = 0; kk < kKV / 16; ++kk)
              mma_f16(tmem + t * kTileCols + kOCol, sw128_desc(p_addr + (kk >> 2) * kTileBytes + (kk & 3) * 32),
                      sw128_desc(v_addr + kk * 2048), kIdPV, (jj > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&p_done[t]);
          }
          if (!ok) break;
          mma_commit(&kv_empty[stj]);
        }
      }
    }
  } else {
    const int t = (warp - 2) >> 2;  // query tile of this warpgroup
    const int q = warp & 3;
    const int r = q * 32 + lane;    // row within the tile
    if (t < ntiles) {
      const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
      const uint32_t s_addr = tmem + t * kTileCols + lane_off;
      const uint32_t o_addr = tmem + t * kTileCols + kOCol + lane_off;
      const float c = P.scale_log2;
      float m = -INFINITY;  // the maximum P is taken relative to (log2 units)
      float l = 0.f;
      bool ok = true;
      uint8_t* prow = sP + t * kPBytes + r * 128;
      const int sw = r & 7;

      for (int j = 0; j < nkv; ++j) {
        if (!mbar_wait(&s_full[t], j & 1, err, kDevTimeoutSoftmax)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t v0[32], v1[32], v2[32], v3[32];
        tmem_ld32(s_addr, v0);
        tmem_ld32(s_addr + 32, v1);
        tmem_ld32(s_addr + 64, v2);
        tmem_ld32(s_addr + 96, v3);
        tmem_wait_ld();
        // S is in registers: the MMA may write the next tile's scores now.
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[t]);
        const int nvalid = min(kKV, s1 - (s0 + j * kKV));
        if (nvalid < kKV) {
          mask_chunk(v0, 0, nvalid);
          mask_chunk(v1, 32, nvalid);
          mask_chunk(v2, 64, nvalid);
          mask_chunk(v3, 96, nvalid);
        }
        const float cand = max_chunk(v3, max_chunk(v2, max_chunk(v1, max_chunk(v0, -INFINITY)))) * c;
        const float m_new = cand > m + kRescaleLog2 ? cand : m;
        const float alpha = ex2_approx(m - m_new);  // 1 when m is kept, 0 on the first tile
        // The previous P*V has finished: its P tile is free and O is stable.
        if (j > 0 && !mbar_wait(&p_done[t], (j - 1) & 1, err, kDevTimeoutSoftmax)) {
          ok = false;
          break;
        }
        float sum = exp_chunk(v0, 0, c, m_new, prow, sw);
        sum += exp_chunk(v1, 1, c, m_new, prow, sw);
        sum += exp_chunk(v2, 2, c, m_new, prow, sw);
        sum += exp_chunk(v3, 3, c, m_new, prow, sw);
        if (j > 0 && __any_sync(0xffffffffu, alpha != 1.f)) {
          tc_fence_after();
          tmem_ld32(o_addr, v0);
          tmem_ld32(o_addr + 32, v1);
          tmem_wait_ld();
          scale_chunk(v0, alpha);
          scale_chunk(v1, alpha);
          tmem_st32(o_addr, v0);
          tmem_st32(o_addr + 32, v1);
          tmem_wait_st();
        }
        l = l * alpha + sum;
        m = m_new;
        tc_fence_before();
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&p_full[t]);
      }
      if (ok && nkv > 0 && mbar_wait(&p_done[t], (nkv - 1) & 1, err, kDevTimeoutSoftmax)) {
        tc_fence_after();
        uint32_t o0[32], o1[32];
        tmem_ld32(o_addr, o0);
        tmem_ld32(o_addr + 32, o1);
        tmem_wait_ld();
        const int row = q0 + t * kQ + r;
        if (row < s1) {
          const float inv = 1.f / l;
          uint4* dst = reinterpret_cast<uint4*>(out + static_cast<size_t>(row) * D + h * kHD);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            dst[u] = make_uint4(pack_bf16x2(__uint_as_float(o0[8 * u]) * inv, __uint_as_float(o0[8 * u + 1]) * inv),
                                pack_bf16x2(__uint_as_float(o0[8 * u + 2]) * inv, __uint_as_float(o0[8 * u + 3]) * inv),
                                pack_bf16x2(__uint_as_float(o0[8 * u + 4]) * inv, __uint_as_float(o0[8 * u + 5]) * inv),
                                pack_bf16x2(__uint_as_float(o0[8 * u + 6]) * inv, __uint_as_float(o0[8 * u + 7]) * inv));
            dst[4 + u] =
                make_uint4(pack_bf16x2(__uint_as_float(o1[8 * u]) * inv, __uint_as_float(o1[8 * u + 1]) * inv),
                           pack_bf16x2(__uint_as_float(o1[8 * u + 2]) * inv, __uint_as_float(o1[8 * u + 3]) * inv),
                           pack_bf16x2(__uint_as_float(o1[8 * u + 4]) * inv, __uint_as_float(o1[8 * u + 5]) * inv),
                           pack_bf16x2(__uint_as_float(o1[8 * u + 6]) * inv, __uint_as_float(o1[8 * u + 7]) * inv));
          }
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
  int items = 0;
  for (int g = 0; g < seg.n; ++g) {
    const int len = seg.start[g + 1] - seg.start[g];
    if (len < 0 || seg.start[g] < 0 || seg.start[g + 1] > M) return cudaErrorInvalidValue;
    P.start[g] = seg.start[g];
    P.item_prefix[g] = items;
    items += (len + kTiles * kQ - 1) / (kTiles * kQ);
  }
  P.start[seg.n] = seg.start[seg.n];
  P.item_prefix[seg.n] = items;
  if (items == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(attn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  attn_tc_kernel<<<dim3(items, heads), kThreads, kSmemBytes, st>>>(qkv_map, static_cast<__nv_bfloat16*>(out), P, err);
  return cudaGetLastError();
}

}  // namespace revo
