// Multi-head softmax attention on the tcgen05 tensor cores (bf16 operands,
// f32 accumulation and softmax).  Exact scaled dot-product attention over
// every token of a segment (Appendix B.1, points 4-5: flash-style attention,
// no token dropping), computed flash-style with an online softmax.
//
// One CTA owns two 128-row query tiles (256 queries) of one head of one
// segment; both tiles share every K/V tile it streams in (128 keys each).  TMA
// reads the head's 64-column slices of Q, K and V straight out of the qkv
// matrix [M][3D] (128-byte swizzle), so no head-split pass is needed.  Per
// K/V tile j and query tile t:
//   S_t(j) = Q_t K_j^T         tcgen05.mma M=128 N=128 K=64 -> the S columns
//   P_t(j) = exp2(S c - m_t)   softmax warpgroup t, bf16, into the P columns
//   O_t  += P_t(j) V_j         tcgen05.mma M=128 N=64 K=128, A = P from TMEM,
//                              V read N-major from shared memory
// Each query tile has S (128 columns), P (64: bf16 pairs) and O (64): 256 of
// TMEM's 512 columns.  S and P live apart, so S_t(j+1) is issued as soon as the
// softmax has loaded S_t(j) into registers (it runs during that block's
// exponentials) and PV_t(j) during the next block's; the softmax only waits
// for PV_t(j-1) before it writes P_t(j), by which time it has finished.  A
// rescale of O happens only when a row's maximum grows by more than 2^8 (P
// stays below 256; the result is the same softmax).
//
// Warp roles (352 threads): warp 0 TMA, warp 1 TMEM allocator + MMA issuer
// of tile 0, warps 2..5 softmax of tile 0, warps 6..9 softmax of tile 1 (warp
// w owns rows 32*(w%4) .. +31 of its tile, the TMEM lanes it may access),
// warp 10 MMA issuer of tile 1.  Handoffs: K/V tiles, S ready and PV done are
// mbarriers (TMA transaction counts, tcgen05.commit); S free and P ready are
// named barriers on which the MMA warp waits suspended.
#include <algorithm>

#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kQ = 128;
constexpr int kTiles = 2;  // query tiles per CTA
constexpr int kKV = 128;   // keys per K/V tile
constexpr int kHD = 64;
constexpr int kKvStages = 5;
constexpr int kBoxRows = 32;  // TMA box height: Q = 4 boxes, a K or V tile = 4
constexpr int kThreads = 64 + kTiles * 128 + 32;  // + the second tile's MMA warp
constexpr int kQBytes = kQ * kHD * 2;    // 16 KB: 128 rows x 128 B
constexpr int kKVBytes = kKV * kHD * 2;  // 16 KB
constexpr int kBoxBytes = kBoxRows * kHD * 2;
constexpr int kSmemBytes = 1024 + kQBytes * kTiles + 2 * kKVBytes * kKvStages + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTileCols = 256;   // per tile: S at 0 (128 columns), P at 128 (64), O at 192 (64)
constexpr uint32_t kSCol = 0;
constexpr uint32_t kPCol = 128;
constexpr uint32_t kOCol = 192;
constexpr float kRescaleLog2 = 8.0f;  // rescale once a row max grows by more than 2^8

struct TcAttnParams {
  int D, n_seg, heads, items;
  float scale_log2;
  int start[kMaxSegments + 1];
  int item_prefix[kMaxSegments + 1];  // work items (256-query blocks) before each segment
  // Work unit u = head * items + item; this launch covers units
  // [unit_base, unit_base + gridDim.x / chunks), each split into `chunks`
  // contiguous K/V ranges.  part == null: whole rows, bf16 out; else each CTA
  // writes its rows' unnormalised O, reference maximum and sum to slot
  // blockIdx.x of `part` for attn_combine_kernel.
  int unit_base, chunks;
  float* part;  // [slots][256][64] O, then [slots][256][2] (m, l)
};

constexpr int kPartRows = kTiles * kQ;  // 256 rows per partial slot

// Keys at or beyond `nvalid` in columns [col0, col0 + 32) get a score of -inf.
REVO_DEVI void mask_chunk(uint32_t (&v)[32], int col0, int nvalid) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (col0 + i >= nvalid) v[i] = 0xff800000u;
}

// Three-input maximum (one instruction for two new values).
REVO_DEVI float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Running maxima in 8 independent lanes (short dependency chains), two new
// values per instruction.
REVO_DEVI void max_chunk(const uint32_t (&v)[32], float (&mx)[8]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2)
    mx[(i >> 1) & 7] = max3(mx[(i >> 1) & 7], __uint_as_float(v[i]), __uint_as_float(v[i + 1]));
}

// p = 2^(s c - m) for 32 keys (scale and shift as packed pairs); packs them as
// bf16 pairs (key 2i in the low half) into pk[off .. off + 15] and adds them
// into 4 packed pairs of partial sums.
REVO_DEVI void exp_chunk(const uint32_t (&v)[32], uint64_t c2, uint64_t negm2, uint32_t (&pk)[32], int off,
                         uint64_t (&sum2)[4]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float a0, a1;
    unpk2(fma2(pk2(__uint_as_float(v[i]), __uint_as_float(v[i + 1])), c2, negm2), a0, a1);
    const float p0 = ex2_approx(a0);
    const float p1 = ex2_approx(a1);
    sum2[(i >> 1) & 3] = add2(sum2[(i >> 1) & 3], pk2(p0, p1));
    pk[off + i / 2] = pack_bf16x2(p0, p1);
  }
}

// Handoffs from the softmax warpgroup of tile t to its MMA warp, on named
// barriers (128 softmax threads arrive, the 32 threads of the MMA warp wait
// suspended in hardware: a polling MMA thread would take issue and MIO slots
// from the softmax warps of its SM sub-partition).  S-free (1 + 2 t): S(j) is
// in the softmax registers, the S columns may take S(j + 1).  P-ready (2 + 2 t):
// P(j) is in the P columns.  One barrier of each kind per tile suffices: the
// arrivals for j + 1 need S(j + 1) (issued after the MMA warp passed S-free(j))
// and, for P-ready, PV(j) (issued after it passed P-ready(j)).
constexpr uint32_t kSoftmaxPlusMma = 128 + 32;
REVO_DEVI uint32_t s_free_id(int t) { return 1u + 2u * static_cast<uint32_t>(t); }
REVO_DEVI uint32_t p_ready_id(int t) { return 2u + 2u * static_cast<uint32_t>(t); }
REVO_DEVI void bar_arrive_named(uint32_t id, uint32_t n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
REVO_DEVI void bar_sync_named(uint32_t id, uint32_t n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Producer wait for a free K/V stage: polls with a short sleep in between
// (the ring runs kKvStages tiles ahead, so a late wake-up costs nothing),
// leaving the issue slots of its sub-partition to the softmax warps there.
REVO_DEVI bool mbar_wait_sleepy(uint64_t* bar, uint32_t parity, int* err, int code) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_test(a, parity)) return true;
    __nanosleep(128);
    if ((it & 63u) == 63u) {
      if (*reinterpret_cast<volatile int*>(err) != 0) return false;
      if (clock64() - t0 > kWaitLimitCycles) {
        atomicCAS(err, 0, code);
        return false;
      }
    }
  }
}

REVO_DEVI float reduce8_max(const float (&a)[8]) {
  return fmaxf(fmaxf(fmaxf(a[0], a[1]), fmaxf(a[2], a[3])), fmaxf(fmaxf(a[4], a[5]), fmaxf(a[6], a[7])));
}

REVO_DEVI float reduce8_sum(const float (&a)[8]) {
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

__global__ void __launch_bounds__(kThreads, 1)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tm, __nv_bfloat16* __restrict__ out,
                   const __grid_constant__ TcAttnParams P, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sQ = smem;                        // kTiles x 16 KB
  uint8_t* sK = sQ + kTiles * kQBytes;       // kKvStages x 16 KB
  uint8_t* sV = sK + kKvStages * kKVBytes;   // kKvStages x 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sV + kKvStages * kKVBytes);
  uint64_t* q_full = bars;
  uint64_t* kv_full = q_full + 1;
  uint64_t* kv_empty = kv_full + kKvStages;
  uint64_t* s_full = kv_empty + kKvStages;  // [kTiles] S_t(j) in the S columns
  uint64_t* pv_done = s_full + kTiles;      // [kTiles] PV_t(j) accumulated: P columns free, O stable
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pv_done + kTiles);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int unit = P.unit_base + static_cast<int>(blockIdx.x) / P.chunks;
  const int chunk = static_cast<int>(blockIdx.x) % P.chunks;
  const int h = unit / P.items;
  const int item = unit % P.items;
  int g = 0;
  while (g + 1 < P.n_seg && P.item_prefix[g + 1] <= item) ++g;
  const int s0 = P.start[g];
  const int s1 = P.start[g + 1];
  const int q0 = s0 + (item - P.item_prefix[g]) * (kTiles * kQ);
  const int nkv_all = (s1 - s0 + kKV - 1) / kKV;
  const int per = (nkv_all + P.chunks - 1) / P.chunks;
  const int kv0 = chunk * per;                             // first K/V tile of this CTA
  const int nkv = max(0, min(nkv_all, kv0 + per) - kv0);   // K/V tiles of this CTA
  const int ntiles = (s1 - q0) > kQ ? kTiles : 1;  // the second tile may lie past the segment end
  const int D = P.D;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tm);
    mbar_init(q_full, 1);
    for (int s = 0; s < kKvStages; ++s) {
      mbar_init(&kv_full[s], 1);
      mbar_init(&kv_empty[s], ntiles);  // one release per query tile's MMA thread
    }
    for (int t = 0; t < kTiles; ++t) {
      mbar_init(&s_full[t], 1);
      mbar_init(&pv_done[t], 1);
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
      mbar_arrive_expect_tx(q_full, ntiles * kQBytes);
      for (int t = 0; t < ntiles; ++t)
        for (int b = 0; b < kQ / kBoxRows; ++b)
          tma_load_2d(sQ + t * kQBytes + b * kBoxBytes, &tm, h * kHD, q0 + t * kQ + b * kBoxRows, q_full);
      for (int j = 0; j < nkv; ++j) {
        const int st = j % kKvStages;
        if (!mbar_wait_sleepy(&kv_empty[st], ((j / kKvStages) & 1) ^ 1u, err, kDevTimeoutProducer)) break;
        mbar_arrive_expect_tx(&kv_full[st], 2 * kKVBytes);
        for (int b = 0; b < kKV / kBoxRows; ++b) {
          const int row = s0 + (kv0 + j) * kKV + b * kBoxRows;
          tma_load_2d(sK + st * kKVBytes + b * kBoxBytes, &tm, D + h * kHD, row, &kv_full[st]);
          tma_load_2d(sV + st * kKVBytes + b * kBoxBytes, &tm, 2 * D + h * kHD, row, &kv_full[st]);
        }
      }
    }
  } else if (warp == 1 || warp == kThreads / 32 - 1) {
    // One MMA warp per query tile (warp 1: tile 0, the last warp: tile 1);
    // lane 0 issues, in a fixed order per K/V tile j: S(j+1) once the softmax
    // has read S(j) out of the S columns (S-free barrier), PV(j) once it has
    // written P(j) (P-ready barrier).  The whole warp takes part in both named
    // barriers for every j, also after a failed wait.
    const int t = warp == 1 ? 0 : 1;
    if (t < ntiles) {
      constexpr uint32_t kIdS = idesc_bf16(kQ, kKV);
      constexpr uint32_t kIdPV = idesc_bf16(kQ, kHD, /*b_mn_major=*/true);
      const uint32_t tbase = tmem + t * kTileCols;
      const uint32_t q_lo = sw128_lo(smem_u32(sQ + t * kQBytes));
      auto issue_s = [&](int j) {
        const uint32_t k_lo = sw128_lo(smem_u32(sK + (j % kKvStages) * kKVBytes));
#pragma unroll
        for (int kk = 0; kk < kHD / 16; ++kk)  // 16 dims: 32 B of the swizzled rows
          mma_f16_hl(tbase + kSCol, q_lo + kk * 2, kSw128Hi, k_lo + kk * 2, kSw128Hi, kIdS, kk > 0 ? 1u : 0u);
        mma_commit(&s_full[t]);
      };
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait(q_full, 0, err, kDevTimeoutMma) && (nkv == 0 || mbar_wait(&kv_full[0], 0, err, kDevTimeoutMma));
        if (ok && nkv > 0) {
          tc_fence_after();
          issue_s(0);
        }
      }
      for (int j = 0; j < nkv; ++j) {
        __syncwarp();
        bar_sync_named(s_free_id(t), kSoftmaxPlusMma);
        if (lane == 0 && ok && j + 1 < nkv) {
          const int jn = j + 1;
          ok = mbar_wait(&kv_full[jn % kKvStages], (jn / kKvStages) & 1, err, kDevTimeoutMma);
          if (ok) {
            tc_fence_after();
            issue_s(jn);
          }
        }
        __syncwarp();
        bar_sync_named(p_ready_id(t), kSoftmaxPlusMma);
        if (lane == 0 && ok) {
          tc_fence_after();
          const uint32_t v_lo = sw128_lo(smem_u32(sV + (j % kKvStages) * kKVBytes));
#pragma unroll
          for (int kk = 0; kk < kKV / 16; ++kk)  // 16 keys: 8 TMEM columns of P, 2048 B of V
            mma_f16_tmem_a_hl(tbase + kOCol, tbase + kPCol + kk * 8, v_lo + kk * 128, kSw128Hi, kIdPV,
                              (j > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&pv_done[t]);
          mma_commit(&kv_empty[j % kKvStages]);  // this tile is done with K_j, V_j
        }
      }
      __syncwarp();
    }
  } else {
    const int t = (warp - 2) >> 2;  // query tile of this warpgroup
    const int q = warp & 3;
    const int r = q * 32 + lane;    // row within the tile
    if (t < ntiles) {
      const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
      const uint32_t tbase = tmem + t * kTileCols + lane_off;
      const uint32_t s_addr = tbase + kSCol;
      const uint32_t p_addr = tbase + kPCol;
      const uint32_t o_addr = tbase + kOCol;
      const uint64_t c2 = pk2(P.scale_log2, P.scale_log2);
      const float c = P.scale_log2;
      float m = -INFINITY;  // the maximum P is taken relative to (log2 units)
      float l = 0.f;
      bool ok = true;
      int j = 0;
      int passed = 0;  // named barriers of tile j already arrived at (0, 1: S-free)
      for (; j < nkv; ++j) {
        passed = 0;
        if (!mbar_wait_warp(&s_full[t], j & 1, err, kDevTimeoutSoftmax, lane)) {
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
        // S(j) is in registers: the S columns may take S(j+1).
        tc_fence_before();
        __syncwarp();
        bar_arrive_named(s_free_id(t), kSoftmaxPlusMma);
        passed = 1;
        const int nvalid = min(kKV, s1 - (s0 + (kv0 + j) * kKV));
        if (nvalid < kKV) {
          mask_chunk(v0, 0, nvalid);
          mask_chunk(v1, 32, nvalid);
          mask_chunk(v2, 64, nvalid);
          mask_chunk(v3, 96, nvalid);
        }
        float mx8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) mx8[i] = -INFINITY;
        max_chunk(v0, mx8);
        max_chunk(v1, mx8);
        max_chunk(v2, mx8);
        max_chunk(v3, mx8);
        const float cand = reduce8_max(mx8) * c;
        const float m_new = cand > m + kRescaleLog2 ? cand : m;
        const float alpha = ex2_approx(m - m_new);  // 1 when m is kept, 0 on the first tile
        uint64_t sum2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) sum2[i] = 0ull;  // +0.0f pairs
        const uint64_t negm2 = pk2(-m_new, -m_new);
        // Keys 0..63 first, so that their registers are free before the
        // second half is computed; each half is stored as soon as the P
        // columns are free.
        uint32_t pk0[32], pk1[32];
        exp_chunk(v0, c2, negm2, pk0, 0, sum2);
        exp_chunk(v1, c2, negm2, pk0, 16, sum2);
        if (j > 0) {
          // PV(j-1) must have read P(j-1) before P(j) replaces it, and O must
          // hold it before a rescale.  pv_done has j-1 or j completions here
          // (PV(j) needs this block's P), so the parity is unambiguous.
          if (!mbar_wait_warp(&pv_done[t], (j - 1) & 1, err, kDevTimeoutSoftmax, lane)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (__any_sync(0xffffffffu, alpha != 1.f)) {
            // Rare: O *= alpha, 16 columns at a time (few live registers).
#pragma unroll 1
            for (int c16 = 0; c16 < kHD; c16 += 16) {
              uint32_t o16[16];
              tmem_ld16(o_addr + c16, o16);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i) o16[i] = __float_as_uint(__uint_as_float(o16[i]) * alpha);
              tmem_st16(o_addr + c16, o16);
              tmem_wait_st();
            }
          }
        }
        tmem_st32(p_addr, pk0);
        exp_chunk(v2, c2, negm2, pk1, 0, sum2);
        exp_chunk(v3, c2, negm2, pk1, 16, sum2);
        tmem_st32(p_addr + 32, pk1);
        float sum8[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) unpk2(sum2[i], sum8[2 * i], sum8[2 * i + 1]);
        const float sum = reduce8_sum(sum8);
        tmem_wait_st();
        l = l * alpha + sum;
        m = m_new;
        tc_fence_before();
        __syncwarp();
        bar_arrive_named(p_ready_id(t), kSoftmaxPlusMma);
      }
      // After a failed wait: take part in the remaining named barriers in
      // order, waiting on each (arriving ahead could complete a later phase).
      for (; j < nkv; ++j) {
        __syncwarp();
        if (passed == 0) bar_sync_named(s_free_id(t), kSoftmaxPlusMma);
        passed = 0;
        __syncwarp();
        bar_sync_named(p_ready_id(t), kSoftmaxPlusMma);
      }
      // The last PV: completion nkv-1 of pv_done (nothing later is issued).
      const int last = nkv - 1;
      uint32_t o0[32], o1[32];
      bool have_o = false;
      if (ok && nkv > 0 && mbar_wait_warp(&pv_done[t], last & 1, err, kDevTimeoutSoftmax, lane)) {
        tc_fence_after();
        tmem_ld32(o_addr, o0);
        tmem_ld32(o_addr + 32, o1);
        tmem_wait_ld();
        have_o = true;
      }
      if (P.part) {
        // Partial: unnormalised O, the reference maximum m (log2 units) and
        // the sum l of this CTA's K/V range (an empty range: O = 0, l = 0).
        const size_t slot_row = static_cast<size_t>(blockIdx.x) * kPartRows + t * kQ + r;
        float4* po = reinterpret_cast<float4*>(P.part + slot_row * kHD);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          po[u] = have_o ? make_float4(__uint_as_float(o0[4 * u]), __uint_as_float(o0[4 * u + 1]),
                                       __uint_as_float(o0[4 * u + 2]), __uint_as_float(o0[4 * u + 3]))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
          po[8 + u] = have_o ? make_float4(__uint_as_float(o1[4 * u]), __uint_as_float(o1[4 * u + 1]),
                                           __uint_as_float(o1[4 * u + 2]), __uint_as_float(o1[4 * u + 3]))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float* pml = P.part + static_cast<size_t>(gridDim.x) * kPartRows * kHD + slot_row * 2;
        pml[0] = have_o ? m : -INFINITY;
        pml[1] = have_o ? l : 0.f;
      } else if (have_o) {
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

// Merges the `chunks` partial results of each split work unit: per query row
// O = sum_c 2^(m_c - M) O_c, l = sum_c 2^(m_c - M) l_c with M = max_c m_c, and
// writes O / l as bf16.  One thread per (unit, row, 4 columns).
__global__ void attn_combine_kernel(const __grid_constant__ TcAttnParams P, __nv_bfloat16* __restrict__ out,
                                    int nunits) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<long long>(nunits) * kPartRows * (kHD / 4)) return;
  const int c4 = static_cast<int>(idx % (kHD / 4));
  const int row = static_cast<int>((idx / (kHD / 4)) % kPartRows);
  const int ul = static_cast<int>(idx / (kHD / 4) / kPartRows);
  const int unit = P.unit_base + ul;
  const int h = unit / P.items;
  const int item = unit % P.items;
  int g = 0;
  while (g + 1 < P.n_seg && P.item_prefix[g + 1] <= item) ++g;
  const int q = P.start[g] + (item - P.item_prefix[g]) * kPartRows + row;
  if (q >= P.start[g + 1]) return;
  const size_t slots = static_cast<size_t>(nunits) * P.chunks;
  const float* ml = P.part + slots * kPartRows * kHD;
  float M = -INFINITY;
  for (int c = 0; c < P.chunks; ++c) {
    const size_t sr = (static_cast<size_t>(ul) * P.chunks + c) * kPartRows + row;
    M = fmaxf(M, ml[sr * 2]);
  }
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  float L = 0.f;
  for (int c = 0; c < P.chunks; ++c) {
    const size_t sr = (static_cast<size_t>(ul) * P.chunks + c) * kPartRows + row;
    const float mc = ml[sr * 2];
    if (mc == -INFINITY) continue;
    const float w = ex2_approx(mc - M);
    const float4 oc = reinterpret_cast<const float4*>(P.part + sr * kHD)[c4];
    o.x = fmaf(w, oc.x, o.x);
    o.y = fmaf(w, oc.y, o.y);
    o.z = fmaf(w, oc.z, o.z);
    o.w = fmaf(w, oc.w, o.w);
    L = fmaf(w, ml[sr * 2 + 1], L);
  }
  const float inv = 1.f / L;
  uint2* dst = reinterpret_cast<uint2*>(out + static_cast<size_t>(q) * P.D + h * kHD + c4 * 4);
  *dst = make_uint2(pack_bf16x2(o.x * inv, o.y * inv), pack_bf16x2(o.z * inv, o.w * inv));
}

}  // namespace

size_t attention_partial_bytes(int num_sms) {
  return static_cast<size_t>(num_sms) * kPartRows * (kHD + 2) * sizeof(float);
}

bool encode_attention_tmap(CUtensorMap* map, const void* qkv, int M, int D) {
  return encode_tmap_bf16_2d(map, qkv, static_cast<uint64_t>(M), 3ull * D, 3ull * D, kBoxRows, kHD);
}

cudaError_t launch_attention_tc(const CUtensorMap& qkv_map, void* out, int M, int D, int heads, const Segments& seg,
                                int* err, cudaStream_t st, float* part, int num_sms, int* launched) {
  if (launched) *launched = 0;
  if (seg.n <= 0 || seg.n > kMaxSegments || D != heads * kHD) return cudaErrorInvalidValue;
  TcAttnParams P{};
  P.D = D;
  P.n_seg = seg.n;
  P.heads = heads;
  P.scale_log2 = 1.4426950408889634f * 0.125f;  // log2(e) / sqrt(64)
  int items = 0, min_nkv = 1 << 30;
  for (int g = 0; g < seg.n; ++g) {
    const int len = seg.start[g + 1] - seg.start[g];
    if (len < 0 || seg.start[g] < 0 || seg.start[g + 1] > M) return cudaErrorInvalidValue;
    P.start[g] = seg.start[g];
    P.item_prefix[g] = items;
    items += (len + kTiles * kQ - 1) / (kTiles * kQ);
    if (len > 0) min_nkv = std::min(min_nkv, (len + kKV - 1) / kKV);
  }
  P.start[seg.n] = seg.start[seg.n];
  P.item_prefix[seg.n] = items;
  if (items == 0) return cudaSuccess;
  P.items = items;
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = ensure_smem_attr(attn_tc_kernel, kSmemBytes, attr_done);
  if (e != cudaSuccess) return e;
  // Work units (head, 256-query item).  Whole waves of units run with their
  // full K/V range; the units of a last, partly filled wave (or all of them,
  // when there are fewer units than SMs) are split into `chunks` K/V ranges so
  // that wave fills the SMs, and their partial results are merged after.
  const int units = items * heads;
  const int G = num_sms > 0 ? num_sms : 148;
  int full = units, chunks = 1;
  if (part) {
    const int base = units >= G ? (units / G) * G : 0;
    const int rest = units - base;
    if (rest > 0) {
      int c = std::min(std::min(G / rest, 8), min_nkv);
      if (c >= 2) {
        full = base;
        chunks = c;
      }
    }
  }
  int n = 0;
  if (full > 0) {
    P.unit_base = 0;
    P.chunks = 1;
    P.part = nullptr;
    attn_tc_kernel<<<full, kThreads, kSmemBytes, st>>>(qkv_map, static_cast<__nv_bfloat16*>(out), P, err);
    ++n;
  }
  if (full < units) {
    const int rest = units - full;
    P.unit_base = full;
    P.chunks = chunks;
    P.part = part;
    attn_tc_kernel<<<rest * chunks, kThreads, kSmemBytes, st>>>(qkv_map, static_cast<__nv_bfloat16*>(out), P, err);
    const long long threads = static_cast<long long>(rest) * kPartRows * (kHD / 4);
    attn_combine_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(
        P, static_cast<__nv_bfloat16*>(out), rest);
    n += 2;
  }
  if (launched) *launched = n;
  return cudaGetLastError();
}

}  // namespace revo
