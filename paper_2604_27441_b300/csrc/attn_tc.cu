// Multi-head softmax attention on the tcgen05 tensor cores (bf16 operands,
// f32 accumulation and softmax).  Exact scaled dot-product attention over
// every token of a segment (Appendix B.1, points 4-5: flash-style attention,
// no token dropping), computed flash-style with an online softmax.
//
// Work decomposition.  A unit is (head, 256-query item) of one segment; its
// work is nkv steps, one per 128-key K/V tile; one CTA runs one piece, a unit
// or a key range of one.  By default every unit is one piece.  With the tail
// cut (an option for a segment that has the GPU to itself), of a segment's U
// units (head-major) the whole waves -- floor(U / SMs) * SMs units -- run as
// one piece each and the rest, which would leave SMs idle in a last, partly
// filled wave, are each cut into c key ranges (c = SMs / rest, at most 8);
// a part writes its unnormalised O, reference maximum and sum to a partial
// slot and attn_combine_kernel merges each cut unit's parts in key order.  The
// cut depends on the segment's length only, so a segment gives bit for bit the
// same result alone and inside a batch of other segments.
//
// One CTA owns two 128-row query tiles (256 queries) of the current unit; both
// share every K/V tile it streams in (128 keys each).  TMA reads the head's
// 64-column slices of Q, K and V straight out of the qkv matrix [M][3D]
// (128-byte swizzle), so no head-split pass is needed.
// Per K/V tile j and query tile t:
//   S_t(j) = Q_t K_j^T         tcgen05.mma M=128 N=128 K=64 -> the S columns
//   P_t(j) = exp2(S c - m_t)   softmax warpgroup t, bf16, into the P columns
//   O_t  += P_t(j) V_j         tcgen05.mma M=128 N=64 K=128, A = P from TMEM,
//                              V read N-major from shared memory
// Each query tile has S (128 columns), P (64: bf16 pairs) and O (64): 256 of
// TMEM's 512 columns.  S and P live apart, so S_t(j+1) is issued as soon as
// the softmax has loaded S_t(j) into registers, and PV_t(j) during the next
// block's exponentials; the softmax
// only waits for PV_t(j-1) before it writes P_t(j).  A rescale of O happens
// only when a row's maximum grows by more than 2^8 (P stays below 256; the
// result is the same softmax).
//
// Warp roles (352 threads): warp 0 TMA, warp 1 TMEM allocator + MMA issuer
// of tile 0, warps 2..5 softmax of tile 0, warps 6..9 softmax of tile 1 (warp
// w owns rows 32*(w%4) .. +31 of its tile, the TMEM lanes it may access),
// warp 10 MMA issuer of tile 1.  Handoffs: Q and K/V tiles, S ready and PV
// done are mbarriers (TMA transaction counts, tcgen05.commit); S free and P
// ready are named barriers on which the MMA warp waits suspended.  A unit
// whose second tile lies past its query rows runs on tile 0 alone.
#include <algorithm>
#include <vector>

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
static_assert(kSmemBytes <= 232448, "shared memory per CTA");
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTileCols = 256;   // per tile: S at 0 (128 columns), P at 128 (64), O at 192 (64)
constexpr uint32_t kSCol = 0;
constexpr uint32_t kPCol = 128;
constexpr uint32_t kOCol = 192;
constexpr float kRescaleLog2 = 8.0f;  // rescale once a row max grows by more than 2^8
constexpr int kMaxChunks = 8;         // key ranges a unit of the last wave is cut into, at most
constexpr int kPartRows = kTiles * kQ;  // 256 rows per partial slot
constexpr int kCombineRows = 16;        // rows per combine block (x 16 column groups = 256 threads)

// The pieces of one launch.  Segments with tokens, in grid order (longest
// units first); slot k covers pieces [piece_prefix[k], piece_prefix[k+1]) of
// the grid: whole[k] whole units, then (units - whole[k]) * chunks[k] parts of
// clen[k] K/V tiles (the last part of a unit shorter), whose partial slots are
// part_prefix[k] + their index among the slot's parts; the combine's blocks
// [split_prefix[k], split_prefix[k+1]) * 16 merge the slot's cut units.
struct TcAttnParams {
  int D, heads, n_slots, pieces, parts;
  float scale_log2;
  int s0[kMaxSegments], s1[kMaxSegments];     // key rows
  int qs0[kMaxSegments], qs1[kMaxSegments];   // query rows (within the key rows)
  int items[kMaxSegments], nkv[kMaxSegments]; // 256-query items, 128-key tiles
  int whole[kMaxSegments], chunks[kMaxSegments], clen[kMaxSegments];
  int piece_prefix[kMaxSegments + 1];
  int part_prefix[kMaxSegments + 1];
  int split_prefix[kMaxSegments + 1];
  // Partial slots: O [parts][256][64], then (m, l) [parts][256][2].  Null:
  // every piece is one whole unit.
  float* part;
};

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

// Independent chains of the row maximum and of the packed partial sums.  Two
// maximum and three sum chains measured fastest on the B300 (the tick's
// batched RGB encoder attention: 1580 us; 1588 with 2 and 2, 1586 with 4 and
// 2, 1627 with 2 and 4, 1658 with 8 and 4 before S was loaded 64 columns at a
// time, 1786 with one sum chain): few live registers and a short final
// reduction, while the other query tile's warp covers the latencies.
constexpr int kMaxChains = 2;
constexpr int kSumChains = 3;

// Running maxima in kMaxChains independent chains, two new values per
// instruction.
REVO_DEVI void max_chunk(const uint32_t (&v)[32], float (&mx)[kMaxChains]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2)
    mx[(i >> 1) % kMaxChains] = max3(mx[(i >> 1) % kMaxChains], __uint_as_float(v[i]), __uint_as_float(v[i + 1]));
}

// p = 2^(s c - m) for 32 keys (scale and shift as packed pairs); packs them as
// bf16 pairs (key 2i in the low half) into pk[off .. off + 15] and adds them
// into kSumChains packed pairs of partial sums.
REVO_DEVI void exp_chunk(const uint32_t (&v)[32], uint64_t c2, uint64_t negm2, uint32_t (&pk)[32], int off,
                         uint64_t (&sum2)[kSumChains]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float a0, a1;
    unpk2(fma2(pk2(__uint_as_float(v[i]), __uint_as_float(v[i + 1])), c2, negm2), a0, a1);
    const float p0 = ex2_approx(a0);
    const float p1 = ex2_approx(a1);
    sum2[(i >> 1) % kSumChains] = add2(sum2[(i >> 1) % kSumChains], pk2(p0, p1));
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

// Producer wait for a free stage: polls with a short sleep in between (the
// ring runs kKvStages tiles ahead, so a late wake-up costs nothing), leaving
// the issue slots of its sub-partition to the softmax warps there.
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

// Short bounded wait used while unwinding (copies or MMAs still in flight
// after another role gave up): never records an error of its own.
constexpr long long kDrainLimitCycles = 20000000LL;
REVO_DEVI void mbar_drain(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (!mbar_try_wait(a, parity))
    if (clock64() - t0 > kDrainLimitCycles) return;
}

REVO_DEVI float reduce_max(const float (&a)[kMaxChains]) {
  float r = a[0];
#pragma unroll
  for (int i = 1; i < kMaxChains; ++i) r = fmaxf(r, a[i]);
  return r;
}

// The row's block sum from its packed partial sums (a fixed order).
REVO_DEVI float reduce_sum(const uint64_t (&s2)[kSumChains]) {
  float lo, hi;
  unpk2(s2[0], lo, hi);
  float r = lo + hi;
#pragma unroll
  for (int i = 1; i < kSumChains; ++i) {
    unpk2(s2[i], lo, hi);
    r += lo + hi;
  }
  return r;
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
  uint64_t* drained = pv_done + kTiles;     // [kTiles] the MMA thread's last operations completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + kTiles);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int k = 0;
  while (k + 1 < P.n_slots && P.piece_prefix[k + 1] <= static_cast<int>(blockIdx.x)) ++k;
  const int piece = static_cast<int>(blockIdx.x) - P.piece_prefix[k];
  int unit = piece, kv0 = 0, kv1 = P.nkv[k];  // this CTA: unit `unit`, K/V tiles [kv0, kv1)
  if (piece >= P.whole[k]) {
    const int q = piece - P.whole[k];
    unit = P.whole[k] + q / P.chunks[k];
    kv0 = (q % P.chunks[k]) * P.clen[k];
    kv1 = min(kv0 + P.clen[k], P.nkv[k]);
  }
  const bool partial = kv0 > 0 || kv1 < P.nkv[k];
  const int nkv = kv1 - kv0;
  const int h = unit / P.items[k];
  const int s0 = P.s0[k];                // key rows
  const int s1 = P.s1[k];
  const int q0 = P.qs0[k] + (unit % P.items[k]) * (kTiles * kQ);
  const int q1 = P.qs1[k];               // query rows end
  const int ntiles = (q1 - q0) > kQ ? kTiles : 1;  // the second tile may lie past the query rows
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
      mbar_init(&drained[t], 1);
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
      int issued = 0;
      for (int j = 0; j < nkv; ++j) {
        const int st = j % kKvStages;
        if (!mbar_wait_sleepy(&kv_empty[st], ((j / kKvStages) & 1) ^ 1u, err, kDevTimeoutProducer)) break;
        mbar_arrive_expect_tx(&kv_full[st], 2 * kKVBytes);
        for (int b = 0; b < kKV / kBoxRows; ++b) {
          const int row = s0 + (kv0 + j) * kKV + b * kBoxRows;
          tma_load_2d(sK + st * kKVBytes + b * kBoxBytes, &tm, D + h * kHD, row, &kv_full[st]);
          tma_load_2d(sV + st * kKVBytes + b * kBoxBytes, &tm, 2 * D + h * kHD, row, &kv_full[st]);
        }
        issued = j + 1;
      }
      // No copy may still write into shared memory when the CTA exits: wait
      // (bounded) for the queries and the last load issued into every stage.
      mbar_drain(q_full, 0);
      for (int j = max(0, issued - kKvStages); j < issued; ++j) mbar_drain(&kv_full[j % kKvStages], (j / kKvStages) & 1);
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
      if (lane == 0) {
        // Nothing this thread issued may still run when TMEM is freed.
        mma_commit(&drained[t]);
        mbar_drain(&drained[t], 0);
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
        tmem_ld64(s_addr, v0, v1);
        tmem_ld64(s_addr + 64, v2, v3);
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
        float mx[kMaxChains];
#pragma unroll
        for (int i = 0; i < kMaxChains; ++i) mx[i] = -INFINITY;
        max_chunk(v0, mx);
        max_chunk(v1, mx);
        max_chunk(v2, mx);
        max_chunk(v3, mx);
        const float cand = reduce_max(mx) * c;
        const float m_new = cand > m + kRescaleLog2 ? cand : m;
        const float alpha = ex2_approx(m - m_new);  // 1 when m is kept, 0 on the first tile
        uint64_t sum2[kSumChains];
#pragma unroll
        for (int i = 0; i < kSumChains; ++i) sum2[i] = 0ull;  // +0.0f pairs
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
        const float sum = reduce_sum(sum2);
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
      if (partial) {
        // Partial: unnormalised O, the reference maximum m (log2 units) and
        // the sum l of this CTA's K/V range.
        const int slot = P.part_prefix[k] + (piece - P.whole[k]);
        const size_t slot_row = static_cast<size_t>(slot) * kPartRows + t * kQ + r;
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
        float* pml = P.part + static_cast<size_t>(P.parts) * kPartRows * kHD + slot_row * 2;
        pml[0] = have_o ? m : -INFINITY;
        pml[1] = have_o ? l : 0.f;
      } else if (have_o) {
        const int row = q0 + t * kQ + r;
        if (row < q1) {
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

// Merges the parts of each cut unit: per query row O = sum_c 2^(m_c - M) O_c,
// l = sum_c 2^(m_c - M) l_c with M = max_c m_c over the unit's parts in key
// order, and writes O / l as bf16.  A block covers 16 rows x 16 groups of 4
// columns of one cut unit.
__global__ void __launch_bounds__(256) attn_combine_kernel(const __grid_constant__ TcAttnParams P,
                                                           __nv_bfloat16* __restrict__ out) {
  constexpr int kBlocksPerUnit = kPartRows / kCombineRows;
  const int cut = static_cast<int>(blockIdx.x) / kBlocksPerUnit;
  const int rblk = static_cast<int>(blockIdx.x) % kBlocksPerUnit;
  int k = 0;
  while (k + 1 < P.n_slots && P.split_prefix[k + 1] <= cut) ++k;
  const int local = cut - P.split_prefix[k];  // cut unit of slot k
  const int u = P.whole[k] + local;
  const int row = rblk * kCombineRows + static_cast<int>(threadIdx.x) / 16;
  const int c4 = static_cast<int>(threadIdx.x) % 16;
  const int h = u / P.items[k];
  const int q = P.qs0[k] + (u % P.items[k]) * kPartRows + row;
  if (q >= P.qs1[k]) return;
  const int first = P.part_prefix[k] + local * P.chunks[k];
  const int nparts = (P.nkv[k] + P.clen[k] - 1) / P.clen[k];
  const float* ml = P.part + static_cast<size_t>(P.parts) * kPartRows * kHD;
  float M = -INFINITY;
  for (int c = 0; c < nparts; ++c) M = fmaxf(M, ml[(static_cast<size_t>(first + c) * kPartRows + row) * 2]);
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  float L = 0.f;
  for (int c = 0; c < nparts; ++c) {
    const size_t sr = static_cast<size_t>(first + c) * kPartRows + row;
    const float w = ex2_approx(ml[sr * 2] - M);
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

int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// Fills the piece table of P (segments with tokens, longest units first).
// whole_units: one piece per unit, nothing cut.
bool plan_pieces(TcAttnParams* P, int M, int heads, const Segments& seg, int num_sms, bool whole_units) {
  const int G = num_sms > 0 ? num_sms : 148;
  struct S {
    int g, q0, q1, items, nkv, whole, chunks, clen, pieces, parts, cut;
  };
  std::vector<S> v;
  for (int g = 0; g < seg.n; ++g) {
    const int len = seg.start[g + 1] - seg.start[g];
    if (len < 0 || seg.start[g] < 0 || seg.start[g + 1] > M) return false;
    S s;
    s.g = g;
    s.q0 = seg.queries ? seg.q_begin[g] : seg.start[g];
    s.q1 = seg.queries ? seg.q_end[g] : seg.start[g + 1];
    if (s.q0 < seg.start[g] || s.q1 > seg.start[g + 1] || s.q1 < s.q0) return false;
    if (s.q1 == s.q0) continue;
    s.items = ceil_div(s.q1 - s.q0, kPartRows);
    s.nkv = ceil_div(len, kKV);
    const long long units = static_cast<long long>(heads) * s.items;
    if (units * s.nkv > (1LL << 30)) return false;
    const int U = static_cast<int>(units);
    const int rest = U % G;
    int c = rest > 0 && !whole_units ? std::min(std::min(G / rest, kMaxChunks), s.nkv) : 1;
    s.whole = c >= 2 ? U - rest : U;
    s.clen = c >= 2 ? ceil_div(s.nkv, c) : s.nkv;
    s.chunks = c >= 2 ? ceil_div(s.nkv, s.clen) : 1;  // parts per cut unit (none empty)
    s.cut = U - s.whole;
    s.parts = s.cut * s.chunks;
    s.pieces = s.whole + s.parts;
    v.push_back(s);
  }
  std::stable_sort(v.begin(), v.end(), [](const S& a, const S& b) { return a.nkv > b.nkv; });
  P->n_slots = static_cast<int>(v.size());
  int pieces = 0, parts = 0, cuts = 0;
  for (int i = 0; i < P->n_slots; ++i) {
    const S& s = v[i];
    P->s0[i] = seg.start[s.g];
    P->s1[i] = seg.start[s.g + 1];
    P->qs0[i] = s.q0;
    P->qs1[i] = s.q1;
    P->items[i] = s.items;
    P->nkv[i] = s.nkv;
    P->whole[i] = s.whole;
    P->chunks[i] = s.chunks;
    P->clen[i] = s.clen;
    P->piece_prefix[i] = pieces;
    P->part_prefix[i] = parts;
    P->split_prefix[i] = cuts;
    pieces += s.pieces;
    parts += s.parts;
    cuts += s.cut;
  }
  P->piece_prefix[P->n_slots] = pieces;
  P->part_prefix[P->n_slots] = parts;
  P->split_prefix[P->n_slots] = cuts;
  P->pieces = pieces;
  P->parts = parts;
  return true;
}

}  // namespace

size_t attention_partial_bytes(int M, int heads, const Segments& seg, int num_sms) {
  TcAttnParams P{};
  if (!plan_pieces(&P, M, heads, seg, num_sms, false)) return 0;
  return static_cast<size_t>(P.parts) * kPartRows * (kHD + 2) * sizeof(float);
}

size_t attention_partial_bytes_bound(int n_seg, int seg_len, int heads, int num_sms) {
  // A segment's parts: its cut units (fewer than the SMs) times the parts per
  // unit (at most SMs / cut units), so at most one part per SM.
  if (n_seg <= 0 || n_seg > kMaxSegments || seg_len <= 0 || heads <= 0) return 0;
  const int G = num_sms > 0 ? num_sms : 148;
  return static_cast<size_t>(G) * n_seg * kPartRows * (kHD + 2) * sizeof(float);
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
  P.heads = heads;
  P.scale_log2 = 1.4426950408889634f * 0.125f;  // log2(e) / sqrt(64)
  P.part = part;
  if (!plan_pieces(&P, M, heads, seg, num_sms, part == nullptr)) return cudaErrorInvalidValue;
  if (P.pieces == 0) return cudaSuccess;
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = ensure_smem_attr(attn_tc_kernel, kSmemBytes, attr_done);
  if (e != cudaSuccess) return e;
  attn_tc_kernel<<<P.pieces, kThreads, kSmemBytes, st>>>(qkv_map, static_cast<__nv_bfloat16*>(out), P, err);
  int n = 1;
  const int cuts = P.split_prefix[P.n_slots];
  if (cuts > 0) {
    attn_combine_kernel<<<cuts * (kPartRows / kCombineRows), 256, 0, st>>>(P, static_cast<__nv_bfloat16*>(out));
    ++n;
  }
  if (launched) *launched = n;
  return cudaGetLastError();
}

}  // namespace revo
