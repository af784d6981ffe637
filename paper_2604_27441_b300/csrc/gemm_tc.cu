// Linear layers on the tcgen05 tensor cores: Y = epilogue(A W^T + b).
//
// Every Linear of the recovery network (tubelet embedding, qkv, attention
// output projection, MLP fc1/fc2, encoder->decoder map, pixel head) is a dense
// contraction over token rows.  A [M][K] (bf16 activations) and W [N][K] (bf16
// weights, the Linear [out][in] layout) are both K-major, so TMA copies 128 x 64
// and BN x 64 tiles with the 128-byte swizzle straight into the operand layout
// tcgen05.mma reads.  The accumulator (128 lanes x BN f32 columns) lives in
// TMEM, double-buffered so the epilogue of one tile overlaps the main loop of
// the next.  The epilogue adds the bias, applies GELU (the tanh form: within
// 4.8e-4 of the erf form, below the bf16 rounding of the output) and the bf16
// downcast in registers, stages 32-row chunks in 128-byte-swizzled shared
// memory and hands them to TMA: a bulk store, or for the residual layers a
// bulk f32 add-reduction into the residual stream (one rounding per element,
// exactly as x += y).
//
// The FP8 variant takes E4M3 operands (tcgen05 kind::f8f6f4, 128 elements =
// one 128-byte swizzle atom per stage row, so the pipeline is byte-for-byte the
// same) and multiplies each accumulator by its row's activation scale times its
// column's weight scale and adds the bias in one FMA.
//
// A second form runs 256-row tiles on a CTA pair (a two-CTA cluster on two
// SMs issuing one tcgen05.mma.cta_group::2 per K step; see gemm_tc_pair_kernel).
// The autotuner times both forms per shape; the results are bit-identical.
//
// Tile order: a persistent CTA takes tiles blockIdx.x, + gridDim.x, ...; tile
// t covers row block t / n_tiles and column block t % n_tiles, so the tiles in
// flight at once cover all the column blocks of a few row blocks: each A row
// block (activations, up to hundreds of MB for a large batch) is read from
// HBM once and its other column tiles hit L2, and W (weights, a few MB) stays
// in L2.  With the column-major order instead, fc1 at 70200 rows read A from
// HBM once per column tile (1.23 GB read for a 108 MB operand).
//
// Warp roles (320 threads, one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer (one thread)
//   warp 1      TMEM allocator + MMA issuer (one thread)
//   warps 2..9  epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (tile rows);
//               warps 2..5 take the left half of the tile's columns, 6..9 the right.
#include <algorithm>

#include "common.cuh"
#include "layernorm_row.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // 64 bf16 = one 128-byte swizzle atom per row
constexpr int kBK8 = 128;  // 128 E4M3 = the same 128 bytes
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kOutChunkBytes = 32 * 128;  // 32 rows x 128 B staging per epilogue warp

// TMEM columns for a double-buffered accumulator of width bn (the allocation
// is a power of two).
constexpr int tmem_cols_for(int bn) { return 2 * bn <= 256 ? 256 : 512; }

// BN = 192 (f32 epilogues only: two halves of three 32-column chunks) gives
// N = 768 four tiles per row block instead of three: fc2 of an encoder block
// alone takes 20.6 us instead of 22.6 (116 of 148 SMs busy instead of 87).
// With two models in flight the SM-time is the same (116 x 0.75 vs 87 x 1) and
// the other model's kernels get fewer SMs, so the network's autotuner, which
// times each GEMM alone, does not offer it; revo_op_linear does.
template <int BN>
struct TcGemmCfg {
  static_assert(BN == 128 || BN == 192 || BN == 256, "tile width");
  static constexpr int kStages = (BN == 128) ? 6 : 4;
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kTmemCols = tmem_cols_for(BN);
  static constexpr int kSmemBytes =
      1024 /*align slack*/ + kStages * kStageBytes + kEpiWarps * kOutChunkBytes + 256 /*barriers*/;
};

// Writes this thread's 128-byte row (eight 16-byte pieces) into a 32 x 128 B
// chunk with the 128-byte swizzle TMA expects: piece k of row i sits at k ^ (i % 8).
REVO_DEVI void stage_row(uint8_t* chunk, int row, const uint4 (&pieces)[8]) {
  uint8_t* base = chunk + row * 128;
#pragma unroll
  for (int k = 0; k < 8; ++k) *reinterpret_cast<uint4*>(base + ((k ^ (row & 7)) << 4)) = pieces[k];
}

// The epilogue works on 16 packed pairs (columns 2i, 2i + 1) so that each
// multiply, add and FMA issues once per two values; every operation rounds
// exactly as its scalar form would.

// v[i] = v[i] * (rs * cs[col + i]) + b[col + i] in one rounding (FP8
// dequantisation -- token scale x channel scale -- fused with the bias).
REVO_DEVI void scales_bias(uint64_t (&v)[16], float rs, const float* __restrict__ cs, const float* __restrict__ bias,
                           int col) {
  const float4* c4 = reinterpret_cast<const float4*>(cs + col);
  const float4* b4 = reinterpret_cast<const float4*>(bias + col);
  const uint64_t rs2 = pk2(rs, rs);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 c = __ldg(c4 + i);
    const float4 b = bias ? __ldg(b4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    v[2 * i] = fma2(v[2 * i], mul2(rs2, pk2(c.x, c.y)), pk2(b.x, b.y));
    v[2 * i + 1] = fma2(v[2 * i + 1], mul2(rs2, pk2(c.z, c.w)), pk2(b.z, b.w));
  }
}

REVO_DEVI void add_bias(uint64_t (&v)[16], const float* __restrict__ bias, int col) {
  if (bias == nullptr) return;
  const float4* b4 = reinterpret_cast<const float4*>(bias + col);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 b = __ldg(b4 + i);
    v[2 * i] = add2(v[2 * i], pk2(b.x, b.y));
    v[2 * i + 1] = add2(v[2 * i + 1], pk2(b.z, b.w));
  }
}

// gelu_tanh on a pair: the same operations as the scalar form, paired.
REVO_DEVI uint64_t gelu_tanh2(uint64_t x) {
  const uint64_t u = mul2(x, fma2(mul2(x, x), pk2(0.0356774081363001f, 0.0356774081363001f),
                                   pk2(0.7978845608028654f, 0.7978845608028654f)));
  const uint64_t hx = mul2(pk2(0.5f, 0.5f), x);
  float u0, u1;
  unpk2(u, u0, u1);
  return fma2(hx, pk2(tanh_approx(u0), tanh_approx(u1)), hx);
}

REVO_DEVI uint32_t pack_bf16_pair(uint64_t v) {
  float lo, hi;
  unpk2(v, lo, hi);
  return pack_bf16x2(lo, hi);
}

// kEpiResidLn with EpiAux mode 2 (E4M3 LayerNorm output): a kernel template
// argument only, chosen by launch_gemm_tc from the mode.
constexpr int kEpiResidLn8 = 5;
__host__ __device__ constexpr bool epi_resid(int epi) { return epi == kEpiResidF32 || epi == kEpiResidLn || epi == kEpiResidLn8; }
__host__ __device__ constexpr bool epi_ln(int epi) { return epi == kEpiResidLn || epi == kEpiResidLn8; }

// One epilogue chunk: 32 rows (this warp's lanes) x 128 bytes of output
// (32 f32 columns or 64 bf16 columns) starting at tile column `c0`.
// The position embedding's values at columns q .. q + 31 of a part for an
// integer position beyond the table (a large temporal distance): the same
// float32 sincosf of pos * w_i the table holds.  Out of line: rarely taken.
__device__ __noinline__ void pe_chunk_computed(const EpiAux& aux, int pos, int q, float* e) {
  const int half = aux.pe_part / 2;
  for (int w = 0; w < 32; ++w) {
    const int i = (q + w) % half;
    float sv, cv;
    sincosf(static_cast<float>(pos) * __ldg(aux.pe_omega + i), &sv, &cv);
    e[w] = q + w < half ? sv : cv;
  }
}

// kEpiF32Pe: adds the position embedding of a row at position d = {tau,
// patch row << 16 | patch column} at columns col .. col + 31 (one part of it)
// to the 16 packed pairs v.
REVO_DEVI void add_pe_chunk(uint64_t (&v)[16], const EpiAux& aux, int2 d, int col) {
  const int which = col / aux.pe_part;
  const int q = col - which * aux.pe_part;
  const int pos = which == 0 ? d.x : which == 1 ? (d.y >> 16) : (d.y & 0xFFFF);
  if (pos >= 0 && pos < aux.pe_rows) {
    const float4* src = reinterpret_cast<const float4*>(aux.pe_tab + static_cast<size_t>(pos) * aux.pe_part + q);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float4 t = __ldg(src + k);
      v[2 * k] = add2(v[2 * k], pk2(t.x, t.y));
      v[2 * k + 1] = add2(v[2 * k + 1], pk2(t.z, t.w));
    }
  } else {
    float e[32];
    pe_chunk_computed(aux, pos, q, e);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = add2(v[i], pk2(e[2 * i], e[2 * i + 1]));
  }
}

// `pe_d`: the row's position (kEpiF32Pe only).  `release` (a shared::cluster
// barrier address, or 0): the accumulator buffer is handed back to the MMA
// warp there as soon as this chunk's TMEM columns are in registers (the last
// chunk of the warp's tile), before its arithmetic and store.
REVO_DEVI void release_accumulator(uint32_t release, int lane) {
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive_cluster(release);
}

template <int EPI, bool F8>
REVO_DEVI void epilogue_chunk(uint32_t taddr, const float* __restrict__ bias, int n0, int c0, uint8_t* chunk,
                              const CUtensorMap* map, int row0, int lane, float rs, const float* __restrict__ cs,
                              const EpiAux& aux, int2 pe_d, uint32_t release = 0, int bufs = 1) {
  uint4 pieces[8];
  if (EPI == kEpiF32 || EPI == kEpiF32Pe || epi_resid(EPI)) {
    uint32_t r[32];
    tmem_ld32(taddr + c0, r);
    tmem_wait_ld();
    if (release) release_accumulator(release, lane);
    uint64_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = pk2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    if (F8)
      scales_bias(v, rs, cs, bias, n0 + c0);
    else
      add_bias(v, bias, n0 + c0);
    if (EPI == kEpiF32Pe) add_pe_chunk(v, aux, pe_d, n0 + c0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float a, b, c, d;
      unpk2(v[2 * k], a, b);
      unpk2(v[2 * k + 1], c, d);
      pieces[k] = make_uint4(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c), __float_as_uint(d));
    }
  } else {
    uint32_t rr[2][32];
    tmem_ld32(taddr + c0, rr[0]);
    tmem_ld32(taddr + c0 + 32, rr[1]);
    tmem_wait_ld();
    if (release) release_accumulator(release, lane);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint64_t v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = pk2(__uint_as_float(rr[half][2 * i]), __uint_as_float(rr[half][2 * i + 1]));
      if (F8)
        scales_bias(v, rs, cs, bias, n0 + c0 + 32 * half);
      else
        add_bias(v, bias, n0 + c0 + 32 * half);
      if (EPI == kEpiGeluBf16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = gelu_tanh2(v[i]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        pieces[4 * half + k] = make_uint4(pack_bf16_pair(v[4 * k]), pack_bf16_pair(v[4 * k + 1]),
                                          pack_bf16_pair(v[4 * k + 2]), pack_bf16_pair(v[4 * k + 3]));
    }
  }
  // The staging chunk is free once the bulk copy that last used it has read it
  // (with two chunks taken in turn: all but the most recent copy).
  if (lane == 0) {
    if (bufs == 2)
      bulk_wait_read1();
    else
      bulk_wait_read0();
  }
  __syncwarp();
  stage_row(chunk, lane, pieces);
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) {
    if (epi_resid(EPI))
      tma_reduce_add_2d(map, chunk, n0 + c0, row0);
    else
      tma_store_2d(map, chunk, n0 + c0, row0);
    bulk_commit();
  }
}

// The rows of one completed row block, R at a time per epilogue warp (warp e
// takes rows e, e + 8, ...), NV float4 of a row per lane.
template <int OUT, int NV, int R>
REVO_DEVI void ln_block_rows(const EpiAux& ln, int m0, int rows, int N, int e, int lane) {
  for (int r = e; r < rows; r += R * kEpiWarps)
    ln_rows<OUT, true, NV, R>(ln.x, ln.g, ln.b, ln.out, ln.row_scale, m0 + r, kEpiWarps, m0 + rows, N, lane);
}

// kEpiResidLn, after the epilogue warps have added a tile into rows
// [m0, m0 + 128) of x: each warp waits for its reduce-adds to complete, fences
// (a proxy fence -- the adds came through the async proxy -- then a gpu-scope
// fence) and arrives on ln_in; warp 0 then counts the tile for the row block
// (after a gpu-scope fence: the count publishes every warp's adds) and
// publishes on ln_out whether this CTA completed it (all n_tiles column tiles
// added); that CTA normalises the rows, reading x through L2.  Every wait is
// bounded (a failed wait leaves the rows alone; the error word reports it).
// `phase`: the parity of this CTA's counted tiles, flipped here.
template <int OUT>
REVO_DEVI void ln_after_tile(const EpiAux& ln, int m0, int M, int N, int n_tiles, int e, int lane, int* flag,
                             uint64_t* ln_in, uint64_t* ln_out, uint32_t& phase, int* err) {
  if (m0 >= M) return;  // a pair tile's rows past the end: no block, no count (same in every warp)
  if (lane == 0) {
    bulk_wait_all();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    mbar_arrive(ln_in);
  }
  int ok = 1;
  if (e == 0 && lane == 0) {
    int last = 0;
    if (mbar_wait(ln_in, phase, err, kDevTimeoutEpilogue)) {
      const int rb = m0 / kBM;
      __threadfence();
      last = atomicAdd(&ln.counters[rb], 1) == n_tiles - 1;
      if (last) ln.counters[rb] = 0;
    }
    *flag = last;
    mbar_arrive(ln_out);
  }
  if (lane == 0) ok = mbar_wait(ln_out, phase, err, kDevTimeoutEpilogue) ? 1 : 0;
  phase ^= 1u;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  if (ok && *reinterpret_cast<volatile int*>(flag)) {
    __threadfence();
    const int rows = min(kBM, M - m0);
    if (N <= 512)
      ln_block_rows<OUT, 4, 2>(ln, m0, rows, N, e, lane);
    else
      ln_block_rows<OUT, kLnMaxVec, 1>(ln, m0, rows, N, e, lane);
  }
}

template <int BN, int EPI, bool F8>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const float* __restrict__ bias,
                   const float* __restrict__ row_scale, const float* __restrict__ col_scale, int M, int N, int K,
                   int* err, const __grid_constant__ EpiAux ln) {
  using Cfg = TcGemmCfg<BN>;
  constexpr int S = Cfg::kStages;
  constexpr uint32_t kIdesc = F8 ? idesc_e4m3(kBM, BN) : idesc_bf16(kBM, BN);
  constexpr int kKe = F8 ? kBK8 : kBK;  // K elements per stage
  constexpr int kChunkCols = (EPI == kEpiF32 || EPI == kEpiF32Pe || epi_resid(EPI)) ? 32 : 64;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S * Cfg::kABytes;
  uint8_t* sOut = sB + S * Cfg::kBBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sOut + kEpiWarps * kOutChunkBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* ln_flag = reinterpret_cast<int*>(tmem_slot + 1);  // kEpiResidLn: this CTA completed the row block
  uint64_t* ln_in = reinterpret_cast<uint64_t*>(tmem_slot + 2);  // 8-byte aligned: tmem_slot follows 8-byte barriers
  uint64_t* ln_out = ln_in + 1;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int m_tiles = (M + kBM - 1) / kBM;
  const int n_tiles = (N + BN - 1) / BN;
  const int num_tiles = m_tiles * n_tiles;
  const int num_kb = K / kKe;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmC);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);
    }
    mbar_init(ln_in, kEpiWarps);
    mbar_init(ln_out, 1);
    fence_mbarrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
        const int m0 = (tile / n_tiles) * kBM;
        const int n0 = (tile % n_tiles) * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, kDevTimeoutProducer)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
          const int kx = (ln.kperm ? embed_kblock(kb) : kb) * kKe;
          tma_load_2d(sA + stage * Cfg::kABytes, &tmA, kx, m0, &full[stage]);
          tma_load_2d(sB + stage * Cfg::kBBytes, &tmB, kx, n0, &full[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int t_local = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++t_local) {
        const int acc = t_local & 1;
        const uint32_t acc_phase = (t_local >> 1) & 1;
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, err, kDevTimeoutMma)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&full[stage], phase, err, kDevTimeoutMma)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_lo = sw128_lo(smem_u32(sA + stage * Cfg::kABytes));
          const uint32_t b_lo = sw128_lo(smem_u32(sB + stage * Cfg::kBBytes));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per stage
            if (F8)
              mma_f8_hl(d_tmem, a_lo + kk * 2, kSw128Hi, b_lo + kk * 2, kSw128Hi, kIdesc, (kb | kk) != 0 ? 1u : 0u);
            else
              mma_f16_hl(d_tmem, a_lo + kk * 2, kSw128Hi, b_lo + kk * 2, kSw128Hi, kIdesc, (kb | kk) != 0 ? 1u : 0u);
          }
          mma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[acc]);
      }
    }
  } else {
    const int e = warp - 2;
    const int q = warp & 3;
    const int half = e >> 2;
    uint8_t* chunk = sOut + e * kOutChunkBytes;
    int t_local = 0;
    uint32_t ln_phase = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++t_local) {
      const int acc = t_local & 1;
      const uint32_t acc_phase = (t_local >> 1) & 1;
      if (!mbar_wait(&tfull[acc], acc_phase, err, kDevTimeoutEpilogue)) break;
      tc_fence_after();
      const int m0 = (tile / n_tiles) * kBM;
      const int n0 = (tile % n_tiles) * BN;
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + acc * BN;
      const int my_row = m0 + q * 32 + lane;
      const float rs = (F8 && my_row < M) ? __ldg(row_scale + my_row) : 0.f;
      const int2 pe_d = (EPI == kEpiF32Pe && my_row < M) ? __ldg(ln.pe_pos + my_row) : make_int2(0, 0);
      const uint32_t rel = smem_u32(&tempty[acc]);
      bool released = false;
#pragma unroll 1
      for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += kChunkCols) {
        if (n0 + c0 >= N) break;
        const bool last = c0 + kChunkCols >= (half + 1) * (BN / 2) || n0 + c0 + kChunkCols >= N;
        epilogue_chunk<EPI, F8>(taddr, bias, n0, c0, chunk, &tmC, m0 + q * 32, lane, rs, col_scale, ln, pe_d,
                                last ? rel : 0u);
        released = released || last;
      }
      if (!released) release_accumulator(rel, lane);
      if constexpr (epi_ln(EPI))
        ln_after_tile<EPI == kEpiResidLn8 ? 2 : 1>(ln, m0, M, N, n_tiles, e, lane, ln_flag, ln_in, ln_out, ln_phase,
                                                   err);
    }
    if (lane == 0) bulk_wait_all();
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

// ---- CTA-pair form: a cluster of two CTAs computes 256 x BN output tiles with
// tcgen05.mma.cta_group::2 (M = 256).  Each CTA holds 128 rows of A and BN/2
// rows of W per stage (32 KB at BN = 256 instead of 48 KB), so the same shared
// memory holds 6 stages instead of 4 and every SM reads a third less operand
// data per FLOP; rank 0 issues the MMAs for both SMs (half the issue work per
// SM).  Both CTAs' loads complete on rank 0's stage barrier; the MMA commits
// release the stage in both CTAs and hand each CTA's epilogue its 128
// accumulator rows (its own TMEM, same column address); the epilogue warps of
// both CTAs free an accumulator buffer on rank 0's barrier.
// Staging chunks per epilogue warp (two in turn measured slower: the fifth
// pipeline stage they cost is worth more, fc2 at the tick's rows 225 -> 235 us).
constexpr int kPairOutBufs = 1;

template <int BN>
struct TcGemmPairCfg {
  static constexpr int kABytes = kBM * 128;         // 128 rows x 128 B of K
  static constexpr int kBBytes = (BN / 2) * 128;    // this CTA's half of the W rows
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = (192 * 1024) / kStageBytes;  // BN 256: 6, BN 128: 8
  static constexpr int kTmemCols = tmem_cols_for(BN);
  static constexpr int kSmemBytes = 1024 /*align slack*/ + kStages * kStageBytes +
                                    kEpiWarps * kPairOutBufs * kOutChunkBytes + 256 /*barriers*/;
};

template <int BN, int EPI, bool F8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm_tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const float* __restrict__ bias,
                        const float* __restrict__ row_scale, const float* __restrict__ col_scale, int M, int N, int K,
                        int* err, const __grid_constant__ EpiAux ln) {
  using Cfg = TcGemmPairCfg<BN>;
  constexpr int S = Cfg::kStages;
  constexpr uint32_t kIdesc = F8 ? idesc_e4m3(2 * kBM, BN) : idesc_bf16(2 * kBM, BN);
  constexpr int kKe = F8 ? kBK8 : kBK;
  constexpr int kChunkCols = (EPI == kEpiF32 || EPI == kEpiF32Pe || epi_resid(EPI)) ? 32 : 64;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S * Cfg::kABytes;
  uint8_t* sOut = sB + S * Cfg::kBBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sOut + kEpiWarps * kPairOutBufs * kOutChunkBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* ln_flag = reinterpret_cast<int*>(tmem_slot + 1);  // kEpiResidLn: this CTA completed the row block
  uint64_t* ln_in = reinterpret_cast<uint64_t*>(tmem_slot + 2);  // 8-byte aligned: tmem_slot follows 8-byte barriers
  uint64_t* ln_out = ln_in + 1;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int pair = static_cast<int>(blockIdx.x) >> 1;
  const int npairs = static_cast<int>(gridDim.x) >> 1;
  const int m_tiles = (M + 2 * kBM - 1) / (2 * kBM);
  const int n_tiles = (N + BN - 1) / BN;
  const int num_tiles = m_tiles * n_tiles;
  const int num_kb = K / kKe;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmC);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);   // rank 0's: its producer's arrival + both CTAs' bytes
      mbar_init(&empty[s], 1);  // one multicast commit per use
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2 * kEpiWarps);  // rank 0's: the epilogue warps of both CTAs
    }
    mbar_init(ln_in, kEpiWarps);  // this CTA's own epilogue warps
    mbar_init(ln_out, 1);
    fence_mbarrier_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any remote completion
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t full0 = mapa_shared(smem_u32(&full[0]), 0);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int tile = pair; tile < num_tiles && ok; tile += npairs) {
        const int m0 = (tile / n_tiles) * (2 * kBM) + kBM * static_cast<int>(rank);
        const int n0 = (tile % n_tiles) * BN + (BN / 2) * static_cast<int>(rank);
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, kDevTimeoutProducer)) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_arrive_expect_tx(&full[stage], 2 * Cfg::kStageBytes);
          const uint32_t bar = full0 + stage * static_cast<uint32_t>(sizeof(uint64_t));
          const int kx = (ln.kperm ? embed_kblock(kb) : kb) * kKe;
          tma_load_2d_pair(sA + stage * Cfg::kABytes, &tmA, kx, m0, bar);
          tma_load_2d_pair(sB + stage * Cfg::kBBytes, &tmB, kx, n0, bar);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int t_local = 0;
      bool ok = true;
      for (int tile = pair; tile < num_tiles && ok; tile += npairs, ++t_local) {
        const int acc = t_local & 1;
        const uint32_t acc_phase = (t_local >> 1) & 1;
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, err, kDevTimeoutMma)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&full[stage], phase, err, kDevTimeoutMma)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_lo = sw128_lo(smem_u32(sA + stage * Cfg::kABytes));
          const uint32_t b_lo = sw128_lo(smem_u32(sB + stage * Cfg::kBBytes));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per stage
            if (F8)
              mma_f8_pair(d_tmem, a_lo + kk * 2, kSw128Hi, b_lo + kk * 2, kSw128Hi, kIdesc, (kb | kk) != 0 ? 1u : 0u);
            else
              mma_f16_pair(d_tmem, a_lo + kk * 2, kSw128Hi, b_lo + kk * 2, kSw128Hi, kIdesc,
                           (kb | kk) != 0 ? 1u : 0u);
          }
          mma_commit_pair(&empty[stage], 0x3);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit_pair(&tfull[acc], 0x3);
      }
    }
  } else {
    const int e = warp - 2;
    const int q = warp & 3;
    const int half = e >> 2;
    uint8_t* chunks = sOut + e * kPairOutBufs * kOutChunkBytes;
    int cc = 0;  // chunks this warp has staged
    int t_local = 0;
    uint32_t ln_phase = 0;
    for (int tile = pair; tile < num_tiles; tile += npairs, ++t_local) {
      const int acc = t_local & 1;
      const uint32_t acc_phase = (t_local >> 1) & 1;
      if (!mbar_wait(&tfull[acc], acc_phase, err, kDevTimeoutEpilogue)) break;
      tc_fence_after();
      const int m0 = (tile / n_tiles) * (2 * kBM) + kBM * static_cast<int>(rank);
      const int n0 = (tile % n_tiles) * BN;
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + acc * BN;
      const int my_row = m0 + q * 32 + lane;
      const float rs = (F8 && my_row < M) ? __ldg(row_scale + my_row) : 0.f;
      const int2 pe_d = (EPI == kEpiF32Pe && my_row < M) ? __ldg(ln.pe_pos + my_row) : make_int2(0, 0);
      const uint32_t rel = mapa_shared(smem_u32(&tempty[acc]), 0);
      bool released = false;
#pragma unroll 1
      for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2) && m0 + q * 32 < M; c0 += kChunkCols) {
        if (n0 + c0 >= N) break;
        const bool last = c0 + kChunkCols >= (half + 1) * (BN / 2) || n0 + c0 + kChunkCols >= N;
        epilogue_chunk<EPI, F8>(taddr, bias, n0, c0, chunks + (cc % kPairOutBufs) * kOutChunkBytes, &tmC, m0 + q * 32,
                                lane, rs, col_scale, ln, pe_d, last ? rel : 0u, kPairOutBufs);
        ++cc;
        released = released || last;
      }
      if (!released) release_accumulator(rel, lane);
      if constexpr (epi_ln(EPI))
        ln_after_tile<EPI == kEpiResidLn8 ? 2 : 1>(ln, m0, M, N, n_tiles, e, lane, ln_flag, ln_in, ln_out, ln_phase,
                                                   err);
    }
    if (lane == 0) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no CTA leaves while its peer's MMAs may read its shared memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
  }
}

}  // namespace

namespace {

// ---- The tubelet embedding as an implicit GEMM (the Conv3d of Section 3.4.1
// with kernel = stride = (T, 16, 16), bias, plus the (tau, row, column)
// embedding in the epilogue).  No token matrix is stored.  A loader warp
// brings the tile's pixels in by TMA bulk copies: for each pixel group (frame t
// of the slot, patch-row quad yq), one copy per patch row of every run of
// tokens that share a patch row -- the run's pixels are one contiguous span of
// a frame row -- into a raw ring (two RGB or four depth groups).  Eight producer warps (two threads
// per tile row, i.e. per token) take the group's bytes into registers, hand
// the raw stage back, and for each channel write the token's 64 K elements
// (patch rows 4 yq .. 4 yq + 3) as bf16 into the 128-byte-swizzled A stage,
// normalised exactly as the assemble kernel does, then fence the writes into
// the async proxy and arrive on the stage's barrier; TMA streams the W tile
// onto the same barrier; one thread issues tcgen05.mma; four epilogue warps add
// bias and position embedding and store the float32 rows by TMA.  Each
// token's position is also written out for the encoder->decoder Linear.  The K
// blocks of the weights' (t, c, y, x) order are taken channel blocks of a
// pixel group together (embed_kblock), so each pixel is copied and converted
// from one load for its three channels; the assemble + GEMM path takes the
// same order (EpiAux::kperm) and gives the same bits.  A tile with a frame row
// that is not 16-byte aligned skips the copies and its producers read the
// frames directly.
//
// Warp roles (480 threads): warp 0 TMA (W), warp 1 TMEM allocator + MMA
// issuer, warps 2..5 epilogue (TMEM lanes 32 (w % 4) .. +31, every column),
// warps 6..13 operand producers (two threads per tile row), warp 14 the
// raw-pixel loader.
constexpr int kEmbEpiWarps = 4;
constexpr int kEmbCvtWarps = 8;  // two per row: 256 threads
constexpr int kEmbRawWarp = 2 + kEmbEpiWarps + kEmbCvtWarps;  // the raw-pixel loader
constexpr int kEmbThreads = 32 * (kEmbRawWarp + 1);
// The raw-pixel ring: 64 KB holding pixel groups of a tile (4 patch rows x 128
// tokens x 48 B RGB or 32 B depth): 2 RGB groups (3 K blocks each) or 4 depth
// groups (1 K block each), enough to cover the copies' latency.
constexpr int kEmbRawRing = 4 * kBM * 4 * 32;
constexpr int kEmbRawMaxStages = 4;
REVO_DEVI int embed_raw_stages(int C) { return C == 3 ? 2 : 4; }

template <int BN>
struct EmbedCfg {
  static constexpr int kStages = (BN == 128) ? 4 : 3;
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kTmemCols = tmem_cols_for(BN);
  static constexpr int kSmemBytes = 1024 /*align slack*/ + kStages * (kABytes + kBBytes) +
                                    kEmbEpiWarps * kOutChunkBytes + kEmbRawRing + 256 /*barriers*/;
};
static_assert(EmbedCfg<256>::kSmemBytes <= 232448 && EmbedCfg<128>::kSmemBytes <= 232448, "shared memory per CTA");

// The request, slot and patch of batch row `row` (false past the last row).
REVO_DEVI bool embed_token(const EmbedParams& ep, int row, int& req, int& s, int& ty, int& tx) {
  if (row < 0 || row >= ep.seg_start[ep.n]) return false;
  int lo = 0, hi = ep.n - 1;  // the last request whose rows start at or before `row`
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ep.seg_start[mid] <= row) lo = mid; else hi = mid - 1;
  }
  const int wp = ep.wp[lo], hw = ep.hp[lo] * wp;
  const int local = row - ep.seg_start[lo];
  req = lo;
  s = local / hw;
  const int rem = local - s * hw;
  ty = rem / wp;
  tx = rem - ty * wp;
  return true;
}

REVO_DEVI const AssembleArgs* embed_job(const EmbedParams& ep, int req) {
  return reinterpret_cast<const AssembleArgs*>(ep.jobs + static_cast<size_t>(req) * ep.stride);
}

// One token's source: its patch origin in each of its slot's T (<= 2) frames.
struct EmbedRow {
  const uint8_t* base[2];
  size_t pitch[2];
  float mu, inv;  // depth statistics (C == 1)
  bool valid, aligned;
};

REVO_DEVI EmbedRow embed_row(const EmbedParams& ep, int row) {
  EmbedRow r{};
  int req, s, ty, tx;
  if (!embed_token(ep, row, req, s, ty, tx)) return r;
  const AssembleArgs* a = embed_job(ep, req);
  const int colb = tx * (ep.C == 3 ? 48 : 32);
  uintptr_t bits = 0;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    if (t >= ep.T) break;
    const int f = s * ep.T + t;
    const size_t pitch = a->pitch[f];
    r.pitch[t] = pitch;
    r.base[t] = static_cast<const uint8_t*>(a->frames[f]) + static_cast<size_t>(ty) * 16 * pitch + colb;
    bits |= reinterpret_cast<uintptr_t>(r.base[t]) | pitch;
  }
  if (ep.C == 1) {
    r.mu = a->mu_sigma[0];
    r.inv = 1.f / a->mu_sigma[1];
  }
  r.aligned = (bits & 15u) == 0;
  r.valid = true;
  return r;
}

// Producer work is split into two threads per row (pieces 4h .. 4h + 3 of
// the row's 8) and into a load step and a convert step, so that the loads of
// the next K block are in flight while this one is converted.
constexpr int kEmbPieces = 4;

// The raw bytes of this thread's 4 pieces for pixel group g = (frame t of the
// slot, patch-row quad yq) = 4 t + yq: 24 bytes (8 RGB pixels, all three
// channels) or 16 bytes (8 depth samples) each, as 6 or 4 words.  The K block
// of channel c of the group holds elements ((t C + c) 4 + yq) * 64 .. +63:
// patch rows 4*yq .. 4*yq + 3, 16 pixels each; piece j (8 elements) is patch
// row 4*yq + j/2, pixels 8*(j%2) .. +7.  Byte loads when a row is not 16-byte aligned.
struct EmbedRaw {
  uint32_t w[kEmbPieces][6];
};

REVO_DEVI void embed_load(const EmbedRow& er, int g, int C, int h, EmbedRaw& raw) {
  if (!er.valid) return;
  const int t = g >> 2, yq = g & 3;
  const size_t pitch = t == 0 ? er.pitch[0] : er.pitch[1];  // no dynamic index: er stays in registers
  const uint8_t* rowp = (t == 0 ? er.base[0] : er.base[1]) + static_cast<size_t>(4 * yq) * pitch;
#pragma unroll
  for (int jj = 0; jj < kEmbPieces; ++jj) {
    const int j = kEmbPieces * h + jj;
    const uint8_t* p = rowp + static_cast<size_t>(j >> 1) * pitch + (j & 1) * (C == 3 ? 24 : 16);
    if (C == 3) {
      if (er.aligned) {
        // 24 bytes at offset 0 or 8 (mod 16) of a 16-byte aligned row: one
        // 16-byte and one 8-byte load.
        if ((j & 1) == 0) {
          const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
          const uint2 b = __ldg(reinterpret_cast<const uint2*>(p + 16));
          raw.w[jj][0] = a.x, raw.w[jj][1] = a.y, raw.w[jj][2] = a.z, raw.w[jj][3] = a.w;
          raw.w[jj][4] = b.x, raw.w[jj][5] = b.y;
        } else {
          const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
          const uint4 b = __ldg(reinterpret_cast<const uint4*>(p + 8));
          raw.w[jj][0] = a.x, raw.w[jj][1] = a.y;
          raw.w[jj][2] = b.x, raw.w[jj][3] = b.y, raw.w[jj][4] = b.z, raw.w[jj][5] = b.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i)
          raw.w[jj][i] = p[4 * i] | (p[4 * i + 1] << 8) | (p[4 * i + 2] << 16) | (static_cast<uint32_t>(p[4 * i + 3]) << 24);
      }
    } else {
      if (er.aligned) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
        raw.w[jj][0] = w.x, raw.w[jj][1] = w.y, raw.w[jj][2] = w.z, raw.w[jj][3] = w.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          raw.w[jj][i] = p[4 * i] | (p[4 * i + 1] << 8) | (p[4 * i + 2] << 16) | (static_cast<uint32_t>(p[4 * i + 3]) << 24);
      }
    }
  }
}

// Channel CH of the pieces as normalised bf16 (the channel is a template
// argument so that every byte index is fixed).
// The float bits of 2^23 + (byte `b` of `word`) (exact).
REVO_DEVI uint32_t magic_byte(uint32_t word, int b) {
  uint32_t bits;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(bits) : "r"(word), "r"(0x4B000000u), "r"(0x7650u | static_cast<uint32_t>(b)));
  return bits;
}

// The float bits of 2^23 + (16-bit half `hf` of `word`) (exact).
REVO_DEVI uint32_t magic_half(uint32_t word, int hf) {
  uint32_t bits;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(bits) : "r"(word), "r"(0x4B000000u), "r"(hf ? 0x7432u : 0x7410u));
  return bits;
}

// Channel CH of the pieces as normalised bf16 (the channel is a template
// argument so that every byte index is fixed): per pair of pixels, the two
// codes as floats (2^23 + b - 2^23, exact) and one packed FMA, each lane
// rounded as the assemble kernel's scalar fmaf.
template <int CH>
REVO_DEVI void rgb_pieces(const EmbedRaw& raw, float sc, float sh, uint4 (&pieces)[kEmbPieces]) {
  const uint64_t m2 = pk2(-8388608.f, -8388608.f), sc2 = pk2(sc, sc), sh2 = pk2(sh, sh);
#pragma unroll
  for (int j = 0; j < kEmbPieces; ++j) {
    uint32_t pw[4];
#pragma unroll
    for (int x = 0; x < 8; x += 2) {
      const int b0 = 3 * x + CH, b1 = 3 * (x + 1) + CH;
      const uint64_t f = add2(pk2(__uint_as_float(magic_byte(raw.w[j][b0 >> 2], b0 & 3)),
                                  __uint_as_float(magic_byte(raw.w[j][b1 >> 2], b1 & 3))), m2);
      pw[x >> 1] = pack_bf16_pair(fma2(f, sc2, sh2));
    }
    pieces[j] = make_uint4(pw[0], pw[1], pw[2], pw[3]);
  }
}

// Depth pieces: (d - mu) * (1 / sigma) per sample, as the assemble kernel's
// scalar operations, two samples per packed instruction.
REVO_DEVI void depth_pieces(const EmbedRaw& raw, float mu, float inv, uint4 (&pieces)[kEmbPieces]) {
  const uint64_t m2 = pk2(-8388608.f, -8388608.f), mu2 = pk2(-mu, -mu), inv2 = pk2(inv, inv);
#pragma unroll
  for (int j = 0; j < kEmbPieces; ++j) {
    uint32_t pw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t d = add2(pk2(__uint_as_float(magic_half(raw.w[j][i], 0)),
                                  __uint_as_float(magic_half(raw.w[j][i], 1))), m2);
      pw[i] = pack_bf16_pair(mul2(add2(d, mu2), inv2));
    }
    pieces[j] = make_uint4(pw[0], pw[1], pw[2], pw[3]);
  }
}

// Converts channel c of the raw pieces exactly as the assemble kernel does
// and writes them into row r of the A stage (128-byte swizzle: piece j of row
// r at 16-byte slot j ^ (r % 8)).  Rows past the batch are zero.
REVO_DEVI void embed_store(uint8_t* stage, int r, int h, const EmbedRow& er, const EmbedRaw& raw, int c, int C) {
  uint4 pieces[kEmbPieces];
  if (!er.valid) {
#pragma unroll
    for (int j = 0; j < kEmbPieces; ++j) pieces[j] = make_uint4(0u, 0u, 0u, 0u);
  } else if (C == 3) {
    if (c == 0)
      rgb_pieces<0>(raw, kRgbScaleR, kRgbShiftR, pieces);
    else if (c == 1)
      rgb_pieces<1>(raw, kRgbScaleG, kRgbShiftG, pieces);
    else
      rgb_pieces<2>(raw, kRgbScaleB, kRgbShiftB, pieces);
  } else {
    depth_pieces(raw, er.mu, er.inv, pieces);
  }
  uint8_t* base = stage + r * 128;
#pragma unroll
  for (int jj = 0; jj < kEmbPieces; ++jj) {
    const int j = kEmbPieces * h + jj;
    *reinterpret_cast<uint4*>(base + ((j ^ (r & 7)) << 4)) = pieces[jj];
  }
}

// This thread's 4 pieces of a pixel group from a raw stage ([4][128][bpt]):
// piece j is patch row j / 2 of the quad, pixels 8 (j % 2) .. + 7 (24 or 16
// bytes at a 16- or 8-byte aligned offset).
REVO_DEVI void embed_load_raw(const uint8_t* raw_stage, int r, int h, int bpt, bool valid, EmbedRaw& raw) {
  if (!valid) return;
#pragma unroll
  for (int jj = 0; jj < kEmbPieces; ++jj) {
    const int j = kEmbPieces * h + jj;
    const uint8_t* p = raw_stage + ((j >> 1) * kBM + r) * bpt + (j & 1) * (bpt / 2);
    if (bpt == 48) {
      if ((j & 1) == 0) {
        const uint4 a = *reinterpret_cast<const uint4*>(p);
        const uint2 b = *reinterpret_cast<const uint2*>(p + 16);
        raw.w[jj][0] = a.x, raw.w[jj][1] = a.y, raw.w[jj][2] = a.z, raw.w[jj][3] = a.w;
        raw.w[jj][4] = b.x, raw.w[jj][5] = b.y;
      } else {
        const uint2 a = *reinterpret_cast<const uint2*>(p);
        const uint4 b = *reinterpret_cast<const uint4*>(p + 8);
        raw.w[jj][0] = a.x, raw.w[jj][1] = a.y;
        raw.w[jj][2] = b.x, raw.w[jj][3] = b.y, raw.w[jj][4] = b.z, raw.w[jj][5] = b.w;
      }
    } else {
      const uint4 a = *reinterpret_cast<const uint4*>(p);
      raw.w[jj][0] = a.x, raw.w[jj][1] = a.y, raw.w[jj][2] = a.z, raw.w[jj][3] = a.w;
    }
  }
}

// Bounded wait for the phase of the given parity while unwinding (copies still
// in flight when the CTA is about to exit); records nothing.
REVO_DEVI void mbar_drain_gemm(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (!mbar_try_wait(a, parity))
    if (clock64() - t0 > 20000000LL) return;
}

// One producer step: waits for the stage to be free, converts and stores this
// thread's pieces of channel c of its raw pixel group, fences them into the
// async proxy and arrives (once per warp) on the stage's barrier.
template <int S>
REVO_DEVI bool embed_step(const EmbedRow& er, const EmbedRaw& raw, int c, int r, int h, int C, uint8_t* sA,
                          uint64_t* full, uint64_t* empty, int& stage, uint32_t& phase, int* err, int lane) {
  if (!mbar_wait_warp(&empty[stage], phase ^ 1u, err, kDevTimeoutProducer, lane)) return false;
  embed_store(sA + stage * (kBM * kBK * 2), r, h, er, raw, c, C);
  fence_proxy_async_smem();  // the generic-proxy writes, visible to tcgen05.mma
  __syncwarp();
  if (lane == 0) mbar_arrive(&full[stage]);
  if (++stage == S) {
    stage = 0;
    phase ^= 1u;
  }
  return true;
}

template <int BN>
__global__ void __launch_bounds__(kEmbThreads, 1)
    embed_tc_kernel(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmC,
                    const float* __restrict__ bias, int M, int N, int K, int* err, const __grid_constant__ EpiAux pe,
                    const __grid_constant__ EmbedParams ep) {
  using Cfg = EmbedCfg<BN>;
  constexpr int S = Cfg::kStages;
  constexpr uint32_t kIdesc = idesc_bf16(kBM, BN);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S * Cfg::kABytes;
  uint8_t* sOut = sB + S * Cfg::kBBytes;
  uint8_t* sRaw = sOut + kEmbEpiWarps * kOutChunkBytes;  // the raw-pixel ring
  uint64_t* full = reinterpret_cast<uint64_t*>(sRaw + kEmbRawRing);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* raw_full = tempty + 2;                    // [raw stages] a pixel group landed
  uint64_t* raw_empty = raw_full + kEmbRawMaxStages;  // [raw stages] the producers hold it in registers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(raw_empty + kEmbRawMaxStages);
  int* raw_bulk = reinterpret_cast<int*>(tmem_slot + 1);  // [raw stages] 1: copied; 0: read the frames directly
  const int RS = embed_raw_stages(ep.C);
  const int raw_bytes = kBM * 4 * (ep.C == 3 ? 48 : 32);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int m_tiles = (M + kBM - 1) / kBM;
  const int n_tiles = (N + BN - 1) / BN;
  const int num_tiles = m_tiles * n_tiles;
  const int num_kb = K / kBK;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmC);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1 + kEmbCvtWarps);  // the W copy's arrival + one per producer warp
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEmbEpiWarps);
    }
    for (int a = 0; a < RS; ++a) {
      mbar_init(&raw_full[a], 1);
      mbar_init(&raw_empty[a], kEmbCvtWarps);
    }
    fence_mbarrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
        const int n0 = (tile % n_tiles) * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, kDevTimeoutProducer)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], Cfg::kBBytes);
          tma_load_2d(sB + stage * Cfg::kBBytes, &tmB, (ep.C == 3 ? embed_kblock(kb) : kb) * kBK, n0, &full[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int t_local = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++t_local) {
        const int acc = t_local & 1;
        const uint32_t acc_phase = (t_local >> 1) & 1;
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, err, kDevTimeoutMma)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&full[stage], phase, err, kDevTimeoutMma)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_lo = sw128_lo(smem_u32(sA + stage * Cfg::kABytes));
          const uint32_t b_lo = sw128_lo(smem_u32(sB + stage * Cfg::kBBytes));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // 4 x 32 bytes of K per stage
            mma_f16_hl(d_tmem, a_lo + kk * 2, kSw128Hi, b_lo + kk * 2, kSw128Hi, kIdesc, (kb | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[acc]);
      }
    }
  } else if (warp < 2 + kEmbEpiWarps) {
    const int e = warp - 2;
    const int q = warp & 3;
    uint8_t* chunk = sOut + e * kOutChunkBytes;
    int t_local = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++t_local) {
      const int acc = t_local & 1;
      const uint32_t acc_phase = (t_local >> 1) & 1;
      const int m0 = (tile / n_tiles) * kBM;
      const int n0 = (tile % n_tiles) * BN;
      const int my_row = m0 + q * 32 + lane;
      int2 pe_d = make_int2(0, 0);
      int req, s, ty, tx;
      if (embed_token(ep, my_row, req, s, ty, tx)) {
        pe_d = make_int2(embed_job(ep, req)->taus[s], (ty << 16) | tx);
        if (n0 == 0) ep.pe_pos[my_row] = pe_d;
      }
      if (!mbar_wait(&tfull[acc], acc_phase, err, kDevTimeoutEpilogue)) break;
      tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + acc * BN;
      const uint32_t rel = smem_u32(&tempty[acc]);
      bool released = false;
#pragma unroll 1
      for (int c0 = 0; c0 < BN && m0 + q * 32 < M; c0 += 32) {
        if (n0 + c0 >= N) break;
        const bool last = c0 + 32 >= BN || n0 + c0 + 32 >= N;
        epilogue_chunk<kEpiF32Pe, false>(taddr, bias, n0, c0, chunk, &tmC, m0 + q * 32, lane, 0.f, nullptr, pe,
                                         pe_d, last ? rel : 0u);
        released = released || last;
      }
      if (!released) release_accumulator(rel, lane);
    }
    if (lane == 0) bulk_wait_all();
  } else if (warp == kEmbRawWarp) {
    // Raw-pixel loader: for each tile and pixel group (frame t of the slot,
    // patch-row quad yq), TMA bulk copies bring the 4 pixel rows of every run
    // of the tile's tokens that share a patch row (one contiguous span of a
    // frame row) into raw stage rs: [4][128 tokens][bytes per token].  Lane l
    // owns tile rows l, l + 32, l + 64, l + 96 and issues the copies of the
    // runs that start there.  A tile with a row that is not 16-byte aligned is
    // marked for direct reads instead.
    const int bpt = ep.C == 3 ? 48 : 32;
    int rs = 0;
    uint32_t rph = 0;
    int armed = 0;  // groups armed so far (group i uses stage i % RS, phase i / RS)
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      const int m0 = (tile / n_tiles) * kBM;
      const int rows = min(kBM, M - m0);
      const uint8_t* src[4][2];
      size_t pitch[4][2];
      int run_r[4], run_len[4];
      bool aligned = true;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        run_len[q] = 0;
        run_r[q] = lane + 32 * q;
        int req, sl, ty, tx;
        if (run_r[q] < rows && embed_token(ep, m0 + run_r[q], req, sl, ty, tx) && (tx == 0 || run_r[q] == 0)) {
          run_len[q] = min(ep.wp[req] - tx, rows - run_r[q]);
          const AssembleArgs* a = embed_job(ep, req);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int f = sl * ep.T + (t < ep.T ? t : 0);
            pitch[q][t] = a->pitch[f];
            src[q][t] = static_cast<const uint8_t*>(a->frames[f]) + static_cast<size_t>(ty) * 16 * pitch[q][t] +
                        static_cast<size_t>(tx) * bpt;
            aligned = aligned && ((reinterpret_cast<uintptr_t>(src[q][t]) | pitch[q][t]) & 15u) == 0;
          }
        }
      }
      const bool bulk = __all_sync(0xffffffffu, aligned);
      const int groups = num_kb / ep.C;
      for (int g = 0; g < groups && ok; ++g) {
        if (!mbar_wait_warp(&raw_empty[rs], rph ^ 1u, err, kDevTimeoutProducer, lane)) {
          ok = false;
          break;
        }
        const int t = g >> 2, yq = g & 3;
        if (lane == 0) {
          raw_bulk[rs] = bulk ? 1 : 0;
          if (bulk)
            mbar_arrive_expect_tx(&raw_full[rs], static_cast<uint32_t>(rows * 4 * bpt));
          else
            mbar_arrive(&raw_full[rs]);
        }
        ++armed;
        __syncwarp();
        if (bulk) {
          uint8_t* dst = sRaw + rs * raw_bytes;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (run_len[q] == 0) continue;
            const uint8_t* p = t == 0 ? src[q][0] : src[q][1];
            const size_t pt = t == 0 ? pitch[q][0] : pitch[q][1];
#pragma unroll
            for (int y = 0; y < 4; ++y)
              bulk_load_1d(dst + (y * kBM + run_r[q]) * bpt, p + static_cast<size_t>(4 * yq + y) * pt,
                           static_cast<uint32_t>(run_len[q] * bpt), &raw_full[rs]);
          }
        }
        if (++rs == RS) {
          rs = 0;
          rph ^= 1u;
        }
      }
    }
    // No copy may still write into shared memory when the CTA exits: wait
    // (bounded) for the last group armed in each stage.
    if (lane == 0)
      for (int k = 0; k < RS && k < armed; ++k) {
        const int last = armed - 1 - ((armed - 1 - k) % RS);
        mbar_drain_gemm(&raw_full[k], static_cast<uint32_t>(last / RS) & 1u);
      }
  } else {
    // Producer thread i fills pieces 4h .. 4h + 3 of A row r (one token).
    const int i = static_cast<int>(threadIdx.x) - 32 * (2 + kEmbEpiWarps);
    const int r = i % kBM, h = i / kBM;
    const int bpt = ep.C == 3 ? 48 : 32;
    int stage = 0, rs = 0;
    uint32_t phase = 0, rph = 0;
    bool ok = true;
    // The next tile's row (request lookup, frame pointers, depth statistics)
    // is read while this tile is converted.
    EmbedRow er_next = embed_row(ep, (static_cast<int>(blockIdx.x) / n_tiles) * kBM + r);
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      const EmbedRow er = er_next;
      const int nt = tile + static_cast<int>(gridDim.x);
      if (nt < num_tiles) er_next = embed_row(ep, (nt / n_tiles) * kBM + r);
      // K steps in pixel groups g = 4 t + yq, the C channel blocks of a group
      // in a row (the W copies follow the same order), so each pixel is read
      // once for all channels.  The group's bytes come from the raw stage the
      // loader filled (or, for an unaligned tile, from the frames); once they
      // are in registers the stage is handed back.
      const int groups = num_kb / ep.C;
      for (int g = 0; g < groups && ok; ++g) {
        if (!mbar_wait_warp(&raw_full[rs], rph, err, kDevTimeoutProducer, lane)) {
          ok = false;
          break;
        }
        EmbedRaw raw;
        if (*reinterpret_cast<volatile int*>(&raw_bulk[rs]))
          embed_load_raw(sRaw + rs * raw_bytes, r, h, bpt, er.valid, raw);
        else
          embed_load(er, g, ep.C, h, raw);
        __syncwarp();
        if (lane == 0) mbar_arrive(&raw_empty[rs]);
        if (++rs == RS) {
          rs = 0;
          rph ^= 1u;
        }
        for (int c = 0; c < ep.C && ok; ++c)
          ok = embed_step<S>(er, raw, c, r, h, ep.C, sA, full, empty, stage, phase, err, lane);
      }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

template <int BN, int EPI, bool F8 = false>
cudaError_t launch_bn_epi(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const float* bias, int M,
                          int N, int K, int* err, int num_sms, cudaStream_t st, const float* row_scale = nullptr,
                          const float* col_scale = nullptr, const EpiAux& ln = EpiAux{}) {
  using Cfg = TcGemmCfg<BN>;
  auto kern = gemm_tc_kernel<BN, EPI, F8>;
  static std::atomic<unsigned long long> attr_done{0};  // one per template instance
  cudaError_t e = ensure_smem_attr(kern, Cfg::kSmemBytes, attr_done);
  if (e != cudaSuccess) return e;
  const int tiles = ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
  const int grid = tiles < num_sms ? tiles : num_sms;
  kern<<<grid, kThreads, Cfg::kSmemBytes, st>>>(a, b, c, bias, row_scale, col_scale, M, N, K, err, ln);
  return cudaGetLastError();
}

template <int BN, int EPI, bool F8 = false>
cudaError_t launch_pair_epi(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const float* bias, int M,
                            int N, int K, int* err, int num_sms, cudaStream_t st, const float* row_scale = nullptr,
                            const float* col_scale = nullptr, const EpiAux& ln = EpiAux{}) {
  using Cfg = TcGemmPairCfg<BN>;
  auto kern = gemm_tc_pair_kernel<BN, EPI, F8>;
  static std::atomic<unsigned long long> attr_done{0};  // one per template instance
  cudaError_t e = ensure_smem_attr(kern, Cfg::kSmemBytes, attr_done);
  if (e != cudaSuccess) return e;
  const int tiles = ((M + 2 * kBM - 1) / (2 * kBM)) * ((N + BN - 1) / BN);
  const int pairs = std::min(tiles, num_sms / 2);
  if (pairs < 1) return cudaErrorInvalidValue;
  kern<<<2 * pairs, kThreads, Cfg::kSmemBytes, st>>>(a, b, c, bias, row_scale, col_scale, M, N, K, err, ln);
  return cudaGetLastError();
}

template <bool F8>
cudaError_t launch_any(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, int bn, int epi,
                       const float* bias, int M, int N, int K, int* err, int num_sms, cudaStream_t st,
                       const float* row_scale, const float* col_scale, const EpiAux& ln = EpiAux{}) {
#define REVO_GEMM_CASE(W, E)                                                                                 \
  if (bn == (W) && epi == (E)) return launch_bn_epi<W, E, F8>(a, b, c, bias, M, N, K, err, num_sms, st, row_scale, \
                                                             col_scale, ln);                                      \
  if (bn == ((W) | kTilePair) && epi == (E))                                                                 \
    return launch_pair_epi<W, E, F8>(a, b, c, bias, M, N, K, err, num_sms, st, row_scale, col_scale, ln);
  if constexpr (!F8) {
    if (bn == 192 && epi == kEpiF32)
      return launch_bn_epi<192, kEpiF32, false>(a, b, c, bias, M, N, K, err, num_sms, st, row_scale, col_scale);
    if (bn == 192 && epi == kEpiResidF32)
      return launch_bn_epi<192, kEpiResidF32, false>(a, b, c, bias, M, N, K, err, num_sms, st, row_scale, col_scale);
    REVO_GEMM_CASE(128, kEpiF32)
    REVO_GEMM_CASE(256, kEpiF32)
    REVO_GEMM_CASE(128, kEpiResidF32)
    REVO_GEMM_CASE(256, kEpiResidF32)
    REVO_GEMM_CASE(128, kEpiResidLn)
    REVO_GEMM_CASE(256, kEpiResidLn)
    REVO_GEMM_CASE(128, kEpiResidLn8)
    REVO_GEMM_CASE(256, kEpiResidLn8)
    if (bn == 192 && epi == kEpiF32Pe)
      return launch_bn_epi<192, kEpiF32Pe, false>(a, b, c, bias, M, N, K, err, num_sms, st, row_scale, col_scale, ln);
    REVO_GEMM_CASE(128, kEpiF32Pe)
    REVO_GEMM_CASE(256, kEpiF32Pe)
  }
  REVO_GEMM_CASE(128, kEpiBf16)
  REVO_GEMM_CASE(256, kEpiBf16)
  REVO_GEMM_CASE(128, kEpiGeluBf16)
  REVO_GEMM_CASE(256, kEpiGeluBf16)
#undef REVO_GEMM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_gemm_tc(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, int bn, int epi,
                           const float* bias, int M, int N, int K, int* err, int num_sms, cudaStream_t st,
                           const EpiAux* ln) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const bool bf16_out = epi == kEpiBf16 || epi == kEpiGeluBf16;
  if (K % kBK != 0 || N % (bf16_out ? 64 : 32) != 0) return cudaErrorInvalidValue;
  if (epi == kEpiResidLn) {
    // The fused LayerNorm: a whole row of x in one warp's registers (N <= 1024).
    if (!ln || !ln->x || !ln->g || !ln->b || !ln->out || !ln->counters || (ln->mode == 2 && !ln->row_scale) ||
        (ln->mode != 1 && ln->mode != 2) || N % 4 != 0 || N > 4 * 32 * kLnMaxVec || (bn & ~kTilePair) == 192)
      return cudaErrorInvalidValue;
    return launch_any<false>(a, b, c, bn, ln->mode == 2 ? kEpiResidLn8 : kEpiResidLn, bias, M, N, K, err, num_sms,
                             st, nullptr, nullptr, *ln);
  }
  if (epi == kEpiF32Pe) {
    if (!ln || !ln->pe_pos || !ln->pe_tab || !ln->pe_omega || ln->pe_part <= 0 || ln->pe_part % 64 != 0 ||
        N != 3 * ln->pe_part || ln->pe_rows < 0)
      return cudaErrorInvalidValue;
    return launch_any<false>(a, b, c, bn, epi, bias, M, N, K, err, num_sms, st, nullptr, nullptr, *ln);
  }
  if (epi != kEpiF32 && epi != kEpiBf16 && epi != kEpiGeluBf16 && epi != kEpiResidF32) return cudaErrorInvalidValue;
  return launch_any<false>(a, b, c, bn, epi, bias, M, N, K, err, num_sms, st, nullptr, nullptr);
}

cudaError_t launch_gemm_tc_fp8(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, int bn, int epi,
                               const float* bias, const float* row_scale, const float* col_scale, int M, int N, int K,
                               int* err, int num_sms, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K % kBK8 != 0 || N % 64 != 0 || !row_scale || !col_scale) return cudaErrorInvalidValue;
  return launch_any<true>(a, b, c, bn, epi, bias, M, N, K, err, num_sms, st, row_scale, col_scale);
}

cudaError_t launch_embed_tc(const CUtensorMap& w, const CUtensorMap& c, int bn, const float* bias, int M, int N,
                            int K, int* err, int num_sms, cudaStream_t st, const EpiAux& pe, const EmbedParams& ep) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (ep.n <= 0 || ep.n > kMaxSegments || ep.seg_start[0] != 0 || ep.seg_start[ep.n] != M || !ep.jobs ||
      !ep.pe_pos || (ep.C != 1 && ep.C != 3) || ep.T < 1 || ep.T > 2 || K != ep.T * ep.C * 256 || K % kBK != 0 ||
      N % 32 != 0 || !pe.pe_tab || !pe.pe_omega || pe.pe_part <= 0 || pe.pe_part % 64 != 0 ||
      N != 3 * pe.pe_part || pe.pe_rows < 0)
    return cudaErrorInvalidValue;
  for (int i = 0; i < ep.n; ++i)
    if (ep.seg_start[i + 1] < ep.seg_start[i] || ep.hp[i] <= 0 || ep.wp[i] <= 0 || ep.hp[i] > 0xFFFF ||
        ep.wp[i] > 0xFFFF || (ep.seg_start[i + 1] - ep.seg_start[i]) % (ep.hp[i] * ep.wp[i]) != 0)
      return cudaErrorInvalidValue;
  const int tiles_m = (M + kBM - 1) / kBM;
  auto go = [&](auto kern, int smem, int tn, std::atomic<unsigned long long>& done) -> cudaError_t {
    cudaError_t e = ensure_smem_attr(kern, smem, done);
    if (e != cudaSuccess) return e;
    const int tiles = tiles_m * ((N + tn - 1) / tn);
    const int grid = tiles < num_sms ? tiles : num_sms;
    kern<<<grid, kEmbThreads, smem, st>>>(w, c, bias, M, N, K, err, pe, ep);
    return cudaGetLastError();
  };
  static std::atomic<unsigned long long> done128{0}, done256{0};
  if (bn == 256) return go(embed_tc_kernel<256>, EmbedCfg<256>::kSmemBytes, 256, done256);
  if (bn == 128) return go(embed_tc_kernel<128>, EmbedCfg<128>::kSmemBytes, 128, done128);
  return cudaErrorInvalidValue;
}

}  // namespace revo
