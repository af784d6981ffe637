// Linear layers on the tcgen05 tensor cores: Y = epilogue(A W^T + b).
//
// Every Linear of the recovery network (tubelet embedding, qkv, attention
// output projection, MLP fc1/fc2, encoder->decoder map, pixel head) is a dense
// contraction over token rows.  A [M][K] (bf16 activations) and W [N][K] (bf16
// weights, the Linear [out][in] layout) are both K-major, so TMA copies 128 x 64
// and BN x 64 tiles with the 128-byte swizzle straight into the operand layout
// tcgen05.mma reads.  The accumulator (128 lanes x BN f32 columns) lives in
// TMEM, double-buffered so the epilogue of one tile overlaps the main loop of
// the next.  The epilogue fuses the bias, the exact GELU, the residual add and
// the bf16 downcast.
//
// Warp roles (192 threads, one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer (one thread)
//   warp 1      TMEM allocator + MMA issuer (one thread)
//   warps 2..5  epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 = tile rows
#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // 64 bf16 = one 128-byte swizzle atom per row

template <int BN>
struct TcGemmCfg {
  static constexpr int kStages = (BN == 256) ? 4 : 6;
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kTmemCols = 2 * BN;
  static constexpr int kSmemBytes = 1024 /*align slack*/ + kStages * kStageBytes + 256 /*barriers*/;
};

template <int EPI>
REVO_DEVI void store_chunk(const uint32_t (&r)[32], const float* __restrict__ bias, void* out, int ldo, int row,
                           int col0) {
  float v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
  if (bias != nullptr) {
    const float4* b4 = reinterpret_cast<const float4*>(bias + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 b = __ldg(b4 + i);
      v[4 * i] += b.x;
      v[4 * i + 1] += b.y;
      v[4 * i + 2] += b.z;
      v[4 * i + 3] += b.w;
    }
  }
  if (EPI == kEpiGeluBf16) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = gelu_exact(v[i]);
  }
  if (EPI == kEpiF32) {
    float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + static_cast<size_t>(row) * ldo + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if (EPI == kEpiResidF32) {
    float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + static_cast<size_t>(row) * ldo + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4 x = o[i];
      x.x += v[4 * i];
      x.y += v[4 * i + 1];
      x.z += v[4 * i + 2];
      x.w += v[4 * i + 3];
      o[i] = x;
    }
  } else {
    uint4* o = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + static_cast<size_t>(row) * ldo + col0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      o[i] = make_uint4(pack_bf16x2(v[8 * i], v[8 * i + 1]), pack_bf16x2(v[8 * i + 2], v[8 * i + 3]),
                        pack_bf16x2(v[8 * i + 4], v[8 * i + 5]), pack_bf16x2(v[8 * i + 6], v[8 * i + 7]));
  }
}

template <int BN, int EPI>
__global__ void __launch_bounds__(192, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const float* __restrict__ bias, void* out, int ldo, int M, int N, int K, int* err) {
  using Cfg = TcGemmCfg<BN>;
  constexpr int S = Cfg::kStages;
  constexpr uint32_t kIdesc = idesc_bf16(kBM, BN);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S * Cfg::kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + S * Cfg::kBBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int m_tiles = (M + kBM - 1) / kBM;
  const int n_tiles = (N + BN - 1) / BN;
  const int num_tiles = m_tiles * n_tiles;
  const int num_kb = K / kBK;

  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
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
        const int m0 = (tile % m_tiles) * kBM;
        const int n0 = (tile / m_tiles) * BN;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, kDevTimeoutProducer)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
          tma_load_2d(sA + stage * Cfg::kABytes, &tmA, kb * kBK, m0, &full[stage]);
          tma_load_2d(sB + stage * Cfg::kBBytes, &tmB, kb * kBK, n0, &full[stage]);
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
          const uint32_t a_addr = smem_u32(sA + stage * Cfg::kABytes);
          const uint32_t b_addr = smem_u32(sB + stage * Cfg::kBBytes);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            mma_f16(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                    (kb | kk) != 0 ? 1u : 0u);
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
    const int q = warp & 3;
    int t_local = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++t_local) {
      const int acc = t_local & 1;
      const uint32_t acc_phase = (t_local >> 1) & 1;
      if (!mbar_wait(&tfull[acc], acc_phase, err, kDevTimeoutEpilogue)) break;
      tc_fence_after();
      const int m0 = (tile % m_tiles) * kBM;
      const int n0 = (tile / m_tiles) * BN;
      const int row = m0 + q * 32 + lane;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) + acc * BN + c * 32, r);
        tmem_wait_ld();
        const int col0 = n0 + c * 32;
        if (row < M && col0 < N) store_chunk<EPI>(r, bias, out, ldo, row, col0);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

template <int BN, int EPI>
cudaError_t launch_bn_epi(const CUtensorMap& a, const CUtensorMap& b, const float* bias, void* out, int ldo, int M,
                          int N, int K, int* err, int num_sms, cudaStream_t st) {
  using Cfg = TcGemmCfg<BN>;
  auto kern = gemm_tc_kernel<BN, EPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  const int tiles = ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
  const int grid = tiles < num_sms ? tiles : num_sms;
  kern<<<grid, 192, Cfg::kSmemBytes, st>>>(a, b, bias, out, ldo, M, N, K, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(const CUtensorMap& a, const CUtensorMap& b, int bn, int epi, const float* bias, void* out,
                           int ldo, int M, int N, int K, int* err, int num_sms, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K % kBK != 0 || N % 32 != 0) return cudaErrorInvalidValue;
  if (bn == 256) {
    switch (epi) {
      case kEpiF32: return launch_bn_epi<256, kEpiF32>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiBf16: return launch_bn_epi<256, kEpiBf16>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiGeluBf16: return launch_bn_epi<256, kEpiGeluBf16>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiResidF32: return launch_bn_epi<256, kEpiResidF32>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
    }
  } else {
    switch (epi) {
      case kEpiF32: return launch_bn_epi<128, kEpiF32>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiBf16: return launch_bn_epi<128, kEpiBf16>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiGeluBf16: return launch_bn_epi<128, kEpiGeluBf16>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
      case kEpiResidF32: return launch_bn_epi<128, kEpiResidF32>(a, b, bias, out, ldo, M, N, K, err, num_sms, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace revo
