// Memory-bound stages of the recovery forward: input unpack + normalisation
// fused with the tubelet gather, the sinusoidal (temporal distance, row,
// column) embedding, LayerNorm, depth statistics, and the warp-level
// de-normalise / quantise / masked-blend writeback.
#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "layernorm_row.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

__constant__ float kRgbMean[3] = {0.485f, 0.456f, 0.406f};
__constant__ float kRgbStd[3] = {0.229f, 0.224f, 0.225f};

// ------------------------------------------------------------- assemble --
// One thread writes one run of p outputs: token n, frame t of its tubelet,
// channel c, patch row y (vector order t, c, y, x; Appendix B.3).
REVO_DEVI void assemble_body(const AssembleArgs& a) {
  const int p = a.p, C = a.C, T = a.T;
  const int Hp = a.H / p, Wp = a.W / p;
  const int S = a.F / T;
  const long long runs = static_cast<long long>(S) * Hp * Wp * T * C * p;
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= runs) return;
  long long rest = idx;
  const int y = rest % p;
  rest /= p;
  const int c = rest % C;
  rest /= C;
  const int t = rest % T;
  const long long n = rest / T;
  const int s = static_cast<int>(n / (Hp * Wp));
  const int rem = static_cast<int>(n % (Hp * Wp));
  const int ty = rem / Wp, tx = rem % Wp;
  const int f = s * T + t;
  const int row = ty * p + y;
  const int col0 = tx * p;
  const uint8_t* src = static_cast<const uint8_t*>(a.frames[f]) + static_cast<size_t>(row) * a.pitch[f];
  const int K = T * C * p * p;
  const size_t o = static_cast<size_t>(n) * K + static_cast<size_t>((t * C + c) * p + y) * p;

  float v[16];
  if (C == 3) {
    const float mean = kRgbMean[c], sd = kRgbStd[c];
#pragma unroll
    for (int x = 0; x < 16; ++x)
      if (x < p) v[x] = (static_cast<float>(src[(col0 + x) * 3 + c]) / 255.0f - mean) / sd;
  } else {
    const float mu = a.mu_sigma[0], sg = a.mu_sigma[1];
    const uint16_t* s16 = reinterpret_cast<const uint16_t*>(src);
#pragma unroll
    for (int x = 0; x < 16; ++x)
      if (x < p) v[x] = (static_cast<float>(s16[col0 + x]) - mu) / sg;
  }
  if (a.out_bf16) {
    __nv_bfloat16* dst = static_cast<__nv_bfloat16*>(a.out) + o;
    if (p == 16) {
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      d4[0] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                         pack_bf16x2(v[6], v[7]));
      d4[1] = make_uint4(pack_bf16x2(v[8], v[9]), pack_bf16x2(v[10], v[11]), pack_bf16x2(v[12], v[13]),
                         pack_bf16x2(v[14], v[15]));
    } else {
#pragma unroll
      for (int x = 0; x < 16; ++x)
        if (x < p) dst[x] = __float2bfloat16_rn(v[x]);
    }
  } else {
    float* dst = static_cast<float*>(a.out) + o;
    if (p == 16) {
      float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
      for (int i = 0; i < 4; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
#pragma unroll
      for (int x = 0; x < 16; ++x)
        if (x < p) dst[x] = v[x];
    }
  }
}

// Arguments by value (step-level calls) or from a device table (the runtime's
// captured graphs read per-request arguments written just before each replay).
__global__ void assemble_kernel(const __grid_constant__ AssembleArgs a) { assemble_body(a); }
__global__ void assemble_kernel_dev(const AssembleArgs* __restrict__ a) { assemble_body(*a); }

// Patch size 16 (the model's): one warp per (frame, token); lane 2y + h
// handles pixels [8h, 8h + 8) of the token's patch row y.  For each channel
// the warp's 32 lanes then write the token's 16 x 16 plane (512 contiguous
// bytes in bf16) with one 16-byte store each, and read 16 row segments of
// 48 (RGB) or 32 (depth) bytes.  RGB codes are normalised as
// x * (1 / (255 std_c)) + (-mean_c / std_c) in one FMA (constants rounded
// once from their exact values; within 2 ulp of (x / 255 - mean_c) / std_c),
// depth as (d - mu) * (1 / sigma).  A row that is not 8-byte aligned falls
// back to byte loads.
__constant__ float kRgbScale[3] = {kRgbScaleR, kRgbScaleG, kRgbScaleB};
__constant__ float kRgbShift[3] = {kRgbShiftR, kRgbShiftG, kRgbShiftB};
constexpr int kAsmThreads = 256;

REVO_DEVI void assemble16_body(const AssembleArgs& a) {
  const int C = a.C, T = a.T, H = a.H;
  const int Wp = a.W >> 4, Hp = H >> 4;
  const long long gw = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  if (gw >= static_cast<long long>(a.F) * Hp * Wp) return;
  const int lane = threadIdx.x & 31;
  const int y = lane >> 1, hx = lane & 1;
  const int tx = static_cast<int>(gw % Wp);
  const long long ft = gw / Wp;
  const int ty = static_cast<int>(ft % Hp);
  const int f = static_cast<int>(ft / Hp);
  const int s = f / T, t = f % T;
  const size_t n = static_cast<size_t>(s * Hp + ty) * Wp + tx;
  if (a.pe_pos && t == 0 && lane == 0) a.pe_pos[n] = make_int2(a.taus[s], (ty << 16) | tx);
  const size_t K = static_cast<size_t>(T) * C * 256;
  const uint8_t* src = static_cast<const uint8_t*>(a.frames[f]) + static_cast<size_t>(ty * 16 + y) * a.pitch[f];
  float v[3][8];
  if (C == 3) {
    const uint8_t* p3 = src + tx * 48 + hx * 24;
    uint32_t b[6];
    if ((reinterpret_cast<uintptr_t>(p3) & 7u) == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(p3) + i);
        b[2 * i] = w.x;
        b[2 * i + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i)
        b[i] = p3[4 * i] | (p3[4 * i + 1] << 8) | (p3[4 * i + 2] << 16) | (static_cast<uint32_t>(p3[4 * i + 3]) << 24);
    }
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int byte = 3 * x + c;
        v[c][x] = fmaf(byte_to_float(b[byte >> 2], byte & 3), kRgbScale[c], kRgbShift[c]);
      }
  } else {
    const uint8_t* p1 = src + tx * 32 + hx * 16;
    uint32_t w16[4];
    if ((reinterpret_cast<uintptr_t>(p1) & 15u) == 0) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(p1));
      w16[0] = w.x, w16[1] = w.y, w16[2] = w.z, w16[3] = w.w;
    } else {
      const uint16_t* q = reinterpret_cast<const uint16_t*>(p1);
#pragma unroll
      for (int i = 0; i < 4; ++i) w16[i] = q[2 * i] | (static_cast<uint32_t>(q[2 * i + 1]) << 16);
    }
    const float mu = a.mu_sigma[0], inv = 1.f / a.mu_sigma[1];
#pragma unroll
    for (int x = 0; x < 8; ++x)
      v[0][x] = (static_cast<float>((w16[x >> 1] >> (16 * (x & 1))) & 0xFFFFu) - mu) * inv;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c >= C) break;
    const size_t o = n * K + static_cast<size_t>((t * C + c) * 16 + y) * 16 + hx * 8;
    if (a.out_bf16) {
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.out) + o) =
          make_uint4(pack_bf16x2(v[c][0], v[c][1]), pack_bf16x2(v[c][2], v[c][3]), pack_bf16x2(v[c][4], v[c][5]),
                     pack_bf16x2(v[c][6], v[c][7]));
    } else {
      float4* d4 = reinterpret_cast<float4*>(static_cast<float*>(a.out) + o);
      d4[0] = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
      d4[1] = make_float4(v[c][4], v[c][5], v[c][6], v[c][7]);
    }
  }
}

__global__ void __launch_bounds__(kAsmThreads) assemble16_kernel(const __grid_constant__ AssembleArgs a) {
  assemble16_body(a);
}
__global__ void __launch_bounds__(kAsmThreads) assemble16_kernel_dev(const AssembleArgs* __restrict__ a) {
  assemble16_body(*a);
}
// One launch for a batch: blockIdx.y picks the request (blocks past its size return).
__global__ void __launch_bounds__(kAsmThreads) assemble16_kernel_batch(const uint8_t* __restrict__ args,
                                                                       size_t stride) {
  assemble16_body(*reinterpret_cast<const AssembleArgs*>(args + blockIdx.y * stride));
}

// ------------------------------------------------------------------- PE --
struct PeArgs {
  float omega[128];  // 10000^(-2i/part), i < part / 2
  int taus[8];
  const int* taus_dev;  // if set, the temporal distances are read from here
  int Hp, Wp, D, part;
};

// The embedding values of one part at integer position `pos`: column i <
// part / 2 holds sin(pos w_i), column part / 2 + i holds cos(pos w_i), both from
// one sincosf of the float32 product pos * w_i.
REVO_DEVI void pe_part(float pos, const float* om, int half, float* out, int tid, int nthreads) {
  for (int i = tid; i < half; i += nthreads) {
    float sv, cv;
    sincosf(pos * om[i], &sv, &cv);
    out[i] = sv;
    out[half + i] = cv;
  }
}

// Table of the column part for positions 0 .. rows-1: tab[c][0 .. part).
__global__ void pe_table_kernel(float* __restrict__ tab, int rows, const __grid_constant__ PeArgs a) {
  __shared__ float om[128];
  const int half = a.part / 2;
  for (int i = threadIdx.x; i < half; i += blockDim.x) om[i] = a.omega[i];
  __syncthreads();
  pe_part(static_cast<float>(blockIdx.x), om, half, tab + static_cast<size_t>(blockIdx.x) * a.part, threadIdx.x,
          blockDim.x);
}

// One CTA per (slot s, run of 8 tokens of the slot): the temporal part of
// slot s is computed once into shared memory; the row and column parts come
// from `ptab` (pe_table_kernel's table: the part's values at integer position
// q, the same for rows and columns), or are computed per element without one.
// Each thread owns a 16-byte column group and adds it to the run's 8 token
// rows (8 independent read-modify-writes in flight).  Every value is the same
// float32 sincosf of pos * w_i as a per-element evaluation, so the result does
// not depend on the table.
constexpr int kPeRun = 8;
__global__ void add_pe_kernel(float* __restrict__ x, const __grid_constant__ PeArgs a,
                              const float* __restrict__ ptab) {
  __shared__ float om[128];
  __shared__ __align__(16) float tp[1024 / 3 + 4];
  const int half = a.part / 2;
  for (int i = threadIdx.x; i < half; i += blockDim.x) om[i] = a.omega[i];
  __syncthreads();
  const int hw = a.Hp * a.Wp;
  const int runs = (hw + kPeRun - 1) / kPeRun;
  const int s = static_cast<int>(blockIdx.x) / runs;
  const int t0 = (static_cast<int>(blockIdx.x) % runs) * kPeRun;
  const int tau = a.taus_dev ? __ldg(a.taus_dev + s) : a.taus[s];
  pe_part(static_cast<float>(tau), om, half, tp, threadIdx.x, blockDim.x);
  __syncthreads();
  const int nv = a.D / 4;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    const int col = 4 * j;
    const int which = col / a.part;  // a part is a multiple of 64 columns: a vector stays in one part
    const int q = col - which * a.part;
    float4 v[kPeRun];
#pragma unroll
    for (int u = 0; u < kPeRun; ++u) {
      const int t = t0 + u;
      if (t >= hw) break;
      const int pos = which == 1 ? t / a.Wp : t % a.Wp;
      if (which == 0) {
        v[u] = *reinterpret_cast<const float4*>(tp + q);
      } else if (ptab) {
        v[u] = __ldg(reinterpret_cast<const float4*>(ptab + static_cast<size_t>(pos) * a.part + q));
      } else {
        float e4[4];
        for (int w = 0; w < 4; ++w) {
          const int i = (q + w) % half;
          float sv, cv;
          sincosf(static_cast<float>(pos) * om[i], &sv, &cv);
          e4[w] = q + w < half ? sv : cv;
        }
        v[u] = make_float4(e4[0], e4[1], e4[2], e4[3]);
      }
    }
    float4* p = reinterpret_cast<float4*>(x + (static_cast<size_t>(s) * hw + t0) * a.D) + j;
    float4 y[kPeRun];
#pragma unroll
    for (int u = 0; u < kPeRun; ++u)
      if (t0 + u < hw) y[u] = p[static_cast<size_t>(u) * nv];
#pragma unroll
    for (int u = 0; u < kPeRun; ++u) {
      if (t0 + u >= hw) break;
      y[u].x += v[u].x;
      y[u].y += v[u].y;
      y[u].z += v[u].z;
      y[u].w += v[u].w;
      p[static_cast<size_t>(u) * nv] = y[u];
    }
  }
}

// ------------------------------------------------------------ LayerNorm --
// One warp per row (ln_row in layernorm_row.cuh, shared with the GEMM
// epilogue that fuses the LayerNorm after a residual add).
// OUT: 0 float32, 1 bf16, 2 E4M3 codes + a per-row scale.
template <int OUT>
__global__ void layernorm_kernel(const float* __restrict__ x, const float* __restrict__ g,
                                 const float* __restrict__ b, void* __restrict__ out, float* __restrict__ row_scale,
                                 int M, int D) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= M) return;
  ln_row<OUT, false>(x, g, b, out, row_scale, warp, D, lane);
}

// One warp per row: amax pass, then the codes.
__global__ void quantize_rows_e4m3_kernel(const float* __restrict__ x, int rows, int cols, uint8_t* __restrict__ q,
                                          float* __restrict__ scale) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float4* xr = reinterpret_cast<const float4*>(x + static_cast<size_t>(row) * cols);
  const int nv = cols / 4;
  float amax = 0.f;
  for (int c = lane; c < nv; c += 32) {
    const float4 a = __ldg(xr + c);
    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  float sc, inv;
  e4m3_row_scale(amax, &sc, &inv);
  uint32_t* qr = reinterpret_cast<uint32_t*>(q + static_cast<size_t>(row) * cols);
  for (int c = lane; c < nv; c += 32) {
    const float4 a = __ldg(xr + c);
    qr[c] = pack_e4m3x4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
  }
  if (lane == 0) scale[row] = sc;
}

// ---------------------------------------------------------- depth stats --
// Two passes over the frame.  Pass 1: exact integer count and sum of the
// non-zero pixels -> mean.  Pass 2: float sum of squared deviations -> biased
// standard deviation.  Per-block partials go to scratch; the last block to
// finish (atomic ticket) reduces them in a fixed order, so the result is
// deterministic.
constexpr int kStatsBlocks = 256;
constexpr int kStatsThreads = 256;

struct StatsScratch {
  unsigned int ticket[4];
  unsigned long long count[kStatsBlocks];
  unsigned long long sum[kStatsBlocks];
  float sq[kStatsBlocks];
  float mean;
  float pad[3];
};

template <typename T>
REVO_DEVI T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) r += red[i];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kStatsThreads) depth_stats_pass1(const uint16_t* __restrict__ d, int H, int W,
                                                                   size_t pitch, StatsScratch* sc) {
  __shared__ unsigned long long red[kStatsThreads / 32];
  __shared__ bool last;
  unsigned long long cnt = 0, sum = 0;
  const long long total = static_cast<long long>(H) * W;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int y = static_cast<int>(i / W), x = static_cast<int>(i % W);
    const uint16_t v = *reinterpret_cast<const uint16_t*>(reinterpret_cast<const uint8_t*>(d) + y * pitch + 2 * x);
    if (v) {
      ++cnt;
      sum += v;
    }
  }
  cnt = block_sum(cnt, red);
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) {
    sc->count[blockIdx.x] = cnt;
    sc->sum[blockIdx.x] = sum;
    __threadfence();
    last = atomicAdd(&sc->ticket[0], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    unsigned long long c = 0, s = 0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) {
      c += *reinterpret_cast<volatile unsigned long long*>(&sc->count[b]);
      s += *reinterpret_cast<volatile unsigned long long*>(&sc->sum[b]);
    }
    sc->mean = c ? static_cast<float>(s) / static_cast<float>(c) : 0.f;
    sc->count[0] = c;  // total, read by pass 2
    sc->ticket[0] = 0;
  }
}

__global__ void __launch_bounds__(kStatsThreads) depth_stats_pass2(const uint16_t* __restrict__ d, int H, int W,
                                                                   size_t pitch, StatsScratch* sc,
                                                                   float* mu_sigma) {
  __shared__ float red[kStatsThreads / 32];
  __shared__ bool last;
  const float mean = *reinterpret_cast<volatile float*>(&sc->mean);
  float sq = 0.f;
  const long long total = static_cast<long long>(H) * W;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int y = static_cast<int>(i / W), x = static_cast<int>(i % W);
    const uint16_t v = *reinterpret_cast<const uint16_t*>(reinterpret_cast<const uint8_t*>(d) + y * pitch + 2 * x);
    if (v) {
      const float e = static_cast<float>(v) - mean;
      sq += e * e;
    }
  }
  sq = block_sum(sq, red);
  if (threadIdx.x == 0) {
    sc->sq[blockIdx.x] = sq;
    __threadfence();
    last = atomicAdd(&sc->ticket[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    float s = 0.f;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) s += *reinterpret_cast<volatile float*>(&sc->sq[b]);
    const unsigned long long c = *reinterpret_cast<volatile unsigned long long*>(&sc->count[0]);
    float mu = 0.f, sigma = 1.f;
    if (c) {
      mu = mean;
      sigma = fmaxf(sqrtf(s / static_cast<float>(c)), 1.0f);
    }
    mu_sigma[0] = mu;
    mu_sigma[1] = sigma;
    sc->ticket[1] = 0;
  }
}

// ---------------------------------------------------------------- blend --
// One warp per run of 32 pixels of one row; lane i owns pixel 32*w + i and bit
// i of the row's mask word w.  Received pixels copy the decoded value; lost
// pixels take the quantised recovery (round half to even, clamped).  The
// de-normalisation is done as separate float32 multiply and add (no fused
// multiply-add), so a float32 restatement reproduces every code exactly.
REVO_DEVI void blend_body(const BlendArgs& a) {
  const int words = (a.W + 31) / 32;
  const long long gw = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= static_cast<long long>(a.H) * words) return;
  const int y = static_cast<int>(gw / words);
  const int w = static_cast<int>(gw % words);
  const int x = w * 32 + lane;
  const uint32_t word = __ldg(a.mask + static_cast<size_t>(y) * a.mask_pitch + w);
  if (x >= a.W) return;
  const bool lost = (word >> lane) & 1u;
  const int p = a.p, C = a.C;
  const int Wp = a.W / p;
  const size_t n = static_cast<size_t>(y / p) * Wp + x / p;
  const float* hrow = a.head + n * (C * p * p) + (y % p) * p + (x % p);
  if (C == 3) {
    const uint8_t* dec = static_cast<const uint8_t*>(a.decoded) + static_cast<size_t>(y) * a.pitch + 3 * x;
    uint8_t* o = static_cast<uint8_t*>(a.out) + static_cast<size_t>(y) * a.out_pitch + 3 * x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = __fadd_rn(__fmul_rn(__ldg(hrow + c * p * p), kRgbStd[c]), kRgbMean[c]);
      if (a.values) a.values[(static_cast<size_t>(y) * a.W + x) * 3 + c] = v;
      const float q = fminf(fmaxf(rintf(__fmul_rn(v, 255.0f)), 0.f), 255.f);
      o[c] = lost ? static_cast<uint8_t>(q) : dec[c];
    }
  } else {
    const uint16_t* dec = reinterpret_cast<const uint16_t*>(static_cast<const uint8_t*>(a.decoded) +
                                                            static_cast<size_t>(y) * a.pitch) + x;
    uint16_t* o = reinterpret_cast<uint16_t*>(static_cast<uint8_t*>(a.out) + static_cast<size_t>(y) * a.out_pitch) + x;
    const float v = __fadd_rn(__fmul_rn(__ldg(hrow), a.mu_sigma[1]), a.mu_sigma[0]);
    if (a.values) a.values[static_cast<size_t>(y) * a.W + x] = v;
    const float q = fminf(fmaxf(rintf(v), 0.f), 65535.f);
    *o = lost ? static_cast<uint16_t>(q) : *dec;
  }
}

__global__ void blend_kernel(const __grid_constant__ BlendArgs a) { blend_body(a); }
__global__ void blend_kernel_dev(const BlendArgs* __restrict__ a) { blend_body(*a); }

// Patch size 16: one thread per (row, 8-pixel run) with all channels.  The
// head's 8 values per channel are 32 contiguous bytes of the token's row; the
// decoded and output pixels are 24 (RGB) or 16 (depth) contiguous bytes,
// moved with 8- or 16-byte accesses when aligned (bytes otherwise).  All loads
// are issued before the arithmetic, which is blend_body's.
constexpr int kBlendThreads = 128;

// `block`: this block's index within the frame's launch blocks.
REVO_DEVI void blend16_body(const BlendArgs& a, long long block) {
  const int C = a.C, W = a.W;
  const int runs = W >> 3;
  const long long idx = block * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(a.H) * runs) return;
  const int r8 = static_cast<int>(idx % runs);
  const int y = static_cast<int>(idx / runs);
  const int x0 = r8 * 8;
  const uint32_t bits = (__ldg(a.mask + static_cast<size_t>(y) * a.mask_pitch + (x0 >> 5)) >> (x0 & 31)) & 0xFFu;
  const size_t n = static_cast<size_t>(y >> 4) * (W >> 4) + (x0 >> 4);
  const float* hrow = a.head + n * (C * 256) + (y & 15) * 16 + (x0 & 15);
  const bool hvec = (reinterpret_cast<uintptr_t>(hrow) & 15u) == 0;
  const int bpp = C == 3 ? 3 : 2;  // bytes per pixel
  const uint8_t* dec = static_cast<const uint8_t*>(a.decoded) + static_cast<size_t>(y) * a.pitch + x0 * bpp;
  uint8_t* out = static_cast<uint8_t*>(a.out) + static_cast<size_t>(y) * a.out_pitch + x0 * bpp;
  float h[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c >= C) break;
    if (hvec) {
      const float4 q0 = __ldg(reinterpret_cast<const float4*>(hrow + c * 256));
      const float4 q1 = __ldg(reinterpret_cast<const float4*>(hrow + c * 256) + 1);
      h[c][0] = q0.x, h[c][1] = q0.y, h[c][2] = q0.z, h[c][3] = q0.w;
      h[c][4] = q1.x, h[c][5] = q1.y, h[c][6] = q1.z, h[c][7] = q1.w;
    } else {
#pragma unroll
      for (int x = 0; x < 8; ++x) h[c][x] = __ldg(hrow + c * 256 + x);
    }
  }
  if (C == 3) {
    uint32_t dw[6], ow[6];
    const bool dvec = ((reinterpret_cast<uintptr_t>(dec) | reinterpret_cast<uintptr_t>(out)) & 7u) == 0;
    if (dvec) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(dec) + i);
        dw[2 * i] = w.x, dw[2 * i + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i)
        dw[i] = dec[4 * i] | (dec[4 * i + 1] << 8) | (dec[4 * i + 2] << 16) | (static_cast<uint32_t>(dec[4 * i + 3]) << 24);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) ow[i] = 0u;
    float* vals = a.values ? a.values + (static_cast<size_t>(y) * W + x0) * 3 : nullptr;
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = __fadd_rn(__fmul_rn(h[c][x], kRgbStd[c]), kRgbMean[c]);
        if (vals) vals[x * 3 + c] = v;
        const float q = fminf(fmaxf(rintf(__fmul_rn(v, 255.0f)), 0.f), 255.f);
        const int byte = 3 * x + c;
        const uint32_t code =
            ((bits >> x) & 1u) ? static_cast<uint32_t>(q) : (dw[byte >> 2] >> (8 * (byte & 3))) & 0xFFu;
        ow[byte >> 2] |= code << (8 * (byte & 3));
      }
    if (dvec) {
#pragma unroll
      for (int i = 0; i < 3; ++i) reinterpret_cast<uint2*>(out)[i] = make_uint2(ow[2 * i], ow[2 * i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < 24; ++i) out[i] = static_cast<uint8_t>(ow[i >> 2] >> (8 * (i & 3)));
    }
  } else {
    uint32_t dw[4], ow[4];
    const bool dvec = ((reinterpret_cast<uintptr_t>(dec) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    if (dvec) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(dec));
      dw[0] = w.x, dw[1] = w.y, dw[2] = w.z, dw[3] = w.w;
    } else {
      const uint16_t* d16 = reinterpret_cast<const uint16_t*>(dec);
#pragma unroll
      for (int i = 0; i < 4; ++i) dw[i] = d16[2 * i] | (static_cast<uint32_t>(d16[2 * i + 1]) << 16);
    }
    const float mu = a.mu_sigma[0], sg = a.mu_sigma[1];
    float* vals = a.values ? a.values + static_cast<size_t>(y) * W + x0 : nullptr;
#pragma unroll
    for (int i = 0; i < 4; ++i) ow[i] = 0u;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const float v = __fadd_rn(__fmul_rn(h[0][x], sg), mu);
      if (vals) vals[x] = v;
      const float q = fminf(fmaxf(rintf(v), 0.f), 65535.f);
      const uint32_t code = ((bits >> x) & 1u) ? static_cast<uint32_t>(q) : (dw[x >> 1] >> (16 * (x & 1))) & 0xFFFFu;
      ow[x >> 1] |= code << (16 * (x & 1));
    }
    if (dvec) {
      *reinterpret_cast<uint4*>(out) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
    } else {
      uint16_t* o16 = reinterpret_cast<uint16_t*>(out);
#pragma unroll
      for (int x = 0; x < 8; ++x) o16[x] = static_cast<uint16_t>(ow[x >> 1] >> (16 * (x & 1)));
    }
  }
}

__global__ void __launch_bounds__(kBlendThreads) blend16_kernel(const __grid_constant__ BlendArgs a) {
  blend16_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(kBlendThreads) blend16_kernel_dev(const BlendArgs* __restrict__ a) {
  blend16_body(*a, blockIdx.x);
}
// One launch for a batch with no idle blocks: the frames' blocks are laid end
// to end (block_start[i] = the first block of frame i, a prefix over the
// frames' sizes); a block finds its frame by binary search.
struct BlendBatchPlan {
  int n;
  int block_start[kMaxSegments + 1];
};
__global__ void __launch_bounds__(kBlendThreads) blend16_kernel_batch(const uint8_t* __restrict__ args, size_t stride,
                                                                      const __grid_constant__ BlendBatchPlan plan) {
  const int b = static_cast<int>(blockIdx.x);
  int lo = 0, hi = plan.n - 1;  // the last frame whose blocks start at or before b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (plan.block_start[mid] <= b) lo = mid; else hi = mid - 1;
  }
  blend16_body(*reinterpret_cast<const BlendArgs*>(args + lo * stride), b - plan.block_start[lo]);
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

}  // namespace

cudaError_t launch_assemble(const AssembleArgs& a, cudaStream_t st, const AssembleArgs* dev) {
  if (a.T <= 0 || a.F % a.T != 0 || a.p <= 0 || a.p > 16 || a.H % a.p || a.W % a.p || a.F > kMaxRefs + 1 ||
      (a.C != 1 && a.C != 3) || (a.pe_pos && a.p != 16))
    return cudaErrorInvalidValue;
  if (a.p == 16) {
    const long long threads = static_cast<long long>(a.F) * (a.H / 16) * (a.W / 16) * 32;  // a warp per token-frame
    if (threads == 0) return cudaSuccess;
    const unsigned grid = static_cast<unsigned>((threads + kAsmThreads - 1) / kAsmThreads);
    if (dev)
      assemble16_kernel_dev<<<grid, kAsmThreads, 0, st>>>(dev);
    else
      assemble16_kernel<<<grid, kAsmThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  const long long runs = static_cast<long long>(a.F / a.T) * (a.H / a.p) * (a.W / a.p) * a.T * a.C * a.p;
  if (runs == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((runs + 255) / 256);
  if (dev)
    assemble_kernel_dev<<<grid, 256, 0, st>>>(dev);
  else
    assemble_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_assemble_batch(const AssembleArgs* host, int n, const AssembleArgs* dev, size_t stride,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > 65535 || !dev) return cudaErrorInvalidValue;
  long long threads = 0;
  for (int i = 0; i < n; ++i) {
    const AssembleArgs& a = host[i];
    if (a.T <= 0 || a.F % a.T != 0 || a.p != 16 || a.H % 16 || a.W % 16 || a.F > kMaxRefs + 1 ||
        (a.C != 1 && a.C != 3))
      return cudaErrorInvalidValue;
    threads = std::max(threads, static_cast<long long>(a.F) * (a.H / 16) * (a.W / 16) * 32);
  }
  if (threads == 0) return cudaSuccess;
  const dim3 grid(static_cast<unsigned>((threads + kAsmThreads - 1) / kAsmThreads), static_cast<unsigned>(n));
  assemble16_kernel_batch<<<grid, kAsmThreads, 0, st>>>(reinterpret_cast<const uint8_t*>(dev), stride);
  return cudaGetLastError();
}

cudaError_t launch_blend_batch(const BlendArgs* host, int n, const BlendArgs* dev, size_t stride, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxSegments || !dev) return cudaErrorInvalidValue;
  BlendBatchPlan plan{};
  plan.n = n;
  long long blocks = 0;
  for (int i = 0; i < n; ++i) {
    const BlendArgs& a = host[i];
    if (a.p != 16 || a.H % 16 || a.W % 16 || (a.C != 1 && a.C != 3)) return cudaErrorInvalidValue;
    plan.block_start[i] = static_cast<int>(blocks);
    blocks += (static_cast<long long>(a.H) * (a.W / 8) + kBlendThreads - 1) / kBlendThreads;
    if (blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  }
  plan.block_start[n] = static_cast<int>(blocks);
  if (blocks == 0) return cudaSuccess;
  blend16_kernel_batch<<<static_cast<unsigned>(blocks), kBlendThreads, 0, st>>>(reinterpret_cast<const uint8_t*>(dev),
                                                                                 stride, plan);
  return cudaGetLastError();
}

bool pe_omega(int D, float* omega) {
  const int part = D / 3;
  if (D <= 0 || D % 192 != 0 || part / 2 > 128) return false;
  for (int i = 0; i < part / 2; ++i) omega[i] = static_cast<float>(pow(10000.0, -2.0 * i / part));
  return true;
}

namespace {
bool pe_args(PeArgs* a, int D) {
  a->D = D;
  a->part = D / 3;
  return pe_omega(D, a->omega);
}

// One thread per token of one request.
__global__ void pe_positions_kernel(int2* __restrict__ pe_pos, int Hp, int Wp, int n, const __grid_constant__ PeArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int hw = Hp * Wp;
  const int t = i % hw;
  pe_pos[i] = make_int2(a.taus[i / hw], ((t / Wp) << 16) | (t % Wp));
}
}  // namespace

cudaError_t launch_pe_positions(int2* pe_pos, int Hp, int Wp, int slots, const int* taus, cudaStream_t st) {
  if (Hp < 0 || Wp < 0 || Hp > 0xFFFF || Wp > 0xFFFF || slots < 0 || slots > 8) return cudaErrorInvalidValue;
  const long long n = static_cast<long long>(slots) * Hp * Wp;
  if (n == 0) return cudaSuccess;
  if (n > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  PeArgs a{};
  for (int s = 0; s < slots; ++s) a.taus[s] = taus[s];
  pe_positions_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(pe_pos, Hp, Wp, static_cast<int>(n), a);
  return cudaGetLastError();
}

cudaError_t launch_pe_table(float* tab, int rows, int D, cudaStream_t st) {
  PeArgs a{};
  if (!pe_args(&a, D) || rows < 0) return cudaErrorInvalidValue;
  if (rows == 0) return cudaSuccess;
  pe_table_kernel<<<rows, 128, 0, st>>>(tab, rows, a);
  return cudaGetLastError();
}

cudaError_t launch_add_pe(float* x, int Hp, int Wp, int slots, const int* taus, int D, cudaStream_t st,
                          const int* taus_dev, const float* ptab, int ptab_rows) {
  PeArgs a{};
  a.taus_dev = taus_dev;
  a.Hp = Hp;
  a.Wp = Wp;
  if (!pe_args(&a, D) || slots > 8 || slots < 0 || Hp < 0 || Wp < 0) return cudaErrorInvalidValue;
  if (!taus_dev)
    for (int s = 0; s < slots; ++s) a.taus[s] = taus[s];
  if (ptab && (Wp > ptab_rows || Hp > ptab_rows)) ptab = nullptr;
  const long long hw = static_cast<long long>(Hp) * Wp;
  const long long blocks = static_cast<long long>(slots) * ((hw + kPeRun - 1) / kPeRun);
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFll || hw > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  const int threads = std::min(256, ((D / 4 + 31) / 32) * 32);
  add_pe_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(x, a, ptab);
  return cudaGetLastError();
}

cudaError_t launch_layernorm(const float* x, const float* g, const float* b, void* out, int M, int D, int out_bf16,
                             cudaStream_t st) {
  if (D % 4 != 0 || D > 4 * 32 * kLnMaxVec) return cudaErrorInvalidValue;
  if (M <= 0) return cudaSuccess;
  if (out_bf16)
    layernorm_kernel<1><<<(M + 7) / 8, 256, 0, st>>>(x, g, b, out, nullptr, M, D);
  else
    layernorm_kernel<0><<<(M + 7) / 8, 256, 0, st>>>(x, g, b, out, nullptr, M, D);
  return cudaGetLastError();
}

cudaError_t launch_layernorm_e4m3(const float* x, const float* g, const float* b, uint8_t* out, float* row_scale,
                                  int M, int D, cudaStream_t st) {
  if (D % 4 != 0 || D > 4 * 32 * kLnMaxVec || !row_scale) return cudaErrorInvalidValue;
  if (M <= 0) return cudaSuccess;
  layernorm_kernel<2><<<(M + 7) / 8, 256, 0, st>>>(x, g, b, out, row_scale, M, D);
  return cudaGetLastError();
}

cudaError_t launch_quantize_rows_e4m3(const float* x, int rows, int cols, uint8_t* q, float* scale, cudaStream_t st) {
  if (cols % 4 != 0 || cols <= 0 || rows < 0) return cudaErrorInvalidValue;
  if (rows == 0) return cudaSuccess;
  quantize_rows_e4m3_kernel<<<(rows + 7) / 8, 256, 0, st>>>(x, rows, cols, q, scale);
  return cudaGetLastError();
}

size_t depth_stats_scratch_bytes() { return sizeof(StatsScratch); }
size_t depth_stats_scratch_align() { return alignof(StatsScratch); }

cudaError_t launch_depth_stats(const uint16_t* d, int H, int W, size_t pitch, float* mu_sigma, void* scratch,
                               cudaStream_t st) {
  StatsScratch* sc = static_cast<StatsScratch*>(scratch);
  cudaError_t e = cudaMemsetAsync(sc->ticket, 0, sizeof(sc->ticket), st);
  if (e != cudaSuccess) return e;
  const long long total = static_cast<long long>(H) * W;
  const long long want = (total + kStatsThreads * 8 - 1) / (kStatsThreads * 8);
  const int blocks = static_cast<int>(want < 1 ? 1 : (want > kStatsBlocks ? kStatsBlocks : want));
  depth_stats_pass1<<<blocks, kStatsThreads, 0, st>>>(d, H, W, pitch, sc);
  depth_stats_pass2<<<blocks, kStatsThreads, 0, st>>>(d, H, W, pitch, sc, mu_sigma);
  return cudaGetLastError();
}

cudaError_t launch_blend(const BlendArgs& a, cudaStream_t st, const BlendArgs* dev) {
  if (a.p <= 0 || a.H % a.p || a.W % a.p || (a.C != 1 && a.C != 3)) return cudaErrorInvalidValue;
  if (a.p == 16) {
    const long long threads = static_cast<long long>(a.H) * (a.W / 8);
    if (threads == 0) return cudaSuccess;
    const unsigned grid = static_cast<unsigned>((threads + kBlendThreads - 1) / kBlendThreads);
    if (dev)
      blend16_kernel_dev<<<grid, kBlendThreads, 0, st>>>(dev);
    else
      blend16_kernel<<<grid, kBlendThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  const long long warps = static_cast<long long>(a.H) * ((a.W + 31) / 32);
  if (warps == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((warps * 32 + 255) / 256);
  if (dev)
    blend_kernel_dev<<<grid, 256, 0, st>>>(dev);
  else
    blend_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One CTA per destination row: the float32 row of x and the row of a
// (16-byte vectors).
__global__ void __launch_bounds__(128) gather_rows_kernel(const float* __restrict__ x, const uint8_t* __restrict__ a,
                                                          int elem_bytes, int D, const __grid_constant__ RowRuns runs,
                                                          float* __restrict__ xc, uint8_t* __restrict__ ac) {
  const int row = static_cast<int>(blockIdx.x);
  int i = 0;
  while (i + 1 < runs.n && runs.dst[i + 1] <= row) ++i;
  const size_t src = static_cast<size_t>(runs.src[i] + (row - runs.dst[i]));
  const uint4* xs = reinterpret_cast<const uint4*>(x + src * D);
  uint4* xd = reinterpret_cast<uint4*>(xc + static_cast<size_t>(row) * D);
  for (int c = threadIdx.x; c < D / 4; c += blockDim.x) xd[c] = xs[c];
  const size_t rb = static_cast<size_t>(D) * elem_bytes;
  const uint4* as = reinterpret_cast<const uint4*>(a + src * rb);
  uint4* ad = reinterpret_cast<uint4*>(ac + static_cast<size_t>(row) * rb);
  for (int c = threadIdx.x; c < static_cast<int>(rb / 16); c += blockDim.x) ad[c] = as[c];
}

cudaError_t launch_gather_rows(const float* x, const void* a, int elem_bytes, int D, const RowRuns& runs, float* xc,
                               void* ac, cudaStream_t st) {
  if (runs.n <= 0 || runs.n > kMaxSegments || D % 8 || (elem_bytes != 2 && elem_bytes != 4))
    return cudaErrorInvalidValue;
  const int rows = runs.dst[runs.n];
  if (rows <= 0) return cudaSuccess;
  gather_rows_kernel<<<rows, 128, 0, st>>>(x, static_cast<const uint8_t*>(a), elem_bytes, D, runs, xc,
                                           static_cast<uint8_t*>(ac));
  return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float* in, void* out, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  f32_to_bf16_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(in, static_cast<__nv_bfloat16*>(out), n);
  return cudaGetLastError();
}

}  // namespace revo
