// FP32 Linear layers on the CUDA cores (plain FMA, no TF32): the full-precision
// path of the recovery network.  Y = epilogue(A W^T + b), A [M][K], W [N][K]
// (Linear [out][in]), both K-contiguous.  128 x 128 output tile per CTA,
// 256 threads x (8 x 8) outputs, K step 8, double-buffered shared memory.
// K must be a multiple of 8 and A, W 16-byte aligned.
#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr int kT = 128;
constexpr int kKs = 8;
constexpr int kPad = 4;

template <int EPI>
__global__ void __launch_bounds__(256) sgemm_kernel(const float* __restrict__ A, const float* __restrict__ W,
                                                    const float* __restrict__ bias, float* __restrict__ out,
                                                    int ldo, int M, int N, int K) {
  __shared__ __align__(16) float As[2][kKs][kT + kPad];
  __shared__ __align__(16) float Bs[2][kKs][kT + kPad];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * kT;
  const int n0 = blockIdx.x * kT;
  const int lrow = tid >> 1;
  const int lk = (tid & 1) * 4;
  const bool a_ok = (m0 + lrow) < M;
  const bool b_ok = (n0 + lrow) < N;
  const float* Ap = A + static_cast<size_t>(a_ok ? m0 + lrow : 0) * K + lk;
  const float* Wp = W + static_cast<size_t>(b_ok ? n0 + lrow : 0) * K + lk;
  const int tx = tid & 15;
  const int ty = tid >> 4;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 ra = a_ok ? __ldg(reinterpret_cast<const float4*>(Ap)) : zero;
  float4 rb = b_ok ? __ldg(reinterpret_cast<const float4*>(Wp)) : zero;
  auto stash = [&](int buf) {
    As[buf][lk + 0][lrow] = ra.x;
    As[buf][lk + 1][lrow] = ra.y;
    As[buf][lk + 2][lrow] = ra.z;
    As[buf][lk + 3][lrow] = ra.w;
    Bs[buf][lk + 0][lrow] = rb.x;
    Bs[buf][lk + 1][lrow] = rb.y;
    Bs[buf][lk + 2][lrow] = rb.z;
    Bs[buf][lk + 3][lrow] = rb.w;
  };
  stash(0);
  __syncthreads();

  const int nk = K / kKs;
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      ra = a_ok ? __ldg(reinterpret_cast<const float4*>(Ap + (kt + 1) * kKs)) : zero;
      rb = b_ok ? __ldg(reinterpret_cast<const float4*>(Wp + (kt + 1) * kKs)) : zero;
    }
#pragma unroll
    for (int kk = 0; kk < kKs; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) stash(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (row >= M) continue;
#pragma unroll
    for (int jh = 0; jh < 2; ++jh) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = n0 + jh * 64 + tx * 4 + j;
        if (col >= N) continue;
        float v = acc[i][jh * 4 + j] + (bias ? bias[col] : 0.f);
        if (EPI == kEpiGeluBf16) v = gelu_exact(v);
        float* o = out + static_cast<size_t>(row) * ldo + col;
        if (EPI == kEpiResidF32)
          *o += v;
        else
          *o = v;
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_simt(int epi, const float* A, const float* W, const float* bias, void* out, int ldo, int M,
                             int N, int K, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K % kKs != 0) return cudaErrorInvalidValue;
  dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  float* o = static_cast<float*>(out);
  switch (epi) {
    case kEpiF32:
    case kEpiBf16: sgemm_kernel<kEpiF32><<<grid, 256, 0, st>>>(A, W, bias, o, ldo, M, N, K); break;
    case kEpiGeluBf16: sgemm_kernel<kEpiGeluBf16><<<grid, 256, 0, st>>>(A, W, bias, o, ldo, M, N, K); break;
    case kEpiResidF32: sgemm_kernel<kEpiResidF32><<<grid, 256, 0, st>>>(A, W, bias, o, ldo, M, N, K); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace revo
