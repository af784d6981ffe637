// Internal interfaces between the kernel files and the runtime.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

#include "revo.h"

namespace revo {

// GEMM epilogues (Y = A W^T + b, then):
enum Epilogue : int {
  kEpiF32 = 0,       // store float32
  kEpiBf16 = 1,      // store bf16
  kEpiGeluBf16 = 2,  // store bf16(gelu(.))
  kEpiResidF32 = 3,  // float32 out += .
  kEpiResidLn = 4,   // float32 out += ., then the LayerNorm of every completed row block (EpiAux)
  kEpiF32Pe = 6,     // store float32 (. + the position embedding of the row's token, EpiAux)
};

// GEMM tile widths: 128 or 256 output columns per tile of 128 rows (one CTA);
// kTilePair | 128 or kTilePair | 256: tiles of 256 rows on a CTA pair (two
// SMs, tcgen05.mma.cta_group::2), whose W tensor map has width/2-row boxes.
constexpr int kTilePair = 0x1000;
static_assert(kTilePair == REVO_TILE_PAIR, "internal and public pair flags agree");

constexpr int kMaxSegments = 64;
constexpr int kMaxRefs = 7;  // k <= 7

// Token segments (one per request) for attention: tokens attend within their
// segment only.  With `queries` set, only rows [q_begin[g], q_end[g]) of
// segment g are queries (the keys stay the whole segment) and only those
// output rows are written (tensor-core path; the FP32 path writes every row).
struct Segments {
  int n;
  int start[kMaxSegments + 1];
  bool queries;
  int q_begin[kMaxSegments], q_end[kMaxSegments];
};

// ---- tensor maps
bool encode_tmap_bf16_2d(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t row_stride_elems,
                         uint32_t box_rows, uint32_t box_cols);

bool encode_tmap_out_2d(CUtensorMap* map, const void* base, bool f32, uint64_t rows, uint64_t cols,
                        uint64_t row_stride_elems);

bool encode_tmap_u8_2d(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t row_stride_elems,
                       uint32_t box_rows);

// ---- GEMMs
// `c` is the output map (encode_tmap_out_2d): float32 for kEpiF32 and
// kEpiResidF32 (the residual epilogue adds into it), bf16 otherwise.  `bn` is a
// tile width (see kTilePair); `a` has 128-row boxes, `b` bn-row boxes, or
// bn/2-row boxes for a pair width.
// Operands of the fused epilogues.
// kEpiResidLn, a LayerNorm fused after a residual GEMM (x += A W^T + b): each
// CTA counts the column tiles it has added into a 128-row block of x; the one
// that completes the block normalises those rows (the standalone LayerNorm's
// arithmetic, bit for bit) into `out`.
// kEpiF32Pe, the position embedding added in the embedding GEMMs' epilogue:
// out[m][n] = (acc + b[n]) + pe(m, n) with the values launch_add_pe adds (the
// same float32 sums, bit for bit).  Row m's token has the temporal distance
// pe_pos[m].x and the patch position (row, column) = (pe_pos[m].y >> 16,
// pe_pos[m].y & 0xFFFF); column n lies in part n / pe_part (0 temporal, 1 row,
// 2 column), whose value at an integer position below pe_rows comes from
// pe_tab (launch_pe_table), else from sincosf with the frequencies pe_omega.
struct EpiAux {
  const float* x;     // the residual stream the GEMM adds into, [M][N] float32
  const float* g;     // gain [N]
  const float* b;     // shift [N]
  void* out;          // bf16 [M][N] (mode 1) or E4M3 codes [M][N] (mode 2)
  float* row_scale;   // mode 2: per-row scales [M]
  int* counters;      // [ceil(M / 128)] zero between launches (the last CTA resets its own)
  int mode;           // 1 bf16, 2 E4M3 with per-row scales
  const int2* pe_pos;      // [M] token positions
  const float* pe_tab;     // [pe_rows][pe_part]
  const float* pe_omega;   // [pe_part / 2]
  int pe_rows, pe_part;    // N == 3 * pe_part, pe_part % 64 == 0
  // Order of the K blocks (64 wide) for the RGB tubelet embedding with 16 x 16
  // patches (K = T * 3 * 256 in (t, c, y, x) order): 0 natural; 1 the three
  // channel blocks of each (frame t, patch-row quad) consecutive -- step i
  // takes block embed_kblock(i), so the implicit GEMM reads each pixel quad
  // once for all three channels.
  int kperm;
};
cudaError_t launch_gemm_tc(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, int bn, int epi,
                           const float* bias, int M, int N, int K, int* err, int num_sms, cudaStream_t st,
                           const EpiAux* ln = nullptr);
// FP8 (E4M3) operands with per-row scales of A (`row_scale`, M entries: one per
// token) and per-output-channel scales of W (`col_scale`, N entries):
// Y = epilogue(row_scale[m] * col_scale[n] * (A8 W8^T)[m][n] + b[n]).  `a` and
// `b` are encode_tmap_u8_2d maps (128-row / bn-row boxes).  K % 128 == 0;
// epilogues kEpiBf16 and kEpiGeluBf16.
cudaError_t launch_gemm_tc_fp8(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, int bn, int epi,
                               const float* bias, const float* row_scale, const float* col_scale, int M, int N, int K,
                               int* err, int num_sms, cudaStream_t st);

// Per-row E4M3 quantisation: scale[r] = max_k |x[r][k]| / 448 (1 for an
// all-zero row), q[r][k] = e4m3_satfinite(x[r][k] * (448 / max)).  x float32
// [rows][cols] (cols % 4 == 0), q [rows][cols].
cudaError_t launch_quantize_rows_e4m3(const float* x, int rows, int cols, uint8_t* q, float* scale, cudaStream_t st);
cudaError_t launch_gemm_simt(int epi, const float* A, const float* W, const float* bias, void* out, int ldo, int M,
                             int N, int K, cudaStream_t st);

// ---- attention (qkv [M][3D] row-major; out [M][D])
cudaError_t launch_attention_simt(const float* qkv, float* out, int M, int D, int heads, const Segments& seg,
                                  cudaStream_t st);
// `part` (attention_partial_bytes(...) bytes): each segment's work is cut into
// pieces that fill the SMs once, chosen from the segment's length alone; split
// units are merged by a second kernel.  Null: one CTA per (head, 256 queries)
// unit, no second kernel.  *launched: kernels enqueued.
cudaError_t launch_attention_tc(const CUtensorMap& qkv_map, void* out, int M, int D, int heads, const Segments& seg,
                                int* err, cudaStream_t st, float* part = nullptr, int num_sms = 0,
                                int* launched = nullptr);
// Partial-result bytes launch_attention_tc needs for these segments (0 if invalid).
size_t attention_partial_bytes(int M, int heads, const Segments& seg, int num_sms);
// The most any batch of up to n_seg segments of up to seg_len tokens needs.
size_t attention_partial_bytes_bound(int n_seg, int seg_len, int heads, int num_sms);
bool encode_attention_tmap(CUtensorMap* map, const void* qkv, int M, int D);

// ---- element-wise stages
struct AssembleArgs {
  const void* frames[kMaxRefs + 1];  // k refs oldest first, then the current frame
  size_t pitch[kMaxRefs + 1];        // bytes
  const float* mu_sigma;             // depth statistics (C == 1)
  void* out;                         // [S*Hp*Wp][T*C*p*p]
  int C, F, T, p, H, W;
  int out_bf16;
  // Optional (p = 16 kernels): each token's position for kEpiF32Pe,
  // pe_pos[(s*Hp + r)*Wp + c] = {taus[s], r << 16 | c}.
  int2* pe_pos;
  int taus[8];
};
// `dev` (optional): a device copy of `a` that the kernel reads instead of its
// by-value arguments (the launch shape still comes from `a`).
cudaError_t launch_assemble(const AssembleArgs& a, cudaStream_t st, const AssembleArgs* dev = nullptr);
// All n requests of a batch in one launch (p = 16): request i's arguments are
// read from the device at (const char*)dev + i * stride; `host` holds the same
// n argument sets (the launch shape: the largest request).
cudaError_t launch_assemble_batch(const AssembleArgs* host, int n, const AssembleArgs* dev, size_t stride,
                                  cudaStream_t st);

// The tubelet embedding as an implicit GEMM (p = 16): x[M][N] = tokens W^T + b
// + the position embedding, where the token rows are never stored: producer
// warps read each token's pixels straight from the frames of its request
// (the same normalisation as the assemble kernel, bit for bit) into the
// swizzled shared-memory operand, TMA streams W, tcgen05.mma accumulates in
// TMEM.  The batch's rows are the requests' tokens stacked in order: request
// i owns rows [seg_start[i], seg_start[i+1]) of Hp[i] x Wp[i] patches per
// slot; its frames, pitches, depth statistics and temporal distances are read
// from the device table at jobs + i * stride (AssembleArgs; the runtime writes
// it before each graph replay).  Each token's position {tau, r << 16 | c} is
// also written to pe_pos[row] for the encoder->decoder Linear's epilogue.
// K block taken at step i of the channel-grouped order (kperm 1).
__host__ __device__ inline int embed_kblock(int i) {
  const int t = i / 12, rem = i - 12 * t, yq = rem / 3, c = rem - 3 * yq;
  return (3 * t + c) * 4 + yq;
}

struct EmbedParams {
  int n, C, T;
  int seg_start[kMaxSegments + 1];
  int hp[kMaxSegments], wp[kMaxSegments];
  const uint8_t* jobs;
  size_t stride;
  int2* pe_pos;
};
// `w`: the embedding weight map (bn-row boxes, K-major bf16 [N][K] with K =
// T*C*256 in (t, c, y, x) order); `c`: the float32 output map (32-column boxes).
// bn 128 or 256; M = seg_start[n]; `pe` holds the embedding table operands.
cudaError_t launch_embed_tc(const CUtensorMap& w, const CUtensorMap& c, int bn, const float* bias, int M, int N,
                            int K, int* err, int num_sms, cudaStream_t st, const EpiAux& pe, const EmbedParams& ep);

// x[(s*Hp + r)*Wp + c][:] += sincos(tau_s) | sincos(r) | sincos(c), each D/3 wide
// (D a multiple of 192).  `taus_dev` (optional): device copy of the temporal
// distances, read instead of `taus`.  `ptab` (optional): launch_pe_table's
// table of a part at integer positions 0 .. ptab_rows-1, used for the row and
// the column parts (the same values as computing them).
cudaError_t launch_add_pe(float* x, int Hp, int Wp, int slots, const int* taus, int D, cudaStream_t st,
                          const int* taus_dev = nullptr, const float* ptab = nullptr, int ptab_rows = 0);
// tab[q][0 .. D/3) = the embedding's part at position q, for q < rows.
cudaError_t launch_pe_table(float* tab, int rows, int D, cudaStream_t st);
// The frequencies of a part at width D (D / 6 floats, host): false if D is not
// a multiple of 192 or above 1536.
bool pe_omega(int D, float* omega);
// pe_pos of one request's S*Hp*Wp tokens (see AssembleArgs::pe_pos).
cudaError_t launch_pe_positions(int2* pe_pos, int Hp, int Wp, int slots, const int* taus, cudaStream_t st);

cudaError_t launch_layernorm(const float* x, const float* g, const float* b, void* out, int M, int D, int out_bf16,
                             cudaStream_t st);
// LayerNorm whose output row is quantised to E4M3 with a per-row scale, the
// same rule as launch_quantize_rows_e4m3 applied to the float32 LN output.
cudaError_t launch_layernorm_e4m3(const float* x, const float* g, const float* b, uint8_t* out, float* row_scale,
                                  int M, int D, cudaStream_t st);

size_t depth_stats_scratch_bytes();
size_t depth_stats_scratch_align();
// Largest frame (height * width) the statistics accept: the pixel count must be
// exact in float32, where it divides the sum.
constexpr long long kDepthStatsMaxPixels = 1LL << 24;
cudaError_t launch_depth_stats(const uint16_t* d, int H, int W, size_t pitch, float* mu_sigma, void* scratch,
                               cudaStream_t st);

struct BlendArgs {
  int C, p, H, W;
  const float* head;  // [Hp*Wp][C*p*p]
  const void* decoded;
  size_t pitch;
  const uint32_t* mask;
  size_t mask_pitch;  // words
  const float* mu_sigma;
  void* out;
  size_t out_pitch;
  float* values;  // optional dense [H][W][C]
};
cudaError_t launch_blend(const BlendArgs& a, cudaStream_t st, const BlendArgs* dev = nullptr);
cudaError_t launch_blend_batch(const BlendArgs* host, int n, const BlendArgs* dev, size_t stride, cudaStream_t st);

cudaError_t launch_f32_to_bf16(const float* in, void* out, size_t n, cudaStream_t st);

// Row gather: for each of n runs, rows [src[i], src[i] + (dst[i+1] - dst[i]))
// of x (float32 [.][D]) and a (elem_bytes 2 or 4, [.][D]) go to rows
// [dst[i], dst[i+1]) of xc and ac.  D % 8 == 0.
struct RowRuns {
  int n;
  int src[kMaxSegments];
  int dst[kMaxSegments + 1];
};
cudaError_t launch_gather_rows(const float* x, const void* a, int elem_bytes, int D, const RowRuns& runs, float* xc,
                               void* ac, cudaStream_t st);

// Reed-Solomon erasure code of I-frame packets over GF(2^8) (systematic,
// Cauchy parity rows): encode n data packets into r parity packets; decode n
// received packets (indices `present`, data 0..n-1, parity n..n+r-1) into the
// n data packets.  packet_bytes and pitches multiples of 4; n + r <= 256.
cudaError_t fec_encode(int n, int r, size_t packet_bytes, const uint8_t* data, size_t data_pitch, uint8_t* parity,
                       size_t parity_pitch, cudaStream_t st);
size_t fec_decode_scratch_bytes(int n);
cudaError_t fec_decode(int n, int r, size_t packet_bytes, const int* present, const uint8_t* received,
                       size_t received_pitch, uint8_t* data_out, size_t out_pitch, void* scratch, cudaStream_t st);

// RGB-D unprojection + point splatting (render.cu).
struct RenderCall {
  const uint8_t* rgb;
  size_t rgb_pitch;
  int rgb_h, rgb_w;
  const uint16_t* depth;
  size_t depth_pitch;
  int h, w;
  float src[4], r[9], t[3], dst[4];  // intrinsics (fx, fy, cx, cy), pose x' = R x + t
  int out_h, out_w, splat;
  void* scratch;  // render_scratch_bytes(out_h, out_w)
  uint8_t* out_rgb;
  size_t out_rgb_pitch;
  uint16_t* out_depth;
  size_t out_depth_pitch;
};
size_t render_scratch_bytes(int out_h, int out_w);
cudaError_t launch_render(const RenderCall& c, cudaStream_t st);

// SSIM and PSNR of frame a against frame b (uint8 or uint16 samples, C = 1
// or 3 interleaved): out[0] = mean SSIM, out[1] = MSE, out[2] = PSNR (dB).
size_t frame_metrics_scratch_bytes(int H, int W, int C);
cudaError_t launch_frame_metrics(const void* a, size_t pitch_a, const void* b, size_t pitch_b, int H, int W, int C,
                                 int sample_bytes, float data_range, float* out, void* scratch, cudaStream_t st);

int device_sm_count();

// Raises a kernel's dynamic shared-memory limit once per device (the attribute
// call costs microseconds; launches happen hundreds of times per frame).
// `done` is the caller's per-kernel mask of devices already set (bit = ordinal).
template <typename Kernel>
cudaError_t ensure_smem_attr(Kernel k, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && (done.load(std::memory_order_acquire) >> dev) & 1ull) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev, std::memory_order_release);
  return e;
}

// ---- errors
void set_last_error(const char* fmt, ...);
revo_status cuda_status(cudaError_t e, const char* what);

}  // namespace revo
