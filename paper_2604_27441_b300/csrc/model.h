// The recovery network on the device: weights, work arena, and the forward of
// a ragged batch of same-modality requests whose tokens are concatenated
// along the row dimension of every activation matrix.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "revo_internal.h"

namespace revo {

struct NetShape {
  int C, k, T, p;
  int D, L, H;     // encoder width, blocks, heads
  int Dd, Ld, Hd;  // decoder width, blocks, heads
  int r;           // MLP ratio
  int frames() const { return k + 1; }
  int slots() const { return (k + 1) / T; }
  int token_dim() const { return T * C * p * p; }
  int head_dim_out() const { return C * p * p; }  // head rows kept: the last frame of a tubelet
};

size_t param_count(const NetShape& s);
// Empty string if the shape is supported by the kernels, else the reason.
std::string check_shape(const NetShape& s);

struct LinearW {
  const float* w32 = nullptr;
  const float* b = nullptr;
  const __nv_bfloat16* w16 = nullptr;
  int out = 0, in = 0;
  CUtensorMap map64{}, map128{}, map256{};  // W boxes of 64 / 128 / 256 rows
  // FP8 precision, the LayerNorm-fed layers (qkv, fc1): E4M3 codes with one
  // scale per output channel, and their maps.
  const uint8_t* w8 = nullptr;
  const float* w8_scale = nullptr;
  CUtensorMap map8_64{}, map8_128{}, map8_256{};
};

struct BlockW {
  const float *ln1g, *ln1b, *ln2g, *ln2b;
  LinearW qkv, proj, fc1, fc2;
};

struct Net {
  NetShape s{};
  int precision = 0;
  float* blob = nullptr;            // float32 master copy of every parameter
  __nv_bfloat16* blob16 = nullptr;  // bf16 copy (tensor-core path)
  uint8_t* blob8 = nullptr;         // E4M3 copies of the qkv and fc1 weights (FP8 precision)
  float* blob8_scale = nullptr;     // their per-output-channel scales
  LinearW patch, enc2dec, head;     // head: the rows that produce the target frame
  std::vector<BlockW> enc, dec;
  const float *enc_norm_g, *enc_norm_b, *dec_norm_g, *dec_norm_b;
  // GEMM tile-width autotuner (tensor-core path): choices per shape key
  // (tune_key), timed at create by net_autotune or read from a cache file.
  // Off, or a shape without a choice: a fixed rule (256 when N >= 256).
  bool autotune = false;
  // FP8 precision: E4M3 layers (bit 0 encoder qkv, 1 encoder fc1, 2 decoder
  // qkv, 3 decoder fc1).
  int fp8_mask = 0;
  std::map<uint64_t, int> tuned_bn;
  int tuned_shapes_256 = 0, tuned_shapes_128 = 0, tuned_shapes_pair = 0;
};

// One request of one modality inside a batch (all pointers are device pointers).
struct PlaneJob {
  int H, W;
  const void* frames[kMaxRefs + 1];  // k refs (oldest first) then the decoded current frame
  size_t pitch[kMaxRefs + 1];
  const uint32_t* mask;
  size_t mask_pitch;  // words
  const float* mu_sigma;  // depth statistics (C == 1)
  int taus[8];            // temporal distance per slot
  void* out;              // blended frame
  size_t out_pitch;
  float* values;          // optional dense float32 output
};

struct Workspace {
  int cap_tokens = 0, cap_patches = 0;
  void* tok = nullptr;   // [cap][T*C*p*p]
  float* x = nullptr;    // [cap][D]   residual stream
  void* h = nullptr;     // [cap][D]   LayerNorm output
  void* qkv = nullptr;   // [cap][3D]
  void* att = nullptr;   // [cap][D]
  void* mlp = nullptr;   // [cap][rD]
  float* head = nullptr; // [cap_patches][C*p*p]
  // The last decoder block's rows (the final slot of each request, stacked):
  float* xc = nullptr;    // [cap_patches][D'] residual stream
  void* attc = nullptr;   // [cap_patches][D'] attention output
  // The position embedding's part at integer positions 0 .. pe_rows-1, at
  // the encoder and the decoder width (launch_pe_table).
  float* pe_enc = nullptr;
  float* pe_dec = nullptr;
  int pe_rows = 0;
  float* pe_om_enc = nullptr;  // the parts' frequencies at the two widths
  float* pe_om_dec = nullptr;
  int2* pe_pos = nullptr;      // [cap] each token's temporal distance and patch position (assemble writes it)
  uint8_t* h8 = nullptr;  // [cap][max width] E4M3 LayerNorm output (FP8 precision)
  float* h8_scale = nullptr;  // [cap] its per-token scales
  int sms = 0;
  int* err = nullptr;    // device error word of the tensor-core kernels
  size_t bytes = 0;
  // Tensor maps of the A operands, valid for `maps_rows` rows.
  int maps_rows = -1;
  CUtensorMap m_tok{}, m_h_enc{}, m_att_enc{}, m_mlp_enc{}, m_h_dec{}, m_att_dec{}, m_mlp_dec{};
  CUtensorMap m_qkv_enc{}, m_qkv_dec{};
  CUtensorMap m_h8_enc{}, m_h8_dec{};
  // Output maps of the GEMM epilogues.
  CUtensorMap o_x_enc{}, o_x_dec{}, o_qkv_enc{}, o_qkv_dec{}, o_mlp_enc{}, o_mlp_dec{};
  // Maps of the last decoder block's stacked rows, valid for `maps_rows_c` rows.
  int maps_rows_c = -1;
  CUtensorMap c_h{}, c_att{}, c_mlp{}, c_h8{}, c_o_x{}, c_o_mlp{}, c_o_head{};
};

Net* net_create(const NetShape& s, int precision, const float* host_weights, std::string* err);
void net_destroy(Net* n);
size_t net_bytes(const NetShape& s, int precision);

// max_segments: requests per batch; max_wp: patch rows or columns of the largest frame.
size_t workspace_bytes(const NetShape& s, int precision, int cap_tokens, int cap_patches, int max_segments,
                       int max_wp);
Workspace* workspace_create(const NetShape& s, int precision, int cap_tokens, int cap_patches, int max_segments,
                            int max_wp, std::string* err);
void workspace_destroy(Workspace* w);

// Tokens of one request of height H and width W.
inline int request_tokens(const NetShape& s, int H, int W) { return s.slots() * (H / s.p) * (W / s.p); }
inline int request_patches(const NetShape& s, int H, int W) { return (H / s.p) * (W / s.p); }

// The per-request kernel arguments of a batch: everything that changes from one
// batch to the next when the request sizes do not (frame, mask, output and
// statistics pointers; temporal distances).  A batch whose sizes match an
// earlier one can replay that batch's captured graph after writing these.
struct JobArgs {
  AssembleArgs assemble;
  BlendArgs blend;
  int taus[8];
};

// Fills args[0..n) for `jobs` (host only; the token offsets follow from the sizes).
cudaError_t prepare_job_args(const Net* net, const Workspace* ws, const PlaneJob* jobs, int n, JobArgs* args);

// Enqueues the whole forward (assemble ... blend) of `n` jobs on `st`; *launches
// receives the number of kernels enqueued.  With `dev_args` (a device copy of
// prepare_job_args' output, written before the kernels run) the per-request
// kernels read their arguments from it instead of taking them by value, so the
// enqueued work depends on the request sizes only and can be captured once.
cudaError_t net_forward(Net* net, Workspace* ws, const PlaneJob* jobs, int n, cudaStream_t st, int num_sms,
                        int* launches, const JobArgs* dev_args = nullptr);

// GEMM tile autotuning (tensor-core path), done once at create: every GEMM
// shape of the network is timed for the row counts of tune_bucket's ladder up
// to max_tokens (the head up to max_patches) on `ws` and `st`, skipping shapes
// that already have a choice (from an autotune cache file).  A forward then
// only looks the choices up.
cudaError_t net_autotune(Net* net, Workspace* ws, int max_tokens, int max_patches, cudaStream_t st, int num_sms);
int tune_bucket(int M);
uint64_t tune_key(int M, int N, int K, bool f8, int epi);

// Host-side weight sources (weights.cu): the documented random initialisation
// of a model from a seed, and a flat float32 file.
void init_weights_random(const NetShape& s, uint64_t seed, float* out);
bool load_weights_file(const char* path, size_t offset_floats, size_t count, float* out, std::string* why);

}  // namespace revo
