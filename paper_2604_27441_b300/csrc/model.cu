// The recovery network on the device (Section 3.4.1, Appendix B.1, B.3):
// tubelet embedding + (temporal distance, row, column) embedding, pre-LN
// encoder blocks, final LN, encoder->decoder Linear + decoder embedding, pre-LN
// decoder blocks, final LN and the pixel head for the target frame, then the
// masked blend.  A batch of same-modality requests runs as one forward whose
// Linear layers see every request's tokens stacked along the rows; attention
// keeps each request's tokens to themselves (one segment per request).
#include <string.h>

#include <algorithm>

#include "model.h"

namespace revo {

namespace {

size_t block_params(int d, int r) {
  return 2ull * d + (3ull * d * d + 3ull * d) + (1ull * d * d + d) + 2ull * d + (1ull * r * d * d + 1ull * r * d) +
         (1ull * r * d * d + d);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// GEMM row counts share a tile choice within buckets: multiples of 128 rows
// up to 8192 (where the number of 128-row tiles against the SM count decides
// the choice), powers of two above; a launch of M rows uses the choice timed
// at its bucket's top.
int tune_bucket(int M) {
  if (M <= 8192) return ((std::max(M, 1) + 127) / 128) * 128;
  int b = 16384;
  while (b < M && b < (1 << 30)) b *= 2;
  return b;
}

// The next bucket after b (the autotuner's ladder of row counts).
int next_tune_bucket(int b) { return b < 8192 ? b + 128 : b * 2; }

uint64_t tune_key(int M, int N, int K, bool f8, int epi) {
  return (static_cast<uint64_t>(tune_bucket(M)) << 36) | (static_cast<uint64_t>(N) << 22) |
         (static_cast<uint64_t>(K) << 4) | (static_cast<uint64_t>(f8) << 3) | static_cast<uint64_t>(epi);
}

namespace {

// 128 x 256 tiles halve the A-operand traffic per FLOP and measured faster than
// 128 x 128 at every Linear shape of the network (also with fewer tiles than
// SMs), so they are used whenever N allows.
int pick_bn(int /*M*/, int N, int /*sms*/) { return N >= 256 ? 256 : 128; }

bool make_weight_maps(LinearW& w) {
  if (!w.w16) return true;
  // 64-row boxes serve the CTA-pair tiles of width 128 (each CTA loads half
  // of the W rows), 128-row boxes the single tiles of width 128 and the pair
  // tiles of width 256, 256-row boxes the single tiles of width 256.
  if (!encode_tmap_bf16_2d(&w.map64, w.w16, w.out, w.in, w.in, 64, 64)) return false;
  if (!encode_tmap_bf16_2d(&w.map128, w.w16, w.out, w.in, w.in, 128, 64)) return false;
  if (w.out >= 256 && !encode_tmap_bf16_2d(&w.map256, w.w16, w.out, w.in, w.in, 256, 64)) return false;
  if (w.w8) {
    if (!encode_tmap_u8_2d(&w.map8_64, w.w8, w.out, w.in, w.in, 64)) return false;
    if (!encode_tmap_u8_2d(&w.map8_128, w.w8, w.out, w.in, w.in, 128)) return false;
    if (w.out >= 256 && !encode_tmap_u8_2d(&w.map8_256, w.w8, w.out, w.in, w.in, 256)) return false;
  }
  return true;
}

// E4M3 weight elements (and scales) of the FP8 layers: qkv and fc1 of every block.
size_t fp8_block_elems(int d, int r) { return 3ull * d * d + 1ull * r * d * d; }
size_t fp8_block_rows(int d, int r) { return 3ull * d + 1ull * r * d; }

}  // namespace

size_t param_count(const NetShape& s) {
  const size_t D = s.D, Dd = s.Dd, K = s.token_dim();
  return D * K + D + s.L * block_params(s.D, s.r) + 2 * D + Dd * D + Dd + s.Ld * block_params(s.Dd, s.r) + 2 * Dd +
         K * Dd + K;
}

std::string check_shape(const NetShape& s) {
  if (s.C != 1 && s.C != 3) return "channels must be 1 or 3";
  if (s.k < 1 || s.k > kMaxRefs) return "k must be in 1..7";
  if (s.T < 1 || (s.k + 1) % s.T) return "(k + 1) must be a multiple of the tubelet size";
  if (s.slots() > 8) return "at most 8 tubelet slots";
  if (s.p != 16) return "patch size must be 16";
  if (s.D % 64 || s.Dd % 64 || s.D <= 0 || s.Dd <= 0) return "widths must be positive multiples of 64";
  if (s.D % 6 || s.Dd % 6) return "widths must split into three even embedding parts";
  if (s.D > 1024 || s.Dd > 1024) return "widths above 1024 are not supported";
  if (s.H * 64 != s.D || s.Hd * 64 != s.Dd) return "head width must be 64";
  if (s.r < 1 || s.L < 0 || s.Ld < 1) return "bad depth or MLP ratio";
  return "";
}

size_t net_bytes(const NetShape& s, int precision) {
  const size_t n = param_count(s);
  size_t b = align_up(n * 4, 256) + (precision != REVO_FP32 ? align_up(n * 2, 256) : 0);
  if (precision == REVO_FP8) {
    b += align_up(s.L * fp8_block_elems(s.D, s.r) + s.Ld * fp8_block_elems(s.Dd, s.r), 256);
    b += align_up(4 * (s.L * fp8_block_rows(s.D, s.r) + s.Ld * fp8_block_rows(s.Dd, s.r)), 256);
  }
  return b;
}

Net* net_create(const NetShape& s, int precision, const float* host_weights, std::string* err) {
  Net* net = new Net();
  net->s = s;
  net->precision = precision;
  const size_t n = param_count(s);
  const bool tc = precision != REVO_FP32;
  if (cudaMalloc(&net->blob, n * 4) != cudaSuccess ||
      cudaMemcpy(net->blob, host_weights, n * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "weight upload failed";
    net_destroy(net);
    return nullptr;
  }
  if (tc) {
    if (cudaMalloc(&net->blob16, n * 2) != cudaSuccess || launch_f32_to_bf16(net->blob, net->blob16, n, 0) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
      *err = "bf16 weight copy failed";
      net_destroy(net);
      return nullptr;
    }
  }
  size_t off = 0;
  auto take = [&](size_t count) {
    const size_t o = off;
    off += count;
    return o;
  };
  auto lin = [&](int out, int in) {
    LinearW w;
    w.out = out;
    w.in = in;
    const size_t ow = take(static_cast<size_t>(out) * in);
    const size_t ob = take(out);
    w.w32 = net->blob + ow;
    w.b = net->blob + ob;
    if (tc) w.w16 = net->blob16 + ow;
    return w;
  };
  auto block = [&](int d) {
    BlockW b;
    b.ln1g = net->blob + take(d);
    b.ln1b = net->blob + take(d);
    b.qkv = lin(3 * d, d);
    b.proj = lin(d, d);
    b.ln2g = net->blob + take(d);
    b.ln2b = net->blob + take(d);
    b.fc1 = lin(s.r * d, d);
    b.fc2 = lin(d, s.r * d);
    return b;
  };
  net->patch = lin(s.D, s.token_dim());
  for (int i = 0; i < s.L; ++i) net->enc.push_back(block(s.D));
  net->enc_norm_g = net->blob + take(s.D);
  net->enc_norm_b = net->blob + take(s.D);
  net->enc2dec = lin(s.Dd, s.D);
  for (int i = 0; i < s.Ld; ++i) net->dec.push_back(block(s.Dd));
  net->dec_norm_g = net->blob + take(s.Dd);
  net->dec_norm_b = net->blob + take(s.Dd);
  {
    // Keep only the head rows of the tubelet's last frame (the target frame).
    const int K = s.token_dim(), Cpp = s.head_dim_out();
    const size_t ow = take(static_cast<size_t>(K) * s.Dd);
    const size_t ob = take(K);
    const size_t row0 = static_cast<size_t>(s.T - 1) * Cpp;
    LinearW w;
    w.out = Cpp;
    w.in = s.Dd;
    w.w32 = net->blob + ow + row0 * s.Dd;
    w.b = net->blob + ob + row0;
    if (tc) w.w16 = net->blob16 + ow + row0 * s.Dd;
    net->head = w;
  }
  if (off != n) {
    *err = "internal parameter layout mismatch";
    net_destroy(net);
    return nullptr;
  }
  if (precision == REVO_FP8) {
    // Per-output-channel E4M3 copies of the LayerNorm-fed layers.
    const size_t elems = s.L * fp8_block_elems(s.D, s.r) + s.Ld * fp8_block_elems(s.Dd, s.r);
    const size_t rows = s.L * fp8_block_rows(s.D, s.r) + s.Ld * fp8_block_rows(s.Dd, s.r);
    if (cudaMalloc(&net->blob8, elems) != cudaSuccess || cudaMalloc(&net->blob8_scale, rows * 4) != cudaSuccess) {
      *err = "fp8 weight allocation failed";
      net_destroy(net);
      return nullptr;
    }
    size_t eo = 0, ro = 0;
    bool ok = true;
    auto quant = [&](LinearW& w) {
      w.w8 = net->blob8 + eo;
      w.w8_scale = net->blob8_scale + ro;
      ok = ok && launch_quantize_rows_e4m3(w.w32, w.out, w.in, net->blob8 + eo, net->blob8_scale + ro, 0) ==
                     cudaSuccess;
      eo += static_cast<size_t>(w.out) * w.in;
      ro += w.out;
    };
    for (auto& b : net->enc) {
      quant(b.qkv);
      quant(b.fc1);
    }
    for (auto& b : net->dec) {
      quant(b.qkv);
      quant(b.fc1);
    }
    if (!ok || eo != elems || ro != rows || cudaDeviceSynchronize() != cudaSuccess) {
      *err = "fp8 weight quantisation failed";
      net_destroy(net);
      return nullptr;
    }
  }
  if (tc) {
    bool ok = make_weight_maps(net->patch) && make_weight_maps(net->enc2dec) && make_weight_maps(net->head);
    for (auto& b : net->enc)
      ok = ok && make_weight_maps(b.qkv) && make_weight_maps(b.proj) && make_weight_maps(b.fc1) &&
           make_weight_maps(b.fc2);
    for (auto& b : net->dec)
      ok = ok && make_weight_maps(b.qkv) && make_weight_maps(b.proj) && make_weight_maps(b.fc1) &&
           make_weight_maps(b.fc2);
    if (!ok) {
      *err = "weight tensor map encoding failed";
      net_destroy(net);
      return nullptr;
    }
  }
  return net;
}

void net_destroy(Net* n) {
  if (!n) return;
  if (n->blob) cudaFree(n->blob);
  if (n->blob16) cudaFree(n->blob16);
  if (n->blob8) cudaFree(n->blob8);
  if (n->blob8_scale) cudaFree(n->blob8_scale);
  delete n;
}

namespace {
// Rows of the position-embedding tables: every patch row and column of the
// largest frame, and temporal distances up to 63 (larger ones are computed).
int pe_table_rows(int max_wp) { return max_wp > 64 ? max_wp : 64; }

struct WsLayout {
  size_t tok, x, h, qkv, att, mlp, head, xc, attc, pe_enc, pe_dec, pe_om, pe_pos, err, h8, h8s, part, total;
};
WsLayout ws_layout(const NetShape& s, int precision, int cap, int capp, int max_seg, int max_wp) {
  const size_t e = precision != REVO_FP32 ? 2 : 4;
  const size_t D = s.D > s.Dd ? s.D : s.Dd;
  WsLayout l{};
  size_t o = 0;
  auto put = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  l.tok = put(static_cast<size_t>(cap) * s.token_dim() * e);
  l.x = put(static_cast<size_t>(cap) * D * 4);
  l.h = put(static_cast<size_t>(cap) * D * e);
  l.qkv = put(static_cast<size_t>(cap) * 3 * D * e);
  l.att = put(static_cast<size_t>(cap) * D * e);
  l.mlp = put(static_cast<size_t>(cap) * s.r * D * e);
  l.head = put(static_cast<size_t>(capp) * s.head_dim_out() * 4);
  l.xc = put(static_cast<size_t>(capp) * s.Dd * 4);
  l.attc = put(static_cast<size_t>(capp) * s.Dd * e);
  const int pe_rows = pe_table_rows(max_wp);
  l.pe_enc = put(static_cast<size_t>(pe_rows) * (s.D / 3) * 4);
  l.pe_dec = put(static_cast<size_t>(pe_rows) * (s.Dd / 3) * 4);
  l.pe_om = put(2 * 128 * 4);
  l.pe_pos = put(static_cast<size_t>(cap) * sizeof(int2));
  l.err = put(256);
  if (precision == REVO_FP8) {
    l.h8 = put(static_cast<size_t>(cap) * D);
    l.h8s = put(static_cast<size_t>(cap) * 4);
  }
  l.total = o;
  return l;
}
}  // namespace

size_t workspace_bytes(const NetShape& s, int precision, int cap_tokens, int cap_patches, int max_segments,
                       int max_wp) {
  return ws_layout(s, precision, cap_tokens, cap_patches, max_segments, max_wp).total;
}

Workspace* workspace_create(const NetShape& s, int precision, int cap_tokens, int cap_patches, int max_segments,
                            int max_wp, std::string* err) {
  const WsLayout l = ws_layout(s, precision, cap_tokens, cap_patches, max_segments, max_wp);
  uint8_t* base = nullptr;
  if (cudaMalloc(&base, l.total) != cudaSuccess) {
    *err = "workspace allocation failed";
    return nullptr;
  }
  // Zero once so that rows never written by a request stay finite.
  if (cudaMemset(base, 0, l.total) != cudaSuccess) {
    cudaFree(base);
    *err = "workspace clear failed";
    return nullptr;
  }
  Workspace* w = new Workspace();
  w->cap_tokens = cap_tokens;
  w->cap_patches = cap_patches;
  w->tok = base + l.tok;
  w->x = reinterpret_cast<float*>(base + l.x);
  w->h = base + l.h;
  w->qkv = base + l.qkv;
  w->att = base + l.att;
  w->mlp = base + l.mlp;
  w->head = reinterpret_cast<float*>(base + l.head);
  w->xc = reinterpret_cast<float*>(base + l.xc);
  w->attc = base + l.attc;
  w->pe_enc = reinterpret_cast<float*>(base + l.pe_enc);
  w->pe_dec = reinterpret_cast<float*>(base + l.pe_dec);
  w->pe_rows = pe_table_rows(max_wp);
  w->pe_om_enc = reinterpret_cast<float*>(base + l.pe_om);
  w->pe_om_dec = w->pe_om_enc + 128;
  w->pe_pos = reinterpret_cast<int2*>(base + l.pe_pos);
  float om[2][128] = {};
  if (!pe_omega(s.D, om[0]) || !pe_omega(s.Dd, om[1]) ||
      cudaMemcpy(w->pe_om_enc, om, sizeof(om), cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_pe_table(w->pe_enc, w->pe_rows, s.D, 0) != cudaSuccess ||
      launch_pe_table(w->pe_dec, w->pe_rows, s.Dd, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(base);
    delete w;
    *err = "position embedding tables failed";
    return nullptr;
  }
  w->err = reinterpret_cast<int*>(base + l.err);
  w->sms = device_sm_count();
  if (precision == REVO_FP8) {
    w->h8 = base + l.h8;
    w->h8_scale = reinterpret_cast<float*>(base + l.h8s);
  }
  w->bytes = l.total;
  return w;
}

void workspace_destroy(Workspace* w) {
  if (!w) return;
  if (w->tok) cudaFree(w->tok);  // the arena's base
  delete w;
}

namespace {

struct Fwd {
  Net* net;
  Workspace* ws;
  cudaStream_t st;
  int sms;
  bool tc;
  size_t e;  // activation element size
  int launched = 0;  // kernels enqueued so far

  // `amap` / `cmap`: the A operand and output tensor maps (tensor-core path).
  // `aux`: the operands of a fused epilogue (kEpiF32Pe; tile choice as kEpiF32).
  cudaError_t linear(const CUtensorMap* amap, const void* A, const LinearW& w, int epi, void* out, int ldo, int M,
                     const CUtensorMap* cmap, const EpiAux* aux = nullptr) {
    ++launched;
    if (!tc) return launch_gemm_simt(epi, static_cast<const float*>(A), w.w32, w.b, out, ldo, M, w.out, w.in, st);
    int bn = pick_bn(M, w.out, sms);
    if (net->autotune && M > 0) {
      cudaError_t e = tuned_width(amap, w, epi == kEpiF32Pe ? kEpiF32 : epi, M, cmap, false, &bn);
      if (e != cudaSuccess) return e;
    }
    return launch(amap, w, epi, M, false, bn, cmap, aux);
  }

  // FP8 Linear: A = the E4M3 LayerNorm output with its per-token scales.
  cudaError_t linear8(const CUtensorMap* amap, const LinearW& w, int epi, int M, const CUtensorMap* cmap) {
    ++launched;
    int bn = pick_bn(M, w.out, sms);
    if (net->autotune && M > 0) {
      cudaError_t e = tuned_width(amap, w, epi, M, cmap, true, &bn);
      if (e != cudaSuccess) return e;
    }
    return launch(amap, w, epi, M, true, bn, cmap);
  }

  // One launch of tile width bn (see kTilePair) writing through `dst`.
  cudaError_t launch(const CUtensorMap* amap, const LinearW& w, int epi, int M, bool f8, int bn,
                     const CUtensorMap* dst, const EpiAux* aux = nullptr) {
    const int rows = (bn & kTilePair) ? (bn & ~kTilePair) / 2 : bn;  // W rows per CTA and tile
    if (f8)
      return launch_gemm_tc_fp8(*amap, rows == 256 ? w.map8_256 : rows == 128 ? w.map8_128 : w.map8_64, *dst, bn,
                                epi, w.b, ws->h8_scale, w.w8_scale, M, w.out, w.in, ws->err, sms, st);
    return launch_gemm_tc(*amap, rows == 256 ? w.map256 : rows == 128 ? w.map128 : w.map64, *dst, bn, epi, w.b, M,
                          w.out, w.in, ws->err, sms, st, aux);
  }

  // The autotuner's choice for this shape.  While serving (tuning == false)
  // only the choices timed at create are looked up: no request waits for
  // tuning.  At create (tuning == true) a shape without a choice has its
  // candidates timed on the stream.  The timed launches write the GEMM's own
  // destination (the real launch overwrites it next), except for the residual
  // epilogue, whose destination accumulates: those write into the qkv buffer,
  // which holds nothing live between attention and the next block.
  bool tuning = false;
  cudaError_t tuned_width(const CUtensorMap* amap, const LinearW& w, int epi, int M, const CUtensorMap* cmap, bool f8,
                          int* bn) {
    const uint64_t key = tune_key(M, w.out, w.in, f8, epi);
    auto it = net->tuned_bn.find(key);
    if (it != net->tuned_bn.end()) {
      *bn = it->second;
      return cudaSuccess;
    }
    if (!tuning) return cudaSuccess;  // keep the default rule
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t rc = cudaStreamIsCapturing(st, &cap);
    if (rc != cudaSuccess || cap != cudaStreamCaptureStatusNone) return rc;
    CUtensorMap scratch;
    const CUtensorMap* dst = cmap;
    if (epi == kEpiResidF32) {
      if (!encode_tmap_out_2d(&scratch, ws->qkv, true, M, w.out, w.out)) return cudaErrorInvalidValue;
      dst = &scratch;
    }
    cudaEvent_t ev[2];
    if ((rc = cudaEventCreate(&ev[0])) != cudaSuccess) return rc;
    if ((rc = cudaEventCreate(&ev[1])) != cudaSuccess) {
      cudaEventDestroy(ev[0]);
      return rc;
    }
    float best = 0.f;
    int best_bn = *bn;
    for (int cand : {128, 256, kTilePair | 128, kTilePair | 256}) {
      if ((cand & ~kTilePair) == 256 && w.out < 256) continue;
      for (int rep = 0; rep < 4 && rc == cudaSuccess; ++rep) {
        if (rep == 1) rc = cudaEventRecord(ev[0], st);
        if (rc == cudaSuccess) rc = launch(amap, w, epi, M, f8, cand, dst);
      }
      if (rc == cudaSuccess) rc = cudaEventRecord(ev[1], st);
      if (rc == cudaSuccess) rc = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (rc == cudaSuccess) rc = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (rc != cudaSuccess) break;
      if (best == 0.f || ms < best) {
        best = ms;
        best_bn = cand;
      }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != cudaSuccess) return rc;
    net->tuned_bn[key] = best_bn;
    ++((best_bn & ~kTilePair) == 256 ? net->tuned_shapes_256 : net->tuned_shapes_128);
    if (best_bn & kTilePair) ++net->tuned_shapes_pair;
    *bn = best_bn;
    return cudaSuccess;
  }



  struct Maps {
    const CUtensorMap *h, *att, *mlp, *qkv;  // operands / attention input
    const CUtensorMap *o_x, *o_qkv, *o_mlp;  // epilogue outputs
    const CUtensorMap* h8;                   // E4M3 LayerNorm output (FP8 precision)
  };

  // FP8 precision: is the layer of bit `bit` (see Net::fp8_mask) an E4M3 layer?
  bool fp8_layer(int bit) const { return net->precision == REVO_FP8 && ((net->fp8_mask >> bit) & 1); }

  // The LayerNorm of x's first M rows in the format of the Linear that reads it
  // (fp8 bit `bit`): E4M3 codes and per-token scales into h8 for an E4M3 layer,
  // else bf16 (float32 on the SIMT path) into h.
  cudaError_t layernorm(const float* x, const float* g, const float* bb, int d, int M, int bit) {
    ++launched;
    if (fp8_layer(bit)) return launch_layernorm_e4m3(x, g, bb, ws->h8, ws->h8_scale, M, d, st);
    return launch_layernorm(x, g, bb, ws->h, M, d, tc, st);
  }

  // The Linear that reads the LayerNorm output (qkv, fc1, enc2dec, head).
  cudaError_t from_ln(const LinearW& w, int epi, void* out, int ldo, int M, const Maps& mp, const CUtensorMap* cmap,
                      int bit) {
    if (fp8_layer(bit)) return linear8(mp.h8, w, epi, M, cmap);
    return linear(mp.h, ws->h, w, epi, out, ldo, M, cmap);
  }

  // A residual Linear x += A W^T + b (proj, fc2) followed by the LayerNorm
  // (g, bb) of x for the Linear of fp8 bit `bit`, as two launches.  (The
  // GEMM can also normalise each completed 128-row block in its epilogue,
  // kEpiResidLn; at these widths that LayerNorm runs on one SM per row block
  // with a few rows in flight and stalls the GEMM longer than the separate,
  // HBM-bound LayerNorm launch takes, so the forward does not use it.)
  cudaError_t resid_ln(const CUtensorMap* amap, const void* A, const LinearW& w, float* x, int d, int M,
                       const CUtensorMap* cmap, const float* g, const float* bb, int bit) {
    cudaError_t e = linear(amap, A, w, kEpiResidF32, x, d, M, cmap);
    return e != cudaSuccess ? e : layernorm(x, g, bb, d, M, bit);
  }

  // What follows a block's fc2: the next block's LN1 (fp8 bit of its qkv) or
  // the stack's final LayerNorm (bf16, read by a plain Linear).
  struct NextLn {
    const float *g, *b;
    int bit;
  };
  static constexpr int kNoFp8 = 30;  // an fp8 bit no layer has

  // One transformer block on rows [0, M) of x whose LN1 output is already in
  // h / h8; leaves `next`'s LayerNorm of the block's output there.
  cudaError_t block(const BlockW& b, int d, int heads, int M, const Segments& seg, const Maps& mp, bool dec,
                    const NextLn& next) {
    cudaError_t e;
    const int bit = dec ? 2 : 0;
    if ((e = from_ln(b.qkv, tc ? kEpiBf16 : kEpiF32, ws->qkv, 3 * d, M, mp, mp.o_qkv, bit)) != cudaSuccess) return e;
    if ((e = attention(d, heads, M, seg, mp)) != cudaSuccess) return e;
    if ((e = resid_ln(mp.att, ws->att, b.proj, ws->x, d, M, mp.o_x, b.ln2g, b.ln2b, bit + 1)) != cudaSuccess) return e;
    if ((e = from_ln(b.fc1, kEpiGeluBf16, ws->mlp, net->s.r * d, M, mp, mp.o_mlp, bit + 1)) != cudaSuccess) return e;
    return resid_ln(mp.mlp, ws->mlp, b.fc2, ws->x, d, M, mp.o_x, next.g, next.b, next.bit);
  }

  cudaError_t attention(int d, int heads, int M, const Segments& seg, const Maps& mp) {
    ++launched;
    if (!tc)
      return launch_attention_simt(static_cast<const float*>(ws->qkv), static_cast<float*>(ws->att), M, d, heads, seg,
                                   st);
    int nl = 1;
    cudaError_t e = launch_attention_tc(*mp.qkv, ws->att, M, d, heads, seg, ws->err, st, nullptr, ws->sms, &nl);
    launched += nl - 1;
    return e;
  }

  // The last decoder block on the rows that reach the pixel head (Section
  // 3.4.1: the output is the target frame, the last frame of the final
  // tubelet slot): qkv on every token (keys and values of the whole request;
  // LN1 is already in h / h8), attention with the final slot's queries only,
  // then those rows are stacked (runs.dst: their row in the head output) and
  // proj, LN2, fc1, fc2 run on them alone, leaving the final LayerNorm of the
  // stacked rows in h.  An exact saving: no other row reaches the head.
  cudaError_t last_block(const BlockW& b, int d, int heads, int M, const Segments& seg, const Maps& mp,
                         const RowRuns& runs, const Maps& cm) {
    cudaError_t e;
    if ((e = from_ln(b.qkv, tc ? kEpiBf16 : kEpiF32, ws->qkv, 3 * d, M, mp, mp.o_qkv, 2)) != cudaSuccess) return e;
    Segments q = seg;
    if (tc) {
      q.queries = true;
      for (int i = 0; i < seg.n; ++i) {
        q.q_begin[i] = runs.src[i];
        q.q_end[i] = runs.src[i] + (runs.dst[i + 1] - runs.dst[i]);
      }
    }
    if ((e = attention(d, heads, M, q, mp)) != cudaSuccess) return e;
    ++launched;
    if ((e = launch_gather_rows(ws->x, ws->att, static_cast<int>(this->e), d, runs, ws->xc, ws->attc, st)) !=
        cudaSuccess)
      return e;
    const int P = runs.dst[runs.n];
    if ((e = resid_ln(cm.att, ws->attc, b.proj, ws->xc, d, P, cm.o_x, b.ln2g, b.ln2b, 3)) != cudaSuccess) return e;
    if ((e = from_ln(b.fc1, kEpiGeluBf16, ws->mlp, net->s.r * d, P, cm, cm.o_mlp, 3)) != cudaSuccess) return e;
    return resid_ln(cm.mlp, ws->mlp, b.fc2, ws->xc, d, P, cm.o_x, net->dec_norm_g, net->dec_norm_b, kNoFp8);
  }
};

bool encode_maps(const NetShape& s, Workspace* ws, int M) {
  if (ws->maps_rows == M) return true;
  const uint64_t rows = M > 0 ? M : 1;
  bool ok = encode_tmap_bf16_2d(&ws->m_tok, ws->tok, rows, s.token_dim(), s.token_dim(), 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_h_enc, ws->h, rows, s.D, s.D, 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_att_enc, ws->att, rows, s.D, s.D, 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_mlp_enc, ws->mlp, rows, s.r * s.D, s.r * s.D, 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_h_dec, ws->h, rows, s.Dd, s.Dd, 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_att_dec, ws->att, rows, s.Dd, s.Dd, 128, 64) &&
            encode_tmap_bf16_2d(&ws->m_mlp_dec, ws->mlp, rows, s.r * s.Dd, s.r * s.Dd, 128, 64) &&
            encode_attention_tmap(&ws->m_qkv_enc, ws->qkv, static_cast<int>(rows), s.D) &&
            encode_attention_tmap(&ws->m_qkv_dec, ws->qkv, static_cast<int>(rows), s.Dd) &&
            encode_tmap_out_2d(&ws->o_x_enc, ws->x, true, rows, s.D, s.D) &&
            encode_tmap_out_2d(&ws->o_x_dec, ws->x, true, rows, s.Dd, s.Dd) &&
            encode_tmap_out_2d(&ws->o_qkv_enc, ws->qkv, false, rows, 3 * s.D, 3 * s.D) &&
            encode_tmap_out_2d(&ws->o_qkv_dec, ws->qkv, false, rows, 3 * s.Dd, 3 * s.Dd) &&
            encode_tmap_out_2d(&ws->o_mlp_enc, ws->mlp, false, rows, s.r * s.D, s.r * s.D) &&
            encode_tmap_out_2d(&ws->o_mlp_dec, ws->mlp, false, rows, s.r * s.Dd, s.r * s.Dd);
  if (ok && ws->h8)
    ok = encode_tmap_u8_2d(&ws->m_h8_enc, ws->h8, rows, s.D, s.D, 128) &&
         encode_tmap_u8_2d(&ws->m_h8_dec, ws->h8, rows, s.Dd, s.Dd, 128);
  ws->maps_rows = ok ? M : -1;
  return ok;
}

// Maps of the last decoder block's stacked rows (P of them) and the head output.
bool encode_compact_maps(const NetShape& s, Workspace* ws, int P) {
  if (ws->maps_rows_c == P) return true;
  const uint64_t rows = P > 0 ? P : 1;
  bool ok = encode_tmap_bf16_2d(&ws->c_h, ws->h, rows, s.Dd, s.Dd, 128, 64) &&
            encode_tmap_bf16_2d(&ws->c_att, ws->attc, rows, s.Dd, s.Dd, 128, 64) &&
            encode_tmap_bf16_2d(&ws->c_mlp, ws->mlp, rows, s.r * s.Dd, s.r * s.Dd, 128, 64) &&
            encode_tmap_out_2d(&ws->c_o_x, ws->xc, true, rows, s.Dd, s.Dd) &&
            encode_tmap_out_2d(&ws->c_o_mlp, ws->mlp, false, rows, s.r * s.Dd, s.r * s.Dd) &&
            encode_tmap_out_2d(&ws->c_o_head, ws->head, true, rows, s.head_dim_out(), s.head_dim_out());
  if (ok && ws->h8) ok = encode_tmap_u8_2d(&ws->c_h8, ws->h8, rows, s.Dd, s.Dd, 128);
  ws->maps_rows_c = ok ? P : -1;
  return ok;
}

}  // namespace

namespace {

// The position-embedding operands of the embedding GEMMs at width D.
EpiAux pe_aux(const Workspace* ws, const float* tab, const float* omega, int D) {
  EpiAux a{};
  a.pe_pos = ws->pe_pos;
  a.pe_tab = tab;
  a.pe_omega = omega;
  a.pe_rows = ws->pe_rows;
  a.pe_part = D / 3;
  return a;
}

// Token segments (one per request) and the patch total; false if a size is invalid.
bool batch_segments(const NetShape& s, const PlaneJob* jobs, int n, Segments* seg, int* patches) {
  seg->n = n;
  seg->start[0] = 0;
  *patches = 0;
  for (int i = 0; i < n; ++i) {
    if (jobs[i].H % s.p || jobs[i].W % s.p || jobs[i].H <= 0 || jobs[i].W <= 0) return false;
    seg->start[i + 1] = seg->start[i] + request_tokens(s, jobs[i].H, jobs[i].W);
    *patches += request_patches(s, jobs[i].H, jobs[i].W);
  }
  return true;
}

}  // namespace

cudaError_t prepare_job_args(const Net* net, const Workspace* ws, const PlaneJob* jobs, int n, JobArgs* args) {
  const NetShape& s = net->s;
  if (n <= 0) return cudaSuccess;
  if (n > kMaxSegments) return cudaErrorInvalidValue;
  Segments seg{};
  int patches = 0;
  if (!batch_segments(s, jobs, n, &seg, &patches)) return cudaErrorInvalidValue;
  const bool tc = net->precision != REVO_FP32;
  const size_t e = tc ? 2 : 4;
  uint8_t* tok = static_cast<uint8_t*>(ws->tok);
  int hoff = 0;
  for (int i = 0; i < n; ++i) {
    JobArgs& j = args[i];
    j = JobArgs{};
    AssembleArgs& a = j.assemble;
    for (int fidx = 0; fidx <= s.k; ++fidx) {
      a.frames[fidx] = jobs[i].frames[fidx];
      a.pitch[fidx] = jobs[i].pitch[fidx];
    }
    a.mu_sigma = jobs[i].mu_sigma;
    a.out = tok + static_cast<size_t>(seg.start[i]) * s.token_dim() * e;
    a.C = s.C;
    a.F = s.frames();
    a.T = s.T;
    a.p = s.p;
    a.H = jobs[i].H;
    a.W = jobs[i].W;
    a.out_bf16 = tc;
    if (tc) {
      // Token positions for the position embedding in the embedding GEMMs.
      a.pe_pos = ws->pe_pos + seg.start[i];
      for (int t = 0; t < 8; ++t) a.taus[t] = jobs[i].taus[t];
    }
    BlendArgs& bl = j.blend;
    bl.C = s.C;
    bl.p = s.p;
    bl.H = jobs[i].H;
    bl.W = jobs[i].W;
    bl.head = ws->head + static_cast<size_t>(hoff) * s.head_dim_out();
    bl.decoded = jobs[i].frames[s.k];
    bl.pitch = jobs[i].pitch[s.k];
    bl.mask = jobs[i].mask;
    bl.mask_pitch = jobs[i].mask_pitch;
    bl.mu_sigma = jobs[i].mu_sigma;
    bl.out = jobs[i].out;
    bl.out_pitch = jobs[i].out_pitch;
    bl.values = jobs[i].values;
    for (int t = 0; t < 8; ++t) j.taus[t] = jobs[i].taus[t];
    hoff += request_patches(s, jobs[i].H, jobs[i].W);
  }
  return cudaSuccess;
}

cudaError_t net_forward(Net* net, Workspace* ws, const PlaneJob* jobs, int n, cudaStream_t st, int num_sms,
                        int* launches, const JobArgs* dev_args) {
  const NetShape& s = net->s;
  if (launches) *launches = 0;
  if (n <= 0) return cudaSuccess;
  if (n > kMaxSegments) return cudaErrorInvalidValue;
  Fwd f{net, ws, st, num_sms, net->precision != REVO_FP32, net->precision != REVO_FP32 ? 2u : 4u};
  Segments seg{};
  int patches = 0;
  if (!batch_segments(s, jobs, n, &seg, &patches)) return cudaErrorInvalidValue;
  const int M = seg.start[n];
  if (M > ws->cap_tokens || patches > ws->cap_patches) return cudaErrorInvalidValue;
  if (f.tc && !encode_maps(s, ws, M)) return cudaErrorInvalidValue;
  std::vector<JobArgs> args(n);
  cudaError_t e = prepare_job_args(net, ws, jobs, n, args.data());
  if (e != cudaSuccess) return e;

  // Tubelet assembly + normalisation, tubelet embedding, embeddings.  With
  // a device argument table (graph replay) on the tensor-core path, p = 16,
  // T <= 2: one implicit-GEMM launch reads the frames directly (no token
  // matrix); otherwise the assemble kernel writes the tokens for the GEMM.
  const bool implicit_embed = f.tc && dev_args && s.p == 16 && s.T <= 2;
  if (implicit_embed) {
    EmbedParams ep{};
    ep.n = n;
    ep.C = s.C;
    ep.T = s.T;
    for (int i = 0; i <= n; ++i) ep.seg_start[i] = seg.start[i];
    for (int i = 0; i < n; ++i) {
      ep.hp[i] = jobs[i].H / s.p;
      ep.wp[i] = jobs[i].W / s.p;
    }
    ep.jobs = reinterpret_cast<const uint8_t*>(&dev_args[0].assemble);
    ep.stride = sizeof(JobArgs);
    ep.pe_pos = ws->pe_pos;
    const EpiAux pe = pe_aux(ws, ws->pe_enc, ws->pe_om_enc, s.D);
    const LinearW& w = net->patch;
    const int bn = w.out % 256 == 0 ? 256 : 128;
    ++f.launched;
    if ((e = launch_embed_tc(bn == 256 ? w.map256 : w.map128, ws->o_x_enc, bn, w.b, M, w.out, w.in, ws->err,
                             f.sms, st, pe, ep)) != cudaSuccess)
      return e;
  } else if (dev_args) {
    // One launch for the batch, each request's arguments from the device table.
    std::vector<AssembleArgs> aa(n);
    for (int i = 0; i < n; ++i) aa[i] = args[i].assemble;
    ++f.launched;
    if ((e = launch_assemble_batch(aa.data(), n, &dev_args[0].assemble, sizeof(JobArgs), st)) != cudaSuccess) return e;
  } else {
    for (int i = 0; i < n; ++i, ++f.launched)
      if ((e = launch_assemble(args[i].assemble, st)) != cudaSuccess) return e;
  }
  // Tubelet embedding + position embedding: on the tensor-core path the
  // embedding is added in the GEMM's epilogue (token positions from the
  // assemble kernel), else by a pass per request.
  if (implicit_embed) {
    // Done: the implicit GEMM above includes both.
  } else if (f.tc) {
    EpiAux pe = pe_aux(ws, ws->pe_enc, ws->pe_om_enc, s.D);
    pe.kperm = s.C == 3 && s.p == 16 ? 1 : 0;  // the implicit GEMM's K-block order: the same bits on both paths
    if ((e = f.linear(&ws->m_tok, ws->tok, net->patch, kEpiF32Pe, ws->x, s.D, M, &ws->o_x_enc, &pe)) != cudaSuccess)
      return e;
  } else {
    if ((e = f.linear(&ws->m_tok, ws->tok, net->patch, kEpiF32, ws->x, s.D, M, &ws->o_x_enc)) != cudaSuccess) return e;
    for (int i = 0; i < n; ++i, ++f.launched)
      if ((e = launch_add_pe(ws->x + static_cast<size_t>(seg.start[i]) * s.D, jobs[i].H / s.p, jobs[i].W / s.p,
                             s.slots(), args[i].taus, s.D, st, dev_args ? dev_args[i].taus : nullptr, ws->pe_enc,
                             ws->pe_rows)) != cudaSuccess)
        return e;
  }

  const Fwd::Maps enc_maps{&ws->m_h_enc, &ws->m_att_enc, &ws->m_mlp_enc, &ws->m_qkv_enc,
                           &ws->o_x_enc, &ws->o_qkv_enc, &ws->o_mlp_enc, &ws->m_h8_enc};
  const Fwd::Maps dec_maps{&ws->m_h_dec, &ws->m_att_dec, &ws->m_mlp_dec, &ws->m_qkv_dec,
                           &ws->o_x_dec, &ws->o_qkv_dec, &ws->o_mlp_dec, &ws->m_h8_dec};
  // Encoder: LN1 of the first block; every later LayerNorm (each block's LN2,
  // the next block's LN1, the encoder's final LN) follows the residual Linear
  // before it.
  if (s.L > 0) {
    if ((e = f.layernorm(ws->x, net->enc[0].ln1g, net->enc[0].ln1b, s.D, M, 0)) != cudaSuccess) return e;
  } else if ((e = f.layernorm(ws->x, net->enc_norm_g, net->enc_norm_b, s.D, M, Fwd::kNoFp8)) != cudaSuccess) {
    return e;
  }
  for (int i = 0; i < s.L; ++i) {
    const Fwd::NextLn next = i + 1 < s.L ? Fwd::NextLn{net->enc[i + 1].ln1g, net->enc[i + 1].ln1b, 0}
                                         : Fwd::NextLn{net->enc_norm_g, net->enc_norm_b, Fwd::kNoFp8};
    if ((e = f.block(net->enc[i], s.D, s.H, M, seg, enc_maps, false, next)) != cudaSuccess) return e;
  }
  // Encoder -> decoder Linear + the decoder's position embedding (the same way).
  if (f.tc) {
    const EpiAux pe = pe_aux(ws, ws->pe_dec, ws->pe_om_dec, s.Dd);
    if ((e = f.linear(&ws->m_h_enc, ws->h, net->enc2dec, kEpiF32Pe, ws->x, s.Dd, M, &ws->o_x_dec, &pe)) !=
        cudaSuccess)
      return e;
  } else {
    if ((e = f.linear(&ws->m_h_enc, ws->h, net->enc2dec, kEpiF32, ws->x, s.Dd, M, &ws->o_x_dec)) != cudaSuccess)
      return e;
    for (int i = 0; i < n; ++i, ++f.launched)
      if ((e = launch_add_pe(ws->x + static_cast<size_t>(seg.start[i]) * s.Dd, jobs[i].H / s.p, jobs[i].W / s.p,
                             s.slots(), args[i].taus, s.Dd, st, dev_args ? dev_args[i].taus : nullptr, ws->pe_dec,
                             ws->pe_rows)) != cudaSuccess)
        return e;
  }
  // The final slot's rows of each request, stacked in request order: the rows
  // the last decoder block, the final LN and the pixel head work on (the head
  // output is then in the order the blend reads it).
  RowRuns runs{};
  runs.n = n;
  runs.dst[0] = 0;
  for (int i = 0; i < n; ++i) {
    const int P = request_patches(s, jobs[i].H, jobs[i].W);
    runs.src[i] = seg.start[i] + (s.slots() - 1) * P;
    runs.dst[i + 1] = runs.dst[i] + P;
  }
  if (f.tc && !encode_compact_maps(s, ws, patches)) return cudaErrorInvalidValue;
  const Fwd::Maps last_maps{&ws->c_h, &ws->c_att, &ws->c_mlp, nullptr, &ws->c_o_x, nullptr, &ws->c_o_mlp, &ws->c_h8};
  // Decoder (check_shape: Ld >= 1), the same chaining; the last block leaves
  // the final LayerNorm of the stacked rows in h.
  if ((e = f.layernorm(ws->x, net->dec[0].ln1g, net->dec[0].ln1b, s.Dd, M, 2)) != cudaSuccess) return e;
  for (int i = 0; i + 1 < s.Ld; ++i) {
    const Fwd::NextLn next{net->dec[i + 1].ln1g, net->dec[i + 1].ln1b, 2};
    if ((e = f.block(net->dec[i], s.Dd, s.Hd, M, seg, dec_maps, true, next)) != cudaSuccess) return e;
  }
  if ((e = f.last_block(net->dec[s.Ld - 1], s.Dd, s.Hd, M, seg, dec_maps, runs, last_maps)) != cudaSuccess) return e;

  // Pixel head on the stacked rows, then the blend per request.
  if ((e = f.linear(&ws->c_h, ws->h, net->head, kEpiF32, ws->head, s.head_dim_out(), patches, &ws->c_o_head)) !=
      cudaSuccess)
    return e;
  if (dev_args) {
    std::vector<BlendArgs> bb(n);
    for (int i = 0; i < n; ++i) bb[i] = args[i].blend;
    ++f.launched;
    if ((e = launch_blend_batch(bb.data(), n, &dev_args[0].blend, sizeof(JobArgs), st)) != cudaSuccess) return e;
  } else {
    for (int i = 0; i < n; ++i, ++f.launched)
      if ((e = launch_blend(args[i].blend, st)) != cudaSuccess) return e;
  }
  if (launches) *launches = f.launched;
  return cudaSuccess;
}

cudaError_t net_autotune(Net* net, Workspace* ws, int max_tokens, int max_patches, cudaStream_t st, int num_sms) {
  const NetShape& s = net->s;
  if (net->precision == REVO_FP32) return cudaSuccess;
  Fwd f{net, ws, st, num_sms, true, 2u};
  f.tuning = true;
  cudaError_t e = cudaSuccess;
  int bn = 0;
  auto tune = [&](const CUtensorMap* amap, const LinearW& w, int epi, int M, const CUtensorMap* cmap, bool f8) {
    if (e == cudaSuccess) e = f.tuned_width(amap, w, epi, M, cmap, f8, &bn);
  };
  const bool f8q_e = net->precision == REVO_FP8 && (net->fp8_mask & 1);
  const bool f8f_e = net->precision == REVO_FP8 && (net->fp8_mask & 2);
  const bool f8q_d = net->precision == REVO_FP8 && (net->fp8_mask & 4);
  const bool f8f_d = net->precision == REVO_FP8 && (net->fp8_mask & 8);
  // Rows of every token: the tubelet embedding, the blocks (all alike within
  // the encoder and within the decoder) and the encoder->decoder Linear.
  for (int b = 128; e == cudaSuccess; b = next_tune_bucket(b)) {
    const int M = std::min(b, max_tokens);
    if (!encode_maps(s, ws, M)) return cudaErrorInvalidValue;
    tune(&ws->m_tok, net->patch, kEpiF32, M, &ws->o_x_enc, false);
    if (s.L > 0) {
      const BlockW& k = net->enc[0];
      tune(f8q_e ? &ws->m_h8_enc : &ws->m_h_enc, k.qkv, kEpiBf16, M, &ws->o_qkv_enc, f8q_e);
      tune(&ws->m_att_enc, k.proj, kEpiResidF32, M, &ws->o_x_enc, false);
      tune(f8f_e ? &ws->m_h8_enc : &ws->m_h_enc, k.fc1, kEpiGeluBf16, M, &ws->o_mlp_enc, f8f_e);
      tune(&ws->m_mlp_enc, k.fc2, kEpiResidF32, M, &ws->o_x_enc, false);
    }
    tune(&ws->m_h_enc, net->enc2dec, kEpiF32, M, &ws->o_x_dec, false);
    const BlockW& d = net->dec[0];
    tune(f8q_d ? &ws->m_h8_dec : &ws->m_h_dec, d.qkv, kEpiBf16, M, &ws->o_qkv_dec, f8q_d);
    tune(&ws->m_att_dec, d.proj, kEpiResidF32, M, &ws->o_x_dec, false);
    tune(f8f_d ? &ws->m_h8_dec : &ws->m_h_dec, d.fc1, kEpiGeluBf16, M, &ws->o_mlp_dec, f8f_d);
    tune(&ws->m_mlp_dec, d.fc2, kEpiResidF32, M, &ws->o_x_dec, false);
    if (M >= max_tokens) break;
  }
  // The final slot's rows: the pixel head (the last block's other shapes are
  // the decoder's, timed above for these row counts).
  for (int b = 128; e == cudaSuccess; b = next_tune_bucket(b)) {
    const int M = std::min(b, max_patches);
    if (!encode_compact_maps(s, ws, M)) return cudaErrorInvalidValue;
    tune(&ws->c_h, net->head, kEpiF32, M, &ws->c_o_head, false);
    if (M >= max_patches) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace revo
