/*
 * revo.h -- C ABI of the B300 (sm_103a) neural loss-recovery library.
 *
 * The library recovers the lost pixels of decoded RGB (uint8) and depth
 * (uint16 mm) video frames, the post-decode recovery step of ReVo's receiver
 * (Section 3.4, the neural loss-recovery module): a ViViT encoder-decoder reads
 * the k closest clean frames and the corrupted current frame and outputs a
 * reconstructed frame (Section 3.4.1); RGB and depth use separate models of the
 * same architecture (Section 3.4.2) and run on independent CUDA streams
 * (Section 3.1, Challenge 2).  Intact and corrupted pixels are fed alike
 * (Appendix B.1, point 3); tokens are tubelets of T frames x p x p pixels
 * (Appendix B.3).  The per-pixel loss mask does not enter the network: it
 * selects, per pixel, the decoded value (received) or the recovered value
 * (lost), so received pixels pass through bit for bit.
 *
 * Conventions for every call:
 *  - Nothing throws across this boundary; every call returns a revo_status.
 *  - Pointers are plain host or device pointers as each argument states.
 *  - Frames: RGB uint8 interleaved [H][W][3] with a row pitch in bytes; depth
 *    uint16 millimetres [H][W] with a row pitch in bytes, 0 = no depth.
 *  - Loss mask: 1 bit per pixel, 1 = lost, row-major, bit (x % 32) of 32-bit
 *    word (x / 32), with a row pitch in words (at least ceil(W / 32)).
 *  - H and W must be multiples of the patch size p.
 *  - A revo_ctx is used by one host thread at a time.
 */
#ifndef REVO_H
#define REVO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define REVO_API __attribute__((visibility("default")))
#else
#define REVO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  REVO_OK = 0,
  REVO_EAGAIN = 1,      /* not finished yet, or no capacity right now          */
  REVO_EINVAL = -1,     /* bad argument: null pointer, bad size, bad shape      */
  REVO_ENOMEM = -2,     /* device memory or the HBM budget cannot hold it       */
  REVO_ETIMEDOUT = -3,  /* poll timed out, or a device-side wait gave up        */
  REVO_ENOREF = -4,     /* the stream holds fewer than k clean reference frames */
  REVO_ECUDA = -5,      /* a CUDA call failed (the message is in revo_last_error) */
  REVO_ENOTSUP = -6     /* the device or the configuration is not supported     */
} revo_status;

typedef enum { REVO_FP32 = 0, REVO_BF16 = 1, REVO_FP8 = 2 } revo_precision;

/* Request flags. */
#define REVO_RGB 1u     /* the request carries an RGB plane                   */
#define REVO_DEPTH 2u   /* the request carries a depth plane                  */
#define REVO_CLEAN 4u   /* intact frame: push it into the stream's reference
                           history and run nothing (Section 3.1.1 forwards intact
                           frames directly; the paper reuses clean references
                           across a GoP, Section 3.4.1)                         */
#define REVO_HOLD 8u    /* admit the request to the pending batch without
                           launching: the batch starts on the submit that fills
                           max_batch, on a submit without this flag, or on
                           flush / a waiting poll (no counterpart in the paper:
                           a serving control)                                   */

/*
 * Network shape and runtime limits.  revo_config_default() fills the ViT-B
 * reading: k = 5 references, tubelet T = 2, patch p = 16, encoder 768 wide x 12
 * blocks x 12 heads, decoder 384 wide x 4 blocks x 6 heads, MLP ratio 4.
 * Requirements: (k + 1) % T == 0, k <= 7; head width (dim / heads) == 64;
 * dims multiples of 64; p == 16.
 *
 * Weights are flat little-endian float32 arrays in this order (Linear weights
 * [out][in]; the tubelet embedding is a Linear over a tubelet flattened as
 * (t, c, y, x); the head's outputs are ordered (t, c, y, x) too):
 *   patch_embed.w [D][T*C*p*p], patch_embed.b [D],
 *   per encoder block: ln1.g [D], ln1.b [D], qkv.w [3D][D], qkv.b [3D],
 *     proj.w [D][D], proj.b [D], ln2.g [D], ln2.b [D], fc1.w [rD][D],
 *     fc1.b [rD], fc2.w [D][rD], fc2.b [D]   (qkv rows: q | k | v),
 *   enc_norm.g [D], enc_norm.b [D], enc2dec.w [D'][D], enc2dec.b [D'],
 *   per decoder block: the same at width D',
 *   dec_norm.g [D'], dec_norm.b [D'], head.w [T*C*p*p][D'], head.b [T*C*p*p].
 * The weights are copied at create; the caller keeps ownership of its arrays.
 */
typedef struct {
  int k, tubelet, patch;
  int enc_dim, enc_depth, enc_heads;
  int dec_dim, dec_depth, dec_heads;
  int mlp_ratio;
  revo_precision precision;
  int device;                    /* CUDA device ordinal                         */
  size_t hbm_budget_bytes;       /* cap on the context's device memory; 0 = 40 GB */
  int max_streams;               /* conference streams with a reference history */
  int max_height, max_width;     /* largest frame any stream will submit        */
  int max_batch;                 /* requests fused into one launch (>= 1)        */
  int lanes;                     /* batches in flight at once (>= 1)             */
  void* cuda_stream;             /* cudaStream_t for the work, NULL = own streams */
  int use_graphs;                /* 1 = replay captured CUDA graphs per batch shape */
  int autotune;                  /* 1 = time the GEMM tile widths per shape on first
                                    use and keep the fastest (tensor-core path)  */
  int fp8_layers;                /* REVO_FP8: which LayerNorm-fed layers run in E4M3,
                                    bits 0-3 for the RGB model, bits 4-7 for the
                                    depth model (per model: bit 0 encoder qkv, 1
                                    encoder fc1, 2 decoder qkv, 3 decoder fc1; the
                                    rest stay bf16); 0 = the default: all four in
                                    the RGB model, none in the depth model (its
                                    8 mm gate fails with E4M3 at 300-5000 mm) */
  const float* rgb_weights;      /* host, flat float32, NULL = see below         */
  size_t rgb_weights_count;
  const float* depth_weights;    /* host, flat float32, NULL = see below         */
  size_t depth_weights_count;
  /* A model whose array is NULL is read from its file (flat little-endian
   * float32 in the order above, exactly the model's parameter count), else,
   * if its bit of random_init is set, gets the random initialisation of
   * revo_init_weights from seed (RGB) or seed + 1 (depth), else is absent. */
  const char* rgb_weights_path;
  const char* depth_weights_path;
  uint64_t seed;
  int random_init;               /* bit 0 RGB, bit 1 depth                        */
  /* Tile choices of the autotuner: with autotune on, create reads this file
   * (entries of another GPU model or SM count are ignored), times every GEMM
   * shape it lacks, and writes the file back; NULL = time them all at create.
   * Requests never wait for tuning. */
  const char* autotune_cache;
  /* 1 = a batch's RGB forward runs before its depth forward instead of beside
   * it on a second CUDA stream (the results are the same).  Two large
   * forwards side by side split the SMs between persistent GEMM kernels and
   * their caches; one after the other each has the GPU to itself. */
  int serial_models;
} revo_config;

typedef struct revo_ctx revo_ctx;

/* One image plane: RGB uint8 [H][W][3] or depth uint16 [H][W]. */
typedef struct {
  const void* data;
  int height, width;
  size_t pitch_bytes;
} revo_plane;

/*
 * One frame of one conference stream (the problem statement of Section 3.4.1:
 * frame, loss mask and reference frames in, recovered frame out).
 *  - stream_id < max_streams; frame_index increases along the stream.  The
 *    temporal distances the network embeds are frame_index minus the indices
 *    of the stream's clean references.
 *  - flags: REVO_RGB and/or REVO_DEPTH, plus REVO_CLEAN for an intact frame.
 *  - inputs_on_device: 1 = data/mask pointers are device pointers and must stay
 *    valid until the request completes; 0 = host pointers, copied during submit.
 *  - outputs: rgb_out (uint8 [H][W][3], pitch rgb_out_pitch) and depth_out
 *    (uint16 [H][W], pitch depth_out_pitch) receive the blended frame; the
 *    optional *_values (float32 [H][W][3] in [0,1] units / float32 [H][W] in mm,
 *    dense) receive the de-normalised network output at every pixel before the
 *    blend.  outputs_on_device says whether these are device or host pointers;
 *    they are borrowed until poll returns REVO_OK for the ticket.
 */
typedef struct {
  uint32_t stream_id;
  int64_t frame_index;
  uint32_t flags;
  int inputs_on_device;
  revo_plane rgb;
  const uint32_t* rgb_lost_mask;
  size_t rgb_mask_pitch_words;
  revo_plane depth;
  const uint32_t* depth_lost_mask;
  size_t depth_mask_pitch_words;
  int outputs_on_device;
  void* rgb_out;
  size_t rgb_out_pitch;
  void* depth_out;
  size_t depth_out_pitch;
  float* rgb_values;
  float* depth_values;
} revo_request;

typedef struct {
  revo_status status;
  uint32_t stream_id;
  int64_t frame_index;
  double latency_ms;   /* host clock, submit -> completion observed            */
  double device_ms;    /* CUDA-event time of the batch that carried the request */
  int batch_size;      /* requests in that batch                                */
  int kernel_launches; /* CUDA kernels the batch launched (both modalities)     */
} revo_result;

/* Fills *cfg with the ViT-B reading above and precision BF16. */
REVO_API void revo_config_default(revo_config* cfg);

/*
 * The random initialisation (no trained weights exist for the paper's model):
 * fills out[0 .. count) with the float32 weights of the model of `channels`
 * (3 RGB, 1 depth) shaped by cfg, in the order above, drawn from one stream of
 * uniform doubles u = (x >> 11) 2^-53 of the PCG64 generator (128-bit LCG,
 * multiplier 0x2360ED051FC65DA44385DF649FCCF645, XSL-RR output) seeded through
 * the SeedSequence mixing of NumPy's random module: [out][in] matrices
 * U(-b, b), b = sqrt(6 / (in + out)), the pixel head times 0.1; LayerNorm
 * gains 1 + U(-0.1, 0.1); every other vector U(-0.02, 0.02); each value in
 * double, rounded to float32.  Host only (no device work).
 * Errors: REVO_EINVAL (null pointer, unsupported shape, count differs from
 * the model's parameter count).
 */
REVO_API revo_status revo_init_weights(const revo_config* cfg, int channels, uint64_t seed, float* out, size_t count);

/*
 * Creates a context on cfg->device: uploads both models' weights (float32
 * master copies and the precision's tensor-core copies), allocates the
 * reference histories and the work arenas within hbm_budget_bytes.
 * Errors: REVO_EINVAL (shape rules above, weight count mismatch, null out),
 * REVO_ENOTSUP (the tensor-core path needs an sm_100-class device),
 * REVO_ENOMEM (budget or device memory), REVO_ECUDA.  On error *out is NULL.
 */
REVO_API revo_status revo_recover_create(const revo_config* cfg, revo_ctx** out);

/*
 * Submits one request and returns a ticket.  REVO_CLEAN requests are queued on
 * the device at once (the frame enters the stream's history).  Other requests
 * join the pending batch; a batch is launched when max_batch requests are
 * pending, when a lane has room (at most one batch running on it: the new one
 * queues behind it on the device) and requests are waiting, on flush, or on a
 * poll that waits (timeout_us != 0) for one of them.
 * Host inputs are copied before return.
 * Errors: REVO_EINVAL (bad ids, flags, shapes, pointers), REVO_ENOREF (fewer
 * than k clean frames in the stream's history for a requested modality),
 * REVO_EAGAIN (pending queue full: poll and retry), REVO_ECUDA.
 */
REVO_API revo_status revo_recover_submit(revo_ctx* ctx, const revo_request* req, uint64_t* ticket);

/* Launches every pending request now (in batches of at most max_batch). */
REVO_API revo_status revo_recover_flush(revo_ctx* ctx);

/*
 * Waits up to timeout_us microseconds (0 = do not wait, < 0 = forever) for a
 * ticket.  REVO_OK: finished, *out filled, outputs written, the ticket is
 * retired.  REVO_EAGAIN: still running or still pending (timeout 0; a pending
 * request is then left to be batched with later arrivals).  REVO_ETIMEDOUT: the wait
 * ran out.  REVO_EINVAL: unknown ticket.  A device-side failure of the batch is
 * reported in out->status.
 */
REVO_API revo_status revo_recover_poll(revo_ctx* ctx, uint64_t ticket, int64_t timeout_us, revo_result* out);

/* Counters of a context (for serving dashboards and tests). */
typedef struct {
  size_t device_bytes;      /* device memory the context holds                     */
  uint64_t batches;         /* forward batches launched                            */
  uint64_t graph_replays;   /* of those modality forwards, replays of a captured graph */
  int graphs_captured;      /* captured forwards held (all lanes, both modalities) */
  int tuned_shapes;         /* GEMM shapes the autotuner has timed                 */
  int tuned_wide;           /* of those, shapes where a 256-wide tile won          */
  int pending;              /* submitted requests not yet in a batch               */
  int in_flight;            /* batches launched and not yet retired                */
  int tuned_pair;           /* tuned shapes where a CTA-pair tile (REVO_TILE_PAIR) won */
  int tuned_timed;          /* of the tuned shapes, those this context timed (the rest
                               came from the autotune cache file)                  */
} revo_stats;

/* Fills *out.  Errors: REVO_EINVAL (null argument). */
REVO_API revo_status revo_recover_stats(revo_ctx* ctx, revo_stats* out);

/* Drains the work in flight, then frees everything the context owns. */
REVO_API void revo_recover_destroy(revo_ctx* ctx);

/* The last error message of the calling thread ("" if none). */
REVO_API const char* revo_last_error(void);

/* ------------------------------------------------------------------------ *
 * Step-level entry points.  Each runs one stage of the recovery forward on
 * caller-owned device buffers, on the given stream (cudaStream_t, NULL = the
 * default stream), asynchronously.  They exist so that each stage can be
 * checked on its own; the context above chains the same kernels.  All return
 * REVO_EINVAL for null pointers or sizes outside the stated limits and
 * REVO_ECUDA if the launch fails.  Row-major everywhere.
 * ------------------------------------------------------------------------ */

/*
 * Tubelet assembly (Appendix B.3) fused with input normalisation: for one
 * request, writes the token matrix A [S*Hp*Wp][T*C*p*p] (token order slot,
 * patch row, patch column; vector order t, c, y, x) from the k reference
 * frames (host array `refs` of k device pointers, oldest first) and the
 * decoded current frame, all in the plane format above with one pitch.  RGB
 * (C = 3): (x/255 - mean_c)/std_c with the ImageNet statistics.  Depth (C = 1):
 * (d - mu)/sigma with mu_sigma[2] a device float pair.  out_bf16 != 0 writes
 * bf16, else float32.  k <= 7, p <= 16.
 */
REVO_API revo_status revo_op_assemble(int channels, int k, int T, int p, int height, int width,
                             const void* const* refs, const void* current, size_t pitch_bytes,
                             const float* mu_sigma, void* out, int out_bf16, void* stream);

/*
 * Depth statistics of one uint16 frame: mean and biased standard deviation of
 * the non-zero pixels, written as float32 to mu_sigma[0..1] (device).  No valid
 * pixel gives (0, 1); the deviation is floored at 1 mm.  scratch is a device
 * buffer of revo_depth_stats_scratch_bytes() bytes, 8-byte aligned, that only
 * one call at a time may use.  Frames up to 2^24 pixels (height * width), so
 * that the pixel count is exact in float32 where it divides the sum; larger
 * frames and a misaligned scratch return REVO_EINVAL.
 */
REVO_API size_t revo_depth_stats_scratch_bytes(void);
REVO_API revo_status revo_op_depth_stats(const uint16_t* depth, int height, int width, size_t pitch_bytes,
                                float* mu_sigma, void* scratch, void* stream);

/*
 * The same depth statistics for callers that cannot allocate device memory:
 * for example a receiver loop that must not call cudaMalloc while frames are in
 * flight (it can synchronise the device and stall other streams past the frame
 * deadline), or a host application whose device memory is all reserved up
 * front by its own pool.  The paper has no counterpart; this is a library
 * convenience.  It allocates nothing: the scratch is a fixed 8 KB array inside
 * the library, held by every GPU that loads the library until the process
 * exits.  The caller still passes the frame and the output pair.
 *  - Frames up to 2^24 pixels (height * width), the same limit as
 *    revo_op_depth_stats (the pixel count stays exact in float32); larger
 *    frames return REVO_EINVAL with a message.
 *  - The first call on a device looks up the array's device address (with that
 *    device current) and keeps it for that device's current CUDA context; a
 *    call in another context (after cudaDeviceReset, or under a context the
 *    caller made current) looks it up again.  Make the first call on a device,
 *    and the first after such a context change, before any CUDA stream
 *    capture.
 *  - Every call shares the one array.  Calls whose work overlaps on the GPU
 *    (other streams, other host threads) race on it and give wrong results;
 *    order them on one stream or serialise them.  Each call clears the
 *    counters it needs at the start, so leftovers of an earlier call do not
 *    matter.
 */
REVO_API revo_status revo_op_depth_stats_noalloc(const uint16_t* depth, int height, int width,
                                                 size_t pitch_bytes, float* mu_sigma, void* stream);

/*
 * Tile choice for the tensor-core Linear entry points: the tile width (128,
 * 192 or 256 output columns; 192 for float32 outputs on single tiles only),
 * optionally ORed with REVO_TILE_PAIR for 256-row tiles
 * computed by a pair of CTAs on two SMs (one tcgen05 MMA with .cta_group::2
 * over both SMs' shared memory and TMEM).  Results are the same for every
 * choice (each output is one float32 dot product in the same K order).
 */
#define REVO_TILE_PAIR 0x1000

/*
 * Y = epilogue(A W^T + b) with A [M][K], W [N][K] (Linear [out][in]), b [N]
 * (b may be NULL).
 *   precision REVO_FP32: A, W float32, SIMT FMA (K % 8 == 0).  REVO_BF16: A, W
 *   bf16 on the tcgen05 tensor cores with float32 accumulation (K % 64 == 0,
 *   N % 32 == 0, N % 64 == 0 for the bf16 epilogues 1 and 2); `tile_n` picks
 *   the 128-, 192- (epilogues 0 and 3, without REVO_TILE_PAIR) or 256-column
 *   tile (other widths: 128), | REVO_TILE_PAIR for the CTA-pair tiles.
 *   epilogue 0: out = acc + b (float32 out)
 *   epilogue 1: out = acc + b (bf16 out; FP32 precision writes float32)
 *   epilogue 2: out = gelu(acc + b) (bf16 out; FP32 precision writes float32)
 *   epilogue 3: out += acc + b (float32 residual, in place)
 */
REVO_API revo_status revo_op_linear(revo_precision precision, int epilogue, const void* A, const void* W,
                           const float* bias, void* out, int M, int N, int K, int tile_n, void* stream);

/*
 * The tubelet (or encoder -> decoder) Linear with the position embedding
 * added in its epilogue, in one launch (Section 3.4.1: token embedding plus
 * the sinusoidal embedding of temporal distance, patch row and patch column):
 *   out[m][n] = (sum_k A[m][k] W[n][k] + bias[n]) + pe(m)[n]
 * for the M = slots * grid_h * grid_w tokens of one request (token m is slot
 * m / (grid_h grid_w), patch row and column from m % (grid_h grid_w), as in
 * revo_op_add_position, whose values pe(m) are; the result equals
 * revo_op_linear(REVO_BF16, epilogue 0) followed by revo_op_add_position, bit
 * for bit).  A [M][K], W [N][K] bf16, bias [N] (may be NULL), out float32
 * [M][N], device; taus host [slots].  N a multiple of 192 up to 1024, K % 64
 * == 0, slots <= 8; tile_n as for revo_op_linear (192 on single tiles).  Uses
 * a per-device scratch of token positions (one call at a time per device).
 * Errors: REVO_EINVAL, REVO_ECUDA.
 */
REVO_API revo_status revo_op_linear_pe(const void* A, const void* W, const float* bias, float* out, int slots,
                                       int grid_h, int grid_w, int N, int K, const int* taus, int tile_n,
                                       void* stream);

/*
 * A residual Linear with the LayerNorm that follows it, in one launch (the
 * transformer block's "x = x + proj(att); h = LN2(x)" and
 * "x = x + fc2(mlp); h = LN1'(x)" steps, Section 3.4.1):
 *   x[m][n] += sum_k A[m][k] W[n][k] + bias[n]        (float32, in place)
 *   ln_out[m] = LayerNorm(x[m]; gamma, beta), eps 1e-6
 * A [M][K] and W [N][K] bf16 (tensor cores, float32 accumulation), x float32
 * [M][N], gamma / beta float32 [N], all device.  ln_fp8 == 0: ln_out bf16
 * [M][N]; ln_fp8 != 0: ln_out E4M3 codes [M][N] with ln_row_scale [M], the
 * per-row rule of revo_op_layernorm_e4m3.  The LayerNorm of a block of 128
 * rows runs in the GEMM epilogue of the CTA that adds the block's last column
 * tile; its values equal revo_op_layernorm (revo_op_layernorm_e4m3) applied
 * to the updated x, bit for bit.  K % 64 == 0, N % 32 == 0, N <= 1024; tile_n
 * 128 or 256, | REVO_TILE_PAIR.  Uses a per-device scratch of row-block
 * counters (one call at a time per device).  Errors: REVO_EINVAL, REVO_ECUDA.
 * Speed: one SM normalises each 128-row block with a few rows in flight, so
 * at the model's widths (768, 384) this is slower than revo_op_linear then
 * revo_op_layernorm, and the recovery forward uses those two.
 */
REVO_API revo_status revo_op_linear_resid_ln(const void* A, const void* W, const float* bias, float* x, int M, int N,
                                             int K, const float* gamma, const float* beta, void* ln_out,
                                             float* ln_row_scale, int ln_fp8, int tile_n, void* stream);

/* Row-wise LayerNorm, eps 1e-6: x float32 [M][D] -> out (bf16 if out_bf16, else float32). */
REVO_API revo_status revo_op_layernorm(const float* x, const float* gamma, const float* beta, void* out,
                              int M, int D, int out_bf16, void* stream);

/*
 * FP8 building blocks (no counterpart in the paper, which runs its model in
 * full precision; this is the reduced-precision path of the linear layers).
 * Codes are OCP FP8 E4M3 (bias 7, largest finite 448, no infinities).
 *
 * revo_op_quantize_rows_e4m3: per-row scale[r] = max_k |x[r][k]| / 448 (1 for
 * an all-zero row) and codes q[r][k] = E4M3(x[r][k] * (448 / max)), rounded to
 * nearest even and saturated to +-448; the product is taken in float32.  x is
 * float32 [rows][cols], cols % 4 == 0; q is [rows][cols] bytes; all device.
 * The weights use it with one row per output channel.
 *
 * revo_op_layernorm_e4m3: revo_op_layernorm (float32 result), then the same
 * per-row quantisation: out [M][D] codes, row_scale [M].
 *
 * revo_op_linear_fp8: out = epilogue(a_scale[m] * w_scale[n] * sum_k A[m][k] W[n][k]
 * + bias[n]) with A [M][K] and W [N][K] E4M3 codes (decoded exactly), the sum
 * accumulated in float32 on the tensor cores.  epilogue 1 (bf16 out) or 2
 * (GELU, bf16 out); out bf16 [M][N].  K % 128 == 0, N % 64 == 0; tile_n 128
 * or 256, | REVO_TILE_PAIR for CTA-pair tiles.  Errors: REVO_EINVAL, REVO_ECUDA.
 */
REVO_API revo_status revo_op_quantize_rows_e4m3(const float* x, int rows, int cols, uint8_t* q, float* scale,
                                                void* stream);
REVO_API revo_status revo_op_layernorm_e4m3(const float* x, const float* gamma, const float* beta, uint8_t* out,
                                            float* row_scale, int M, int D, void* stream);
REVO_API revo_status revo_op_linear_fp8(int epilogue, const uint8_t* A, const float* a_scale, const uint8_t* W,
                                        const float* w_scale, const float* bias, void* out, int M, int N, int K,
                                        int tile_n, void* stream);

/*
 * Reed-Solomon erasure coding of I-frame packets (Section 3.2: an I-frame is
 * cut into n data packets, r parity packets are added (the paper: r = n/2),
 * and any n of the n + r packets rebuild the frame).  The paper fixes no
 * matrix; this is a systematic code over GF(2^8) with field polynomial
 * x^8 + x^4 + x^3 + x^2 + 1 whose parity packet i is, byte by byte,
 * sum_j data[j] / ((n + i) + j) (Cauchy rows; + is XOR in the field).
 * Packets are device buffers of packet_bytes bytes (a multiple of 4; pad the
 * last one), rows `pitch` bytes apart (multiples of 4); 1 <= n, n + r <= 256.
 *
 * revo_fec_encode: data [n] -> parity [r].
 * revo_fec_decode: received [n] = the packets with indices present[0..n-1]
 *   (host array; data packets are 0..n-1, parity packets n..n+r-1), in that
 *   order -> data_out [n].  Arrived data packets are copied, missing ones
 *   rebuilt; the inverse is computed on the host (O(n^3) field operations).
 *   scratch: device memory of revo_fec_decode_scratch_bytes(n) bytes (needed
 *   when a data packet is missing), owned by the caller.
 * Errors: REVO_EINVAL (shape, pointers, repeated or out-of-range indices),
 * REVO_ECUDA.
 */
REVO_API revo_status revo_fec_encode(int n, int r, size_t packet_bytes, const uint8_t* data, size_t data_pitch,
                                     uint8_t* parity, size_t parity_pitch, void* stream);
REVO_API size_t revo_fec_decode_scratch_bytes(int n);
REVO_API revo_status revo_fec_decode(int n, int r, size_t packet_bytes, const int* present, const uint8_t* received,
                                     size_t received_pitch, uint8_t* data_out, size_t out_pitch, void* scratch,
                                     void* stream);

/*
 * RGB-D rendering: unprojection + point splatting of a (recovered) RGB-D
 * frame into the viewer's camera (the receiver's rendering step; RGB-D frames
 * are 2-D projections of the scene, Section 2).  The paper fixes no camera
 * model; this is a pinhole model: intrinsics {fx, fy, cx, cy}, pixel (i, j) at
 * u = i, v = j; a depth sample d (mm, 0 = none) is the point ((u - cx) d / fx,
 * (v - cy) d / fy, d); the pose maps it to x' = R x + t (R row-major, t in
 * mm); it lands on pixel (round(fx' x'/z' + cx'), round(fy' y'/z' + cy')) of the
 * target (round half to even; z' <= 0 dropped) and covers the
 * (2 splat_radius + 1)^2 pixels around it; per pixel the nearest z' wins (ties:
 * the lower row-major depth index).  Output: out_rgb uint8 [out_h][out_w][3]
 * (the winner's colour: RGB pixel (i rgb_w / w, j rgb_h / h), nearest sample),
 * out_depth uint16 [out_h][out_w] (z' rounded half to even, clamped); empty
 * pixels 0.  Every float step is separately rounded in a fixed order, so the
 * result is reproducible bit for bit.  All buffers device; pitches in bytes.
 * scratch: revo_render_scratch_bytes(out_h, out_w) bytes of device memory (the
 * 64-bit z-buffer), owned by the caller.  splat_radius 0..16.
 * Errors: REVO_EINVAL, REVO_ECUDA.
 */
typedef struct {
  float fx, fy, cx, cy;
} revo_intrinsics;

typedef struct {
  float r[9]; /* row-major rotation */
  float t[3]; /* translation, mm */
} revo_pose;

REVO_API size_t revo_render_scratch_bytes(int out_h, int out_w);
REVO_API revo_status revo_render_rgbd(const uint8_t* rgb, int rgb_h, int rgb_w, size_t rgb_pitch,
                                      const uint16_t* depth, int h, int w, size_t depth_pitch,
                                      const revo_intrinsics* src, const revo_pose* pose, const revo_intrinsics* dst,
                                      int out_h, int out_w, int splat_radius, void* scratch, uint8_t* out_rgb,
                                      size_t out_rgb_pitch, uint16_t* out_depth, size_t out_depth_pitch,
                                      void* stream);

/*
 * Frame-quality metrics of the paper's evaluation (Section 5, Metrics: SSIM
 * and PSNR of a reconstructed frame against the original).  a, b: device
 * frames of height x width samples, `channels` (1 or 3) interleaved,
 * `sample_bytes` 1 (uint8) or 2 (uint16), row pitches in bytes.  data_range =
 * L (255 for 8-bit RGB; the caller's choice for depth, e.g. 65535).  SSIM:
 * normalised 11 x 11 Gaussian window (sigma 1.5), C1 = (0.01 L)^2,
 * C2 = (0.03 L)^2, mean over the positions where the window lies inside the
 * frame, channels averaged (the paper cites SSIM without parameters; this is
 * the original definition).  PSNR = 10 log10(L^2 / MSE) over every sample.
 * out (device, 3 floats): mean SSIM, MSE, PSNR in dB (inf for equal frames).
 * scratch: device memory of revo_frame_metrics_scratch_bytes() bytes, owned by
 * the caller (no two calls in flight may share it).  Frames must be larger
 * than 10 x 10.  Deterministic (fixed-order reductions).
 * Errors: REVO_EINVAL, REVO_ECUDA.
 */
REVO_API size_t revo_frame_metrics_scratch_bytes(int height, int width, int channels);
REVO_API revo_status revo_op_frame_metrics(const void* a, size_t pitch_a, const void* b, size_t pitch_b, int height,
                                           int width, int channels, int sample_bytes, float data_range,
                                           void* scratch, float* out, void* stream);

/*
 * Multi-head softmax attention over segments of tokens (the exact scaled
 * dot-product attention of Appendix B.1, point 4).  qkv is [M][3D] (q | k | v,
 * head h owns columns h*64 .. h*64+63 of each part); seg_start[n_seg + 1] is a
 * host array of segment boundaries in [0, M]; tokens attend only within their
 * segment.  out [M][D].  REVO_FP32: float32 in and out.  REVO_BF16: qkv and out
 * bf16, tcgen05 tensor cores, float32 softmax.  n_seg <= 64.
 * q_begin / q_end (host arrays of n_seg, or both NULL): only rows
 * [q_begin[g], q_end[g]) of segment g are queries -- keys and values are still
 * the whole segment -- and, at REVO_BF16, only those output rows are written
 * (REVO_FP32 writes every row).  The recovery network uses it for its last
 * decoder block, whose only consumer is the pixel head on the final slot.
 * REVO_BF16 work split: one CTA per (head, 256-query) unit, one launch.
 * flags bit 0 (REVO_ATTN_SPLIT_TAIL): a segment's whole waves of units (the
 * GPU's SM count each) stay one CTA per unit, and the units of its last,
 * partly filled wave are cut into up to 8 key ranges so that wave fills the
 * SMs; a second kernel merges their parts.  It pays when the launch has the
 * GPU to itself (N = 3600, 12 heads: 84 -> 68 us) and costs SM-time when
 * other kernels run beside it.  The cut depends on the segment's length only,
 * so a segment's output is bit for bit the same alone and among other
 * segments; against the uncut form it is equal within rounding.  The
 * step-level entry point keeps its partial-result buffer per device (grown on
 * demand).
 */
#define REVO_ATTN_SPLIT_TAIL 1
REVO_API revo_status revo_op_attention(revo_precision precision, const void* qkv, void* out, int M, int D,
                              int heads, const int* seg_start, const int* q_begin, const int* q_end, int n_seg,
                              int flags, void* stream);

/*
 * x[(s*Hp + r)*Wp + c][:] += the sinusoidal embedding of (taus[s], r, c), each
 * part D/3 wide, half sines half cosines at frequencies 10000^(-2i/(D/3))
 * (Section 3.4.1: the embedding encodes the temporal distance between the
 * references and the target).  x float32 device; taus host, `slots` <= 8;
 * D a multiple of 192, at most 1024.
 */
REVO_API revo_status revo_op_add_position(float* x, int slots, int grid_h, int grid_w, int D, const int* taus,
                                 void* stream);

/*
 * De-normalise, quantise and blend one recovered frame.  head [Hp*Wp][C*p*p]
 * float32 holds, per patch of the current frame, the pixel head's outputs for
 * that frame ordered (c, y, x).  RGB: v = y*std_c + mean_c in [0,1] units, code
 * = clamp(rint(255 v), 0, 255).  Depth: v = y*sigma + mu mm, code = clamp(rint(v),
 * 0, 65535).  out = lost ? code : decoded, bit for bit for received pixels;
 * values (optional, dense float32 [H][W][C]) gets v at every pixel.
 */
/*
 * Batched forms (p = 16): every job of the batch in one launch, as the
 * recovery forward runs them.  The jobs are copied (on `stream`) into a
 * per-device argument table unless it already holds the same jobs; calls on
 * one device must run in stream order.  Results are bit for bit those of the
 * single-job calls.  n <= 64.
 */
typedef struct {
  int height, width;
  const void* frames[8];   /* device: the k references oldest first, then the current frame */
  size_t pitch_bytes;
  const float* mu_sigma;   /* depth: device (mu, sigma); RGB: NULL */
  void* out;               /* device: [S*Hp*Wp][T*C*p*p] */
} revo_assemble_job;
REVO_API revo_status revo_op_assemble_batch(int channels, int k, int T, int n, const revo_assemble_job* jobs,
                                            int out_bf16, void* stream);

/*
 * The tubelet embedding of a batch as one implicit GEMM (Section 3.4.1: the
 * tubelet Conv3d with kernel = stride = (T, 16, 16), plus the sinusoidal
 * embedding of temporal distance, patch row and patch column).  The token
 * matrix is never stored: the kernel reads each token's pixels from the
 * jobs' frames, normalises them (as revo_op_assemble_batch does) into the
 * tensor-core operand, and adds bias and position embedding in its epilogue.
 * jobs as for revo_op_assemble_batch (frames and pitch device; `out` is not
 * used); taus host [n][8]: job i's temporal distance per slot at taus[i*8 +
 * s]; W bf16 [N][K] device with K = T * channels * 256 in (t, c, y, x) order;
 * bias float32 [N] (may be NULL); out float32 [M][N] device, M = the jobs'
 * token counts ((k + 1) / T * H/16 * W/16 each) summed, rows in job order.
 * T 1 or 2, (k + 1) % T == 0, at most 8 slots, H and W multiples of 16; N a
 * multiple of 192 up to 1024.  The K blocks (64 wide) are accumulated with the
 * channel blocks of each (frame, patch-row quad) together, so that each pixel
 * is read once: depth bit for bit revo_op_assemble_batch (bf16) then
 * revo_op_linear_pe per job, RGB the same sums in another order (equal within
 * float32 rounding).  Uses the per-device position scratch and
 * argument table (calls on one device in stream order).
 * Errors: REVO_EINVAL, REVO_ENOMEM, REVO_ECUDA.
 */
REVO_API revo_status revo_op_embed_batch(int channels, int k, int T, int n, const revo_assemble_job* jobs,
                                         const int* taus, const void* W, const float* bias, float* out, int N,
                                         void* stream);

typedef struct {
  int height, width;
  const float* head;       /* device [Hp*Wp][C*p*p] */
  const void* decoded;     /* device frame */
  size_t pitch_bytes;
  const uint32_t* mask;    /* device */
  size_t mask_pitch_words;
  const float* mu_sigma;   /* depth: device (mu, sigma) */
  void* out;               /* device frame */
  size_t out_pitch;
  float* values;           /* optional */
} revo_blend_job;
REVO_API revo_status revo_op_blend_batch(int channels, int n, const revo_blend_job* jobs, void* stream);

REVO_API revo_status revo_op_blend(int channels, int p, int height, int width, const float* head,
                          const void* decoded, size_t pitch_bytes, const uint32_t* mask,
                          size_t mask_pitch_words, const float* mu_sigma, void* out,
                          size_t out_pitch, float* values, void* stream);

/*
 * Returns and clears the device error word of the step-level tensor-core
 * kernels on the current device: 0 = no failure, otherwise the code of the
 * first pipeline wait that gave up (the kernel then returned early and its
 * output is incomplete).  -1 if the word cannot be read.  Synchronous.
 */
REVO_API int revo_op_take_device_error(void);

/*
 * Diagnostic of the bounded waits: launches one thread that waits on a
 * barrier nothing completes.  After `limit_cycles` SM clocks (1000 ..
 * 2e9) the wait gives up, records code 5 in the step-level device error word
 * (read it with revo_op_take_device_error) and the kernel returns; the device
 * stays usable.  The pipeline kernels give up the same way (codes 1-4).
 * Errors: REVO_EINVAL (limit out of range), REVO_ECUDA.
 */
REVO_API revo_status revo_op_wait_selftest(long long limit_cycles, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* REVO_H */
