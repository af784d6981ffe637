"""Python binding of librevo (the C ABI declared in include/revo.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Importing this module does not load the library; the first call does, and
raises if librevo.so has not been built (``python -m paper_2604_27441_b300.build``).
Tensors may be passed as torch tensors, numpy arrays or raw integer pointers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librevo.so")

REVO_OK, REVO_EAGAIN, REVO_EINVAL, REVO_ENOMEM, REVO_ETIMEDOUT, REVO_ENOREF, REVO_ECUDA, REVO_ENOTSUP = \
    0, 1, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "REVO_OK", 1: "REVO_EAGAIN", -1: "REVO_EINVAL", -2: "REVO_ENOMEM", -3: "REVO_ETIMEDOUT",
                -4: "REVO_ENOREF", -5: "REVO_ECUDA", -6: "REVO_ENOTSUP"}
FP32, BF16, FP8 = 0, 1, 2
RGB, DEPTH, CLEAN, HOLD = 1, 2, 4, 8
EPI_F32, EPI_BF16, EPI_GELU_BF16, EPI_RESID_F32 = 0, 1, 2, 3
TILE_PAIR = 0x1000  # REVO_TILE_PAIR: OR into tile_n for 256-row tiles on a CTA pair


class RevoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("k", C.c_int), ("tubelet", C.c_int), ("patch", C.c_int),
                ("enc_dim", C.c_int), ("enc_depth", C.c_int), ("enc_heads", C.c_int),
                ("dec_dim", C.c_int), ("dec_depth", C.c_int), ("dec_heads", C.c_int),
                ("mlp_ratio", C.c_int), ("precision", C.c_int), ("device", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("max_streams", C.c_int),
                ("max_height", C.c_int), ("max_width", C.c_int), ("max_batch", C.c_int), ("lanes", C.c_int),
                ("cuda_stream", C.c_void_p), ("use_graphs", C.c_int), ("autotune", C.c_int),
                ("fp8_layers", C.c_int),
                ("rgb_weights", C.c_void_p), ("rgb_weights_count", C.c_size_t),
                ("depth_weights", C.c_void_p), ("depth_weights_count", C.c_size_t),
                ("rgb_weights_path", C.c_char_p), ("depth_weights_path", C.c_char_p),
                ("seed", C.c_uint64), ("random_init", C.c_int), ("autotune_cache", C.c_char_p),
                ("serial_models", C.c_int)]


class Plane(C.Structure):
    _fields_ = [("data", C.c_void_p), ("height", C.c_int), ("width", C.c_int), ("pitch_bytes", C.c_size_t)]


class Request(C.Structure):
    _fields_ = [("stream_id", C.c_uint32), ("frame_index", C.c_int64), ("flags", C.c_uint32),
                ("inputs_on_device", C.c_int),
                ("rgb", Plane), ("rgb_lost_mask", C.c_void_p), ("rgb_mask_pitch_words", C.c_size_t),
                ("depth", Plane), ("depth_lost_mask", C.c_void_p), ("depth_mask_pitch_words", C.c_size_t),
                ("outputs_on_device", C.c_int),
                ("rgb_out", C.c_void_p), ("rgb_out_pitch", C.c_size_t),
                ("depth_out", C.c_void_p), ("depth_out_pitch", C.c_size_t),
                ("rgb_values", C.c_void_p), ("depth_values", C.c_void_p)]


class AssembleJob(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("frames", C.c_void_p * 8), ("pitch_bytes", C.c_size_t),
                ("mu_sigma", C.c_void_p), ("out", C.c_void_p)]


class BlendJob(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("head", C.c_void_p), ("decoded", C.c_void_p),
                ("pitch_bytes", C.c_size_t), ("mask", C.c_void_p), ("mask_pitch_words", C.c_size_t),
                ("mu_sigma", C.c_void_p), ("out", C.c_void_p), ("out_pitch", C.c_size_t), ("values", C.c_void_p)]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float)]


class Pose(C.Structure):
    _fields_ = [("r", C.c_float * 9), ("t", C.c_float * 3)]


class Stats(C.Structure):
    _fields_ = [("device_bytes", C.c_size_t), ("batches", C.c_uint64), ("graph_replays", C.c_uint64),
                ("graphs_captured", C.c_int), ("tuned_shapes", C.c_int), ("tuned_wide", C.c_int),
                ("pending", C.c_int), ("in_flight", C.c_int), ("tuned_pair", C.c_int),
                ("tuned_timed", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("stream_id", C.c_uint32), ("frame_index", C.c_int64),
                ("latency_ms", C.c_double), ("device_ms", C.c_double), ("batch_size", C.c_int),
                ("kernel_launches", C.c_int)]


_lib = None

_SIGS = {
    "revo_config_default": (None, [C.POINTER(Config)]),
    "revo_recover_create": (C.c_int, [C.POINTER(Config), C.POINTER(C.c_void_p)]),
    "revo_recover_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "revo_recover_flush": (C.c_int, [C.c_void_p]),
    "revo_recover_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(Result)]),
    "revo_recover_destroy": (None, [C.c_void_p]),
    "revo_recover_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "revo_last_error": (C.c_char_p, []),
    "revo_op_assemble": (C.c_int, [C.c_int] * 6 + [C.POINTER(C.c_void_p), C.c_void_p, C.c_size_t, C.c_void_p,
                                                  C.c_void_p, C.c_int, C.c_void_p]),
    "revo_depth_stats_scratch_bytes": (C.c_size_t, []),
    "revo_op_depth_stats": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_size_t, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "revo_op_linear": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "revo_op_layernorm": (C.c_int, [C.c_void_p] * 4 + [C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "revo_op_linear_pe": (C.c_int, [C.c_void_p] * 4 + [C.c_int] * 5 + [C.POINTER(C.c_int), C.c_int, C.c_void_p]),
    "revo_op_linear_resid_ln": (C.c_int, [C.c_void_p] * 4 + [C.c_int] * 3 + [C.c_void_p] * 4 + [C.c_int, C.c_int,
                                                                                               C.c_void_p]),
    "revo_op_attention": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                    C.c_int, C.c_void_p]),
    "revo_op_add_position": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                       C.c_void_p]),
    "revo_op_blend": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t,
                                C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                C.c_void_p]),
    "revo_op_take_device_error": (C.c_int, []),
    "revo_op_assemble_batch": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "revo_op_embed_batch": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_int), C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "revo_op_blend_batch": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "revo_init_weights": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_void_p, C.c_size_t]),
    "revo_op_wait_selftest": (C.c_int, [C.c_longlong, C.c_void_p]),
    "revo_op_quantize_rows_e4m3": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "revo_frame_metrics_scratch_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "revo_render_scratch_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "revo_render_rgbd": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_size_t, C.c_void_p, C.c_int, C.c_int, C.c_size_t,
                                   C.POINTER(Intrinsics), C.POINTER(Pose), C.POINTER(Intrinsics), C.c_int, C.c_int,
                                   C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "revo_fec_encode": (C.c_int, [C.c_int, C.c_int, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "revo_fec_decode_scratch_bytes": (C.c_size_t, [C.c_int]),
    "revo_fec_decode": (C.c_int, [C.c_int, C.c_int, C.c_size_t, C.POINTER(C.c_int), C.c_void_p, C.c_size_t,
                                  C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "revo_op_frame_metrics": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "revo_op_layernorm_e4m3": (C.c_int, [C.c_void_p] * 5 + [C.c_int, C.c_int, C.c_void_p]),
    "revo_op_linear_fp8": (C.c_int, [C.c_int] + [C.c_void_p] * 6 + [C.c_int] * 4 + [C.c_void_p]),
    "revo_op_depth_stats_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_size_t, C.c_void_p, C.c_void_p]),
}


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librevo.so is not built ({LIB_PATH}); run python -m paper_2604_27441_b300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return (lib().revo_last_error() or b"").decode()


def _check(status: int, where: str) -> int:
    if status not in (REVO_OK, REVO_EAGAIN):
        raise RevoError(status, where, last_error())
    return status


def ptr(x) -> int | None:
    """Raw address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous (the C ABI takes row-major buffers)")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous (the C ABI takes row-major buffers)")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ------------------------------------------------------------ step-level ops

def op_assemble(channels, k, T, p, height, width, refs, current, pitch_bytes, mu_sigma, out, out_bf16,
                stream=None):
    arr = (C.c_void_p * max(k, 1))(*[ptr(r) for r in refs])
    return _check(lib().revo_op_assemble(channels, k, T, p, height, width, arr, ptr(current), pitch_bytes,
                                         ptr(mu_sigma), ptr(out), int(out_bf16), _stream(stream)), "revo_op_assemble")


def depth_stats_scratch_bytes() -> int:
    return lib().revo_depth_stats_scratch_bytes()


def op_depth_stats(depth, height, width, pitch_bytes, mu_sigma, scratch, stream=None):
    return _check(lib().revo_op_depth_stats(ptr(depth), height, width, pitch_bytes, ptr(mu_sigma), ptr(scratch),
                                            _stream(stream)), "revo_op_depth_stats")


def op_depth_stats_noalloc(depth, height, width, pitch_bytes, mu_sigma, stream=None):
    """Depth statistics with the library's built-in scratch (no device allocation)."""
    return _check(lib().revo_op_depth_stats_noalloc(ptr(depth), height, width, pitch_bytes, ptr(mu_sigma),
                                                    _stream(stream)), "revo_op_depth_stats_noalloc")


def op_linear(precision, epilogue, A, W, bias, out, M, N, K, tile_n=0, stream=None):
    return _check(lib().revo_op_linear(precision, epilogue, ptr(A), ptr(W), ptr(bias), ptr(out), M, N, K, tile_n,
                                       _stream(stream)), "revo_op_linear")


def op_linear_pe(A, W, bias, out, slots, grid_h, grid_w, N, K, taus, tile_n=0, stream=None):
    """out = A W^T + bias + the position embedding of one request's tokens, in
    one tensor-core launch (the same floats as op_linear then op_add_position)."""
    t = (C.c_int * max(1, len(taus)))(*[int(v) for v in taus])
    return _check(lib().revo_op_linear_pe(ptr(A), ptr(W), ptr(bias), ptr(out), slots, grid_h, grid_w, N, K, t,
                                          tile_n, _stream(stream)), "revo_op_linear_pe")


def op_linear_resid_ln(A, W, bias, x, M, N, K, gamma, beta, ln_out, ln_row_scale=None, ln_fp8=False, tile_n=0,
                       stream=None):
    """x += A W^T + bias, then ln_out = LayerNorm(x) (bf16, or E4M3 codes with
    per-row scales when ln_fp8), in one tensor-core launch."""
    return _check(lib().revo_op_linear_resid_ln(ptr(A), ptr(W), ptr(bias), ptr(x), M, N, K, ptr(gamma), ptr(beta),
                                                ptr(ln_out), ptr(ln_row_scale), int(bool(ln_fp8)), tile_n,
                                                _stream(stream)), "revo_op_linear_resid_ln")


def op_layernorm(x, gamma, beta, out, M, D, out_bf16, stream=None):
    return _check(lib().revo_op_layernorm(ptr(x), ptr(gamma), ptr(beta), ptr(out), M, D, int(out_bf16),
                                          _stream(stream)), "revo_op_layernorm")


def op_quantize_rows_e4m3(x, rows, cols, q, scale, stream=None):
    return _check(lib().revo_op_quantize_rows_e4m3(ptr(x), rows, cols, ptr(q), ptr(scale), _stream(stream)),
                  "revo_op_quantize_rows_e4m3")


def op_layernorm_e4m3(x, gamma, beta, out, row_scale, M, D, stream=None):
    return _check(lib().revo_op_layernorm_e4m3(ptr(x), ptr(gamma), ptr(beta), ptr(out), ptr(row_scale), M, D,
                                               _stream(stream)), "revo_op_layernorm_e4m3")


def op_linear_fp8(epilogue, A, a_scale, W, w_scale, bias, out, M, N, K, tile_n=0, stream=None):
    return _check(lib().revo_op_linear_fp8(epilogue, ptr(A), ptr(a_scale), ptr(W), ptr(w_scale), ptr(bias), ptr(out),
                                           M, N, K, tile_n, _stream(stream)), "revo_op_linear_fp8")


def fec_encode(n, r, packet_bytes, data, parity, stream=None):
    """Parity [r][packet_bytes] of data [n][packet_bytes] (device, dense rows)."""
    return _check(lib().revo_fec_encode(n, r, packet_bytes, ptr(data), packet_bytes, ptr(parity), packet_bytes,
                                        _stream(stream)), "revo_fec_encode")


def fec_decode_scratch_bytes(n) -> int:
    return int(lib().revo_fec_decode_scratch_bytes(n))


def fec_decode(n, r, packet_bytes, present, received, data_out, scratch, stream=None):
    """Data [n][packet_bytes] from the n packets `present` (indices) stacked in `received`."""
    arr = (C.c_int * n)(*[int(p) for p in present])
    return _check(lib().revo_fec_decode(n, r, packet_bytes, arr, ptr(received), packet_bytes, ptr(data_out),
                                        packet_bytes, ptr(scratch), _stream(stream)), "revo_fec_decode")


def render_scratch_bytes(out_h, out_w) -> int:
    return int(lib().revo_render_scratch_bytes(out_h, out_w))


def render_rgbd(rgb, depth, K_src, R, t, K_dst, out_hw, splat, scratch, out_rgb, out_depth, stream=None):
    """Unproject + splat a device RGB-D frame into the target view (dense rows)."""
    rh, rw = rgb.shape[:2]
    h, w = depth.shape
    oh, ow = out_hw
    src, dst = Intrinsics(*K_src), Intrinsics(*K_dst)
    pose = Pose((C.c_float * 9)(*[float(v) for v in np.asarray(R).reshape(-1)]),
                (C.c_float * 3)(*[float(v) for v in t]))
    return _check(lib().revo_render_rgbd(ptr(rgb), rh, rw, rw * 3, ptr(depth), h, w, w * 2, C.byref(src),
                                         C.byref(pose), C.byref(dst), oh, ow, splat, ptr(scratch), ptr(out_rgb),
                                         ow * 3, ptr(out_depth), ow * 2, _stream(stream)), "revo_render_rgbd")


def frame_metrics_scratch_bytes(height, width, channels) -> int:
    return int(lib().revo_frame_metrics_scratch_bytes(height, width, channels))


def op_frame_metrics(a, b, height, width, channels, sample_bytes, data_range, scratch, out, stream=None,
                     pitch_a=None, pitch_b=None):
    """SSIM / MSE / PSNR of device frame a against b into out (device, 3 floats)."""
    row = width * channels * sample_bytes
    return _check(lib().revo_op_frame_metrics(ptr(a), pitch_a or row, ptr(b), pitch_b or row, height, width, channels,
                                              sample_bytes, float(data_range), ptr(scratch), ptr(out),
                                              _stream(stream)), "revo_op_frame_metrics")


ATTN_SPLIT_TAIL = 1


def op_attention(precision, qkv, out, M, D, heads, seg_start, stream=None, split_tail=False, queries=None):
    """queries: optional list of (begin, end) query rows per segment."""
    n = len(seg_start) - 1
    arr = (C.c_int * len(seg_start))(*[int(v) for v in seg_start])
    qb = qe = None
    if queries is not None:
        qb = (C.c_int * n)(*[int(a) for a, _ in queries])
        qe = (C.c_int * n)(*[int(b) for _, b in queries])
    flags = ATTN_SPLIT_TAIL if split_tail else 0
    return _check(lib().revo_op_attention(precision, ptr(qkv), ptr(out), M, D, heads, arr, qb, qe, n, flags,
                                          _stream(stream)),
                  "revo_op_attention")


def op_add_position(x, slots, grid_h, grid_w, D, taus, stream=None):
    arr = (C.c_int * max(len(taus), 1))(*[int(t) for t in taus])
    return _check(lib().revo_op_add_position(ptr(x), slots, grid_h, grid_w, D, arr, _stream(stream)),
                  "revo_op_add_position")


def op_blend(channels, p, height, width, head, decoded, pitch_bytes, mask, mask_pitch_words, mu_sigma, out,
             out_pitch, values=None, stream=None):
    return _check(lib().revo_op_blend(channels, p, height, width, ptr(head), ptr(decoded), pitch_bytes, ptr(mask),
                                      mask_pitch_words, ptr(mu_sigma), ptr(out), out_pitch, ptr(values),
                                      _stream(stream)), "revo_op_blend")


def op_assemble_batch(channels, k, T, jobs, out_bf16, stream=None):
    """jobs: list of dicts with height, width, frames (k refs + current), pitch_bytes, mu_sigma, out."""
    arr = (AssembleJob * len(jobs))()
    for a, j in zip(arr, jobs):
        a.height, a.width, a.pitch_bytes = j["height"], j["width"], j["pitch_bytes"]
        for f, fr in enumerate(j["frames"]):
            a.frames[f] = ptr(fr)
        a.mu_sigma = ptr(j.get("mu_sigma"))
        a.out = ptr(j["out"])
    return _check(lib().revo_op_assemble_batch(channels, k, T, len(jobs), C.cast(arr, C.c_void_p), out_bf16,
                                               _stream(stream)), "revo_op_assemble_batch")


def op_embed_batch(channels, k, T, jobs, taus, W, bias, out, N, stream=None):
    """jobs as for op_assemble_batch (no "out"); taus: per job a list of its slots' temporal distances."""
    arr = (AssembleJob * len(jobs))()
    for a, j in zip(arr, jobs):
        a.height, a.width, a.pitch_bytes = j["height"], j["width"], j["pitch_bytes"]
        for f, fr in enumerate(j["frames"]):
            a.frames[f] = ptr(fr)
        a.mu_sigma = ptr(j.get("mu_sigma"))
    t8 = (C.c_int * (8 * len(jobs)))()
    for i, ts in enumerate(taus):
        for s_, t in enumerate(ts):
            t8[8 * i + s_] = int(t)
    return _check(lib().revo_op_embed_batch(channels, k, T, len(jobs), C.cast(arr, C.c_void_p), t8, ptr(W), ptr(bias),
                                            ptr(out), N, _stream(stream)), "revo_op_embed_batch")


def op_blend_batch(channels, jobs, stream=None):
    """jobs: list of dicts with height, width, head, decoded, pitch_bytes, mask, mask_pitch_words,
    mu_sigma, out, out_pitch, values."""
    arr = (BlendJob * len(jobs))()
    for a, j in zip(arr, jobs):
        a.height, a.width, a.pitch_bytes = j["height"], j["width"], j["pitch_bytes"]
        a.head, a.decoded, a.mask = ptr(j["head"]), ptr(j["decoded"]), ptr(j["mask"])
        a.mask_pitch_words, a.mu_sigma = j["mask_pitch_words"], ptr(j.get("mu_sigma"))
        a.out, a.out_pitch, a.values = ptr(j["out"]), j["out_pitch"], ptr(j.get("values"))
    return _check(lib().revo_op_blend_batch(channels, len(jobs), C.cast(arr, C.c_void_p), _stream(stream)),
                  "revo_op_blend_batch")


def take_device_error() -> int:
    return lib().revo_op_take_device_error()


def op_wait_selftest(limit_cycles, stream=None):
    """One bounded wait that runs out: sets device error code 5 (see take_device_error)."""
    return _check(lib().revo_op_wait_selftest(int(limit_cycles), _stream(stream)), "revo_op_wait_selftest")


# ------------------------------------------------------------------ context

def config(**kw) -> Config:
    """A revo_config from revo_config_default with the given fields set
    (str values of the path fields are encoded; the Config keeps them alive)."""
    cfg = Config()
    lib().revo_config_default(C.byref(cfg))
    keep = []
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        if isinstance(v, str):
            v = v.encode()
            keep.append(v)
        setattr(cfg, k, v)
    cfg._keep_strings = keep
    return cfg


def init_weights(cfg: Config, channels: int, seed: int) -> np.ndarray:
    """revo_init_weights: the library's seeded random initialisation of one model (host)."""
    n = int(param_count(cfg, channels))
    out = np.empty(n, np.float32)
    _check(lib().revo_init_weights(C.byref(cfg), channels, seed, out.ctypes.data, n), "revo_init_weights")
    return out


def param_count(cfg: Config, channels: int) -> int:
    """Parameters of one model of the configured shape (the order of revo.h)."""
    D, Dd, r = cfg.enc_dim, cfg.dec_dim, cfg.mlp_ratio
    K = cfg.tubelet * channels * cfg.patch * cfg.patch

    def block(d):
        return 2 * d + 3 * d * d + 3 * d + d * d + d + 2 * d + r * d * d + r * d + r * d * d + d
    return D * K + D + cfg.enc_depth * block(D) + 2 * D + Dd * D + Dd + cfg.dec_depth * block(Dd) + 2 * Dd + \
        K * Dd + K


class Context:
    """A recovery context: revo_recover_create / submit / flush / poll / destroy."""

    def __init__(self, cfg: Config, rgb_weights=None, depth_weights=None, stream=None):
        self._keep = (rgb_weights, depth_weights)
        if rgb_weights is not None:
            cfg.rgb_weights = ptr(rgb_weights)
            cfg.rgb_weights_count = int(rgb_weights.size)
        if depth_weights is not None:
            cfg.depth_weights = ptr(depth_weights)
            cfg.depth_weights_count = int(depth_weights.size)
        if stream is not None:
            cfg.cuda_stream = _stream(stream)
        h = C.c_void_p()
        _check(lib().revo_recover_create(C.byref(cfg), C.byref(h)), "revo_recover_create")
        self.cfg = cfg
        self.handle = h

    def submit(self, req: Request) -> int:
        t = C.c_uint64()
        st = lib().revo_recover_submit(self.handle, C.byref(req), C.byref(t))
        if st != REVO_OK:
            raise RevoError(st, "revo_recover_submit", last_error())
        return t.value

    def flush(self):
        _check(lib().revo_recover_flush(self.handle), "revo_recover_flush")

    def poll(self, ticket: int, timeout_us: int = -1):
        """Returns a Result, or None if the request is still running (timeout 0)."""
        r = Result()
        st = lib().revo_recover_poll(self.handle, ticket, timeout_us, C.byref(r))
        if st == REVO_EAGAIN:
            return None
        if st != REVO_OK:
            raise RevoError(st, "revo_recover_poll", last_error())
        return r

    def stats(self) -> dict:
        """The context's counters (device bytes, batches, graph replays, tuned shapes, queue)."""
        st = Stats()
        _check(lib().revo_recover_stats(self.handle, C.byref(st)), "revo_recover_stats")
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def close(self):
        if self.handle:
            lib().revo_recover_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plane(data, height, width, pitch_bytes) -> Plane:
    return Plane(ptr(data), height, width, pitch_bytes)


def request(stream_id, frame_index, flags, *, on_device, rgb=None, rgb_mask=None, depth=None, depth_mask=None,
            rgb_out=None, depth_out=None, rgb_values=None, depth_values=None, outputs_on_device=None) -> Request:
    """A Request from per-modality (data, H, W) tuples; pitches and mask pitches are dense."""
    r = Request()
    r.stream_id = stream_id
    r.frame_index = frame_index
    r.flags = flags
    r.inputs_on_device = int(on_device)
    r.outputs_on_device = int(on_device if outputs_on_device is None else outputs_on_device)
    if rgb is not None:
        d, H, W = rgb
        r.rgb = Plane(ptr(d), H, W, W * 3)
        r.rgb_lost_mask = ptr(rgb_mask)
        r.rgb_mask_pitch_words = (W + 31) // 32
        r.rgb_out = ptr(rgb_out)
        r.rgb_out_pitch = W * 3
        r.rgb_values = ptr(rgb_values)
    if depth is not None:
        d, H, W = depth
        r.depth = Plane(ptr(d), H, W, W * 2)
        r.depth_lost_mask = ptr(depth_mask)
        r.depth_mask_pitch_words = (W + 31) // 32
        r.depth_out = ptr(depth_out)
        r.depth_out_pitch = W * 2
        r.depth_values = ptr(depth_values)
    return r
