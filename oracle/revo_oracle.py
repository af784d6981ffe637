"""FP64 CPU oracle of ReVo's post-decode neural loss recovery (Section 3.4).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA path never imports this
module and this module imports nothing from it.

What it computes, for one modality (RGB, C = 3 or depth, C = 1):

  1. normalise the k clean reference frames and the decoded current frame
     (Section 3.4.1 feeds the k closest clean frames plus the corrupted frame;
     Appendix B.1 point 3 feeds intact and corrupted pixels alike);
  2. cut the k+1 frames into tubelets of T frames x p x p pixels
     (Appendix B.3) and embed each with one linear map (the Conv3d with
     kernel = stride = (T, p, p));
  3. add a sinusoidal embedding of (temporal distance, patch row, patch
     column) -- Section 3.4.1 encodes the temporal distance between the
     references and the target;
  4. run the encoder of pre-LayerNorm transformer blocks with full
     softmax attention over every token (Appendix B.1 points 1, 4, 5: the
     encoder-decoder is kept at inference, attention is exact scaled
     dot-product attention, no token shuffling), a final LayerNorm, a linear
     map to the decoder width, the decoder embedding, the decoder blocks and
     a final LayerNorm;
  5. a linear pixel head per token, un-patchified; the current frame is the
     last frame of the last tubelet (Section 3.4.1: the output is one
     reconstructed frame);
  6. de-normalise, and blend: pixels the loss mask marks as received keep
     their decoded value exactly, lost pixels take the recovered value
     rounded half-to-even and clamped to the integer range.

Readings where the paper is silent (widths, normalisation, embedding, blend
rule, rounding) follow the ViT-B VideoMAE family the paper builds on; they
are listed with the design notes of this repository.  Everything is plain
numpy float64; matrix products use ``@`` as a library step, softmax and
LayerNorm are written out.  Every function is pinned by tests that compare it
with torch's float64 modules, brute-force summation, closed forms and
invariants.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

# ImageNet statistics used by the VideoMAE family for RGB input (reading).
RGB_MEAN = np.array([0.485, 0.456, 0.406], dtype=np.float64)
RGB_STD = np.array([0.229, 0.224, 0.225], dtype=np.float64)
LN_EPS = 1e-6
DEPTH_SIGMA_FLOOR = 1.0  # millimetres


# ---------------------------------------------------------------- step 1 ----

def normalise_rgb(frame: np.ndarray) -> np.ndarray:
    """uint8 [H, W, 3] -> float64 [3, H, W]: (x / 255 - mean_c) / std_c."""
    x = frame.astype(np.float64) / 255.0
    return ((x - RGB_MEAN) / RGB_STD).transpose(2, 0, 1)


def depth_stats(frame: np.ndarray) -> tuple[float, float]:
    """Mean and (biased) standard deviation of the non-zero depth pixels.

    Zero depth means "no measurement" and is excluded.  With no valid pixel
    the statistics are (0, 1); the deviation is floored at 1 mm.
    """
    v = frame[frame > 0].astype(np.float64)
    if v.size == 0:
        return 0.0, 1.0
    mu = v.mean()
    sigma = np.sqrt(((v - mu) ** 2).mean())
    return float(mu), float(max(sigma, DEPTH_SIGMA_FLOOR))


def normalise_depth(frame: np.ndarray, mu: float, sigma: float) -> np.ndarray:
    """uint16 mm [H, W] -> float64 [1, H, W]: (d - mu) / sigma, zeros included."""
    return ((frame.astype(np.float64) - mu) / sigma)[None]


# ---------------------------------------------------------------- step 2 ----

def tubelets(frames: np.ndarray, T: int, p: int) -> np.ndarray:
    """[F, C, H, W] -> [S * Hp * Wp, T * C * p * p], S = F / T.

    Token order (slot s, patch row, patch column); each token's vector is its
    tubelet flattened as (t, c, y, x).  Appendix B.3: a tubelet groups T
    consecutive frames of one p x p patch into one token.
    """
    F, C, H, W = frames.shape
    S, Hp, Wp = F // T, H // p, W // p
    x = frames.reshape(S, T, C, Hp, p, Wp, p)          # s t c ty y tx x
    x = x.transpose(0, 3, 5, 1, 2, 4, 6)               # s ty tx t c y x
    return x.reshape(S * Hp * Wp, T * C * p * p)


def untubelet_frame(tokens: np.ndarray, C: int, T: int, p: int, Hp: int, Wp: int, t: int) -> np.ndarray:
    """Inverse of ``tubelets`` for one slot: [Hp * Wp, T * C * p * p] -> frame t, [C, H, W]."""
    x = tokens.reshape(Hp, Wp, T, C, p, p)[:, :, t]     # ty tx c y x
    return x.transpose(2, 0, 3, 1, 4).reshape(C, Hp * p, Wp * p)


# ---------------------------------------------------------------- step 3 ----

def sincos(pos: float, d: int) -> np.ndarray:
    """[sin(pos w_i) for i < d/2] + [cos(pos w_i) for i < d/2], w_i = 10000^(-2i/d)."""
    i = np.arange(d // 2, dtype=np.float64)
    w = 10000.0 ** (-2.0 * i / d)
    return np.concatenate([np.sin(pos * w), np.cos(pos * w)])


def position_embedding(taus, Hp: int, Wp: int, dim: int) -> np.ndarray:
    """[S * Hp * Wp, dim]: the token (s, r, c) gets sincos(tau_s) | sincos(r) | sincos(c),
    each part dim / 3 wide."""
    part = dim // 3
    rows = []
    for tau in taus:
        for r in range(Hp):
            for c in range(Wp):
                rows.append(np.concatenate([sincos(tau, part), sincos(r, part), sincos(c, part)]))
    return np.array(rows)


def temporal_distances(ref_index, target_index: int, T: int) -> list[int]:
    """tau of each slot: target index minus the index of the slot's first frame.

    The F = k + 1 frames are the refs (oldest first) then the target.
    """
    idx = list(ref_index) + [target_index]
    return [int(target_index - idx[s * T]) for s in range(len(idx) // T)]


# ---------------------------------------------------------------- step 4 ----

def linear(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = x W^T + b for W [out, in]."""
    return x @ w.T + b


def layer_norm(x: np.ndarray, g: np.ndarray, b: np.ndarray, eps: float = LN_EPS) -> np.ndarray:
    """Per-row (x - mean) / sqrt(biased var + eps) * g + b."""
    mu = x.mean(axis=-1, keepdims=True)
    var = ((x - mu) ** 2).mean(axis=-1, keepdims=True)
    return (x - mu) / np.sqrt(var + eps) * g + b


def gelu(x: np.ndarray) -> np.ndarray:
    """Exact GELU: x Phi(x) = x (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def softmax_rows(s: np.ndarray) -> np.ndarray:
    e = np.exp(s - s.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def attention(qkv: np.ndarray, heads: int) -> np.ndarray:
    """Multi-head softmax(Q K^T / sqrt(d_h)) V over every token.

    qkv is [N, 3D] laid out as [q | k | v]; head h owns columns h*d_h..(h+1)*d_h
    of each part.  Returns the concatenated head outputs [N, D].
    """
    N, D3 = qkv.shape
    D = D3 // 3
    dh = D // heads
    q, k, v = qkv[:, :D], qkv[:, D:2 * D], qkv[:, 2 * D:]
    out = np.empty((N, D))
    for h in range(heads):
        cols = slice(h * dh, (h + 1) * dh)
        p = softmax_rows(q[:, cols] @ k[:, cols].T / np.sqrt(dh))
        out[:, cols] = p @ v[:, cols]
    return out


def block(x: np.ndarray, w: dict, prefix: str, heads: int) -> np.ndarray:
    """Pre-LN transformer block: x + proj(attn(LN1 x)); then x + fc2(gelu(fc1(LN2 x)))."""
    h = layer_norm(x, w[prefix + "ln1.g"], w[prefix + "ln1.b"])
    a = attention(linear(h, w[prefix + "qkv.w"], w[prefix + "qkv.b"]), heads)
    x = x + linear(a, w[prefix + "proj.w"], w[prefix + "proj.b"])
    h = layer_norm(x, w[prefix + "ln2.g"], w[prefix + "ln2.b"])
    h = gelu(linear(h, w[prefix + "fc1.w"], w[prefix + "fc1.b"]))
    return x + linear(h, w[prefix + "fc2.w"], w[prefix + "fc2.b"])


# ---------------------------------------------------------------- step 5 ----

def forward(w: dict, cfg, frames: np.ndarray, taus) -> np.ndarray:
    """Network output for the current frame, in normalised units, [C, H, W].

    ``frames`` is [k + 1, C, H, W] normalised (refs oldest first, then the
    decoded current frame); ``w`` maps parameter names to arrays (any float
    type; used as float64); ``cfg`` carries the shape (k, tubelet, patch,
    widths, depths, heads).
    """
    w = {n: np.asarray(a, dtype=np.float64) for n, a in w.items()}
    F, C, H, W = frames.shape
    T, p = cfg.tubelet, cfg.patch
    Hp, Wp = H // p, W // p
    x = linear(tubelets(frames, T, p), w["patch_embed.w"], w["patch_embed.b"])
    x = x + position_embedding(taus, Hp, Wp, cfg.enc_dim)
    for i in range(cfg.enc_depth):
        x = block(x, w, f"enc.{i}.", cfg.enc_heads)
    x = layer_norm(x, w["enc_norm.g"], w["enc_norm.b"])
    x = linear(x, w["enc2dec.w"], w["enc2dec.b"])
    x = x + position_embedding(taus, Hp, Wp, cfg.dec_dim)
    for i in range(cfg.dec_depth):
        x = block(x, w, f"dec.{i}.", cfg.dec_heads)
    x = layer_norm(x, w["dec_norm.g"], w["dec_norm.b"])
    y = linear(x, w["head.w"], w["head.b"])
    S = F // T
    last = y[(S - 1) * Hp * Wp:]
    return untubelet_frame(last, C, T, p, Hp, Wp, T - 1)


# ---------------------------------------------------------------- step 6 ----

# The de-normalise and quantise steps take a ``dtype``: float64 by default; a
# check of codes produced in float32 passes np.float32 so that the rounding
# decision is taken in the same precision (each product and sum rounded once,
# no fused multiply-add).

def denormalise_rgb(y: np.ndarray, dtype=np.float64) -> np.ndarray:
    """[3, H, W] normalised -> [H, W, 3] in [0, 1] units (not clamped): y std_c + mean_c."""
    y = np.asarray(y, dtype=dtype)
    return y.transpose(1, 2, 0) * RGB_STD.astype(dtype) + RGB_MEAN.astype(dtype)


def denormalise_depth(y: np.ndarray, mu: float, sigma: float, dtype=np.float64) -> np.ndarray:
    """[1, H, W] normalised -> [H, W] millimetres (not clamped): y sigma + mu."""
    return np.asarray(y, dtype=dtype)[0] * dtype(sigma) + dtype(mu)


def quantise_rgb(v: np.ndarray, dtype=np.float64) -> np.ndarray:
    """[0, 1] units -> uint8: round half to even of 255 v, clamped to [0, 255]."""
    return np.clip(np.rint(np.asarray(v, dtype=dtype) * dtype(255.0)), 0, 255).astype(np.uint8)


def quantise_depth(v: np.ndarray, dtype=np.float64) -> np.ndarray:
    """millimetres -> uint16: round half to even, clamped to [0, 65535]."""
    return np.clip(np.rint(np.asarray(v, dtype=dtype)), 0, 65535).astype(np.uint16)


def blend(decoded: np.ndarray, lost: np.ndarray, recovered_codes: np.ndarray) -> np.ndarray:
    """Received pixels keep the decoded value bit for bit; lost pixels take the recovery."""
    out = decoded.copy()
    out[lost] = recovered_codes[lost]
    return out


def unpack_mask(words: np.ndarray, W: int) -> np.ndarray:
    """uint32 [H, ceil(W/32)] -> bool [H, W]; bit x % 32 of word x // 32 is pixel x, 1 = lost."""
    H = words.shape[0]
    out = np.zeros((H, W), dtype=bool)
    for x in range(W):
        out[:, x] = (words[:, x // 32] >> np.uint32(x % 32)) & np.uint32(1)
    return out


def recover(modality: str, w: dict, cfg, refs: np.ndarray, ref_index, decoded: np.ndarray,
            mask_words: np.ndarray, target_index: int):
    """One recovery request for one modality.

    Returns (codes, values): ``codes`` is the blended uint8 [H, W, 3] or uint16
    [H, W] frame; ``values`` the de-normalised network output at every pixel
    (float64, [0, 1] units for RGB, millimetres for depth), before blending.
    The depth statistics come from the newest reference frame.
    """
    H, W = decoded.shape[:2]
    lost = unpack_mask(mask_words, W)
    if modality == "rgb":
        frames = np.stack([normalise_rgb(f) for f in refs] + [normalise_rgb(decoded)])
    else:
        mu, sigma = depth_stats(refs[-1])
        frames = np.stack([normalise_depth(f, mu, sigma) for f in refs] + [normalise_depth(decoded, mu, sigma)])
    taus = temporal_distances(ref_index, target_index, cfg.tubelet)
    y = forward(w, cfg, frames, taus)
    if modality == "rgb":
        values = denormalise_rgb(y)
        codes = quantise_rgb(values)
    else:
        values = denormalise_depth(y, mu, sigma)
        codes = quantise_depth(values)
    return blend(decoded, lost, codes), values
