"""Seeded synthetic inputs for the ReVo neural loss-recovery path.

This module only draws numbers: RGB-D frames shaped like the paper's
face-cropped conference video, Gilbert-Elliott slice losses with the
1-bit loss mask, and random-init model weights.  It holds none of the
recovery method's arithmetic, so the CPU oracle and the CUDA path can both
take their inputs from here without sharing any of the computation.

Conventions fixed here (they are input formats, not arithmetic):

* RGB frames: uint8, interleaved [H, W, 3] (what a video decoder emits).
* Depth frames: uint16 millimetres, [H, W]; 0 means "no depth".
* Loss mask: 1 bit per pixel, 1 = lost, row-major, LSB-first inside 32-bit
  words, row pitch ceil(W / 32) words.
* Weights: an ordered dict of float32 arrays (``weights``) and its flat
  concatenation in that order (``flatten``).  Linear weights are [out, in];
  the tubelet embedding is a Linear over a tubelet flattened as (t, c, y, x).
"""
from __future__ import annotations

import dataclasses
from collections import OrderedDict

import numpy as np
from scipy.ndimage import gaussian_filter

# --------------------------------------------------------------------------
# Model shape
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class ModelConfig:
    """Shape of one modality's recovery network (ViT-B VideoMAE family)."""

    channels: int            # 3 for RGB, 1 for depth
    k: int = 5               # clean reference frames
    tubelet: int = 2         # frames per token (T)
    patch: int = 16          # spatial patch (p)
    enc_dim: int = 768
    enc_depth: int = 12
    enc_heads: int = 12
    dec_dim: int = 384
    dec_depth: int = 4
    dec_heads: int = 6
    mlp_ratio: int = 4

    @property
    def frames(self) -> int:
        return self.k + 1

    @property
    def slots(self) -> int:
        return self.frames // self.tubelet

    @property
    def token_dim(self) -> int:
        return self.tubelet * self.channels * self.patch * self.patch

    def tokens(self, height: int, width: int) -> int:
        return self.slots * (height // self.patch) * (width // self.patch)


RGB = ModelConfig(channels=3)
DEPTH = ModelConfig(channels=1)


def tiny(channels: int, **kw) -> ModelConfig:
    """A small network of the same family for fast tests."""
    base = dict(channels=channels, k=1, tubelet=2, patch=4, enc_dim=24, enc_depth=1,
                enc_heads=2, dec_dim=12, dec_depth=1, dec_heads=2, mlp_ratio=4)
    base.update(kw)
    return ModelConfig(**base)


def param_shapes(cfg: ModelConfig) -> "OrderedDict[str, tuple]":
    """Names and shapes of every parameter, in file order."""
    D, Dd, K = cfg.enc_dim, cfg.dec_dim, cfg.token_dim
    out: "OrderedDict[str, tuple]" = OrderedDict()
    out["patch_embed.w"] = (D, K)
    out["patch_embed.b"] = (D,)

    def block(prefix: str, d: int) -> None:
        h = cfg.mlp_ratio * d
        out[prefix + "ln1.g"] = (d,)
        out[prefix + "ln1.b"] = (d,)
        out[prefix + "qkv.w"] = (3 * d, d)
        out[prefix + "qkv.b"] = (3 * d,)
        out[prefix + "proj.w"] = (d, d)
        out[prefix + "proj.b"] = (d,)
        out[prefix + "ln2.g"] = (d,)
        out[prefix + "ln2.b"] = (d,)
        out[prefix + "fc1.w"] = (h, d)
        out[prefix + "fc1.b"] = (h,)
        out[prefix + "fc2.w"] = (d, h)
        out[prefix + "fc2.b"] = (d,)

    for i in range(cfg.enc_depth):
        block(f"enc.{i}.", D)
    out["enc_norm.g"] = (D,)
    out["enc_norm.b"] = (D,)
    out["enc2dec.w"] = (Dd, D)
    out["enc2dec.b"] = (Dd,)
    for i in range(cfg.dec_depth):
        block(f"dec.{i}.", Dd)
    out["dec_norm.g"] = (Dd,)
    out["dec_norm.b"] = (Dd,)
    out["head.w"] = (K, Dd)
    out["head.b"] = (K,)
    return out


def weights(cfg: ModelConfig, seed: int = 0, head_scale: float = 0.1) -> "OrderedDict[str, np.ndarray]":
    """Random-init float32 weights, drawn in file order from PCG64(seed).

    Matrices: Xavier-uniform, bound sqrt(6 / (fan_in + fan_out)) for an
    [out, in] matrix; the pixel head is further scaled by ``head_scale`` so
    the untrained output has a small, trained-model-like residual size.
    Biases: U(-0.02, 0.02).  LayerNorm gain 1 + U(-0.1, 0.1), shift
    U(-0.02, 0.02).  Non-zero biases and gains are deliberate: a dropped
    bias or affine term then shows up in every parity test.
    """
    rng = np.random.default_rng(seed)
    out: "OrderedDict[str, np.ndarray]" = OrderedDict()
    for name, shape in param_shapes(cfg).items():
        if name.endswith(".w"):
            fan_out, fan_in = shape
            bound = np.sqrt(6.0 / (fan_in + fan_out))
            w = rng.uniform(-bound, bound, size=shape)
            if name == "head.w":
                w = w * head_scale
        elif name.endswith(".g"):
            w = 1.0 + rng.uniform(-0.1, 0.1, size=shape)
        else:
            w = rng.uniform(-0.02, 0.02, size=shape)
        out[name] = w.astype(np.float32)
    return out


def flatten(w: "OrderedDict[str, np.ndarray]") -> np.ndarray:
    """The flat float32 weight blob, parameters concatenated in file order."""
    return np.concatenate([np.ascontiguousarray(a, dtype=np.float32).ravel() for a in w.values()])


def normal(seed: int, shape, scale: float = 1.0, dtype=np.float32) -> np.ndarray:
    """Seeded i.i.d. N(0, scale^2) array, for step-level checks."""
    return (np.random.default_rng(seed).normal(0.0, scale, size=shape)).astype(dtype)


# --------------------------------------------------------------------------
# Frames
# --------------------------------------------------------------------------


def _shift(img: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """Integer translation with edge replication: out[y, x] = img[y - dy, x - dx]."""
    H, W = img.shape[:2]
    ys = np.clip(np.arange(H) - dy, 0, H - 1)
    xs = np.clip(np.arange(W) - dx, 0, W - 1)
    return np.ascontiguousarray(img[ys][:, xs])


def rgb_frame(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    """Smooth per-channel gradient plus Gaussian texture, uint8 [H, W, 3].

    Channel c: a_c + b_c x / W + c_c y / H with a in [40, 200] and
    |b|, |c| <= 60, plus white noise blurred by a sigma = 1.5 px Gaussian and
    rescaled to a standard deviation of 12 grey levels.
    """
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.empty((H, W, 3))
    for c in range(3):
        a = rng.uniform(40, 200)
        b = rng.uniform(-60, 60)
        g = rng.uniform(-60, 60)
        img[..., c] = a + b * xx / W + g * yy / H
    noise = gaussian_filter(rng.normal(0.0, 1.0, size=(H, W, 3)), sigma=(1.5, 1.5, 0))
    noise *= 12.0 / max(noise.std(), 1e-12)
    return np.clip(np.rint(img + noise), 0, 255).astype(np.uint8)


def depth_frame(rng: np.random.Generator, H: int, W: int, lo: float, hi: float) -> np.ndarray:
    """Background plane plus 3 random planes/spheres composited by minimum z.

    Returns float64 millimetres in [lo, hi] (quantised by the caller).
    """
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    span = hi - lo
    z = lo + span * (rng.uniform(0.6, 0.8) + rng.uniform(-0.1, 0.1) * xx / W
                     + rng.uniform(-0.1, 0.1) * yy / H)
    for _ in range(3):
        if rng.random() < 0.5:   # sphere
            cx, cy = rng.uniform(0.2, 0.8) * W, rng.uniform(0.2, 0.8) * H
            r = rng.uniform(0.1, 0.3) * min(H, W)
            zc = lo + span * rng.uniform(0.1, 0.5)
            d2 = (xx - cx) ** 2 + (yy - cy) ** 2
            inside = d2 < r * r
            zs = np.where(inside, zc - np.sqrt(np.maximum(r * r - d2, 0.0)) * 2.0, np.inf)
        else:                     # tilted rectangle of a plane
            x0, x1 = np.sort(rng.uniform(0, W, size=2))
            y0, y1 = np.sort(rng.uniform(0, H, size=2))
            z1 = lo + span * rng.uniform(0.2, 0.6)
            gx, gy = rng.uniform(-1, 1, size=2)
            inside = (xx >= x0) & (xx <= x1) & (yy >= y0) & (yy <= y1)
            zs = np.where(inside, z1 + gx * (xx - x0) + gy * (yy - y0), np.inf)
        z = np.minimum(z, zs)
    return np.clip(z, lo, hi)


def quantise_depth(z: np.ndarray, rng: np.random.Generator, invalid_frac: float) -> np.ndarray:
    d = np.clip(np.rint(z), 0, 65535).astype(np.uint16)
    if invalid_frac > 0:
        d[rng.random(d.shape) < invalid_frac] = 0
    return d


# --------------------------------------------------------------------------
# Loss
# --------------------------------------------------------------------------


def gilbert_elliott(rng: np.random.Generator, n: int, p_gb: float, p_bg: float) -> np.ndarray:
    """Loss indicator of n consecutive slices under a two-state Markov chain.

    Good -> Bad with p_gb, Bad -> Good with p_bg; a slice is lost exactly when
    the chain is Bad.  The first state is drawn from the stationary law,
    P(Bad) = p_gb / (p_gb + p_bg).
    """
    bad = rng.random() < p_gb / (p_gb + p_bg)
    out = np.zeros(n, dtype=bool)
    for i in range(n):
        if i > 0:
            u = rng.random()
            bad = (u >= p_bg) if bad else (u < p_gb)
        out[i] = bad
    return out


def p_gb_for_rate(rate: float, p_bg: float = 0.5) -> float:
    """Good->Bad probability whose stationary loss rate is ``rate``."""
    return rate * p_bg / (1.0 - rate)


def pack_mask(lost: np.ndarray) -> np.ndarray:
    """bool [H, W] -> uint32 [H, ceil(W/32)], bit (x % 32) of word x // 32."""
    H, W = lost.shape
    words = (W + 31) // 32
    padded = np.zeros((H, words * 32), dtype=np.uint64)
    padded[:, :W] = lost
    bits = padded.reshape(H, words, 32) << np.arange(32, dtype=np.uint64)
    return bits.sum(axis=2).astype(np.uint32)


def unpack_mask(words: np.ndarray, W: int) -> np.ndarray:
    H = words.shape[0]
    bits = (words[:, :, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)) & 1
    return bits.reshape(H, -1)[:, :W].astype(bool)


def slice_mask(rng: np.random.Generator, H: int, W: int, p_gb: float, p_bg: float,
               slice_rows: int = 16) -> np.ndarray:
    """Per-pixel loss from Gilbert-Elliott losses of slices of ``slice_rows`` rows."""
    n = (H + slice_rows - 1) // slice_rows
    lost_slices = gilbert_elliott(rng, n, p_gb, p_bg)
    return np.repeat(lost_slices, slice_rows)[:H, None] & np.ones((1, W), dtype=bool)


# --------------------------------------------------------------------------
# One request
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Plane:
    """One modality of one request: history, the decoded current frame, the loss."""

    refs: np.ndarray          # [k, H, W, 3] uint8 or [k, H, W] uint16, oldest first
    ref_index: np.ndarray     # [k] int64 frame indices of the refs
    clean: np.ndarray         # current frame before loss
    decoded: np.ndarray       # current frame with lost pixels zeroed
    lost: np.ndarray          # bool [H, W]
    mask: np.ndarray          # uint32 [H, ceil(W/32)]
    index: int                # frame index of the current frame

    @property
    def height(self) -> int:
        return self.decoded.shape[0]

    @property
    def width(self) -> int:
        return self.decoded.shape[1]


def _history(rng: np.random.Generator, cur: np.ndarray, k: int) -> np.ndarray:
    """k refs, oldest first; ref j is the current frame shifted by a cumulative
    integer offset, each step uniform in {-3..3} in x and y."""
    refs = []
    dx = dy = 0
    for _ in range(k):
        dx += int(rng.integers(-3, 4))
        dy += int(rng.integers(-3, 4))
        refs.append(_shift(cur, dx, dy))
    return np.ascontiguousarray(np.stack(refs[::-1]))


def make_plane(rng: np.random.Generator, modality: str, H: int, W: int, k: int,
               p_gb: float, p_bg: float, index: int = 100, delta: int = 1,
               depth_range=(500.0, 4000.0), invalid_frac: float = 0.0) -> Plane:
    if modality == "rgb":
        cur = rgb_frame(rng, H, W)
        refs = _history(rng, cur, k)
    else:
        z = depth_frame(rng, H, W, *depth_range)
        refs_z = _history(rng, z, k)
        cur = quantise_depth(z, rng, invalid_frac)
        refs = np.stack([quantise_depth(r, rng, invalid_frac) for r in refs_z])
    lost = slice_mask(rng, H, W, p_gb, p_bg)
    decoded = cur.copy()
    decoded[lost] = 0
    ref_index = np.arange(index - delta - k + 1, index - delta + 1, dtype=np.int64)
    return _plane(refs, ref_index, cur, decoded, lost, index)


def _plane(refs, ref_index, cur, decoded, lost, index) -> Plane:
    # Every array C-contiguous: the C ABI takes raw row-major pointers.
    c = np.ascontiguousarray
    return Plane(refs=c(refs), ref_index=c(ref_index), clean=c(cur), decoded=c(decoded), lost=c(lost),
                 mask=c(pack_mask(lost)), index=index)


# Workloads shaped like the paper's (face-cropped RGB-D conference frames).
# Each entry: RGB (H, W), depth (H, W), depth range, invalid-depth fraction.
WORKLOADS = {
    "320x240": dict(rgb=(240, 320), depth=(240, 320), depth_range=(500.0, 4000.0), invalid=0.0),
    "640x480": dict(rgb=(480, 640), depth=(480, 640), depth_range=(500.0, 4000.0), invalid=0.0),
    "1280x720+640x576": dict(rgb=(720, 1280), depth=(576, 640), depth_range=(300.0, 5000.0),
                             invalid=0.02),
}


def make_request(seed: int, workload: str = "320x240", k: int = 5, loss_rate: float | None = None,
                 p_gb: float = 0.05, p_bg: float = 0.5, index: int = 100, delta: int = 1):
    """An RGB plane and a depth plane for one frame of one stream.

    With ``loss_rate`` set, p_gb is chosen so the stationary slice-loss rate
    equals it (p_bg stays 0.5); otherwise p_gb / p_bg are used as given.
    """
    wl = WORKLOADS[workload]
    if loss_rate is not None:
        p_gb = p_gb_for_rate(loss_rate, p_bg)
    rng = np.random.default_rng(seed)
    rgb = make_plane(rng, "rgb", *wl["rgb"], k, p_gb, p_bg, index, delta)
    dep = make_plane(rng, "depth", *wl["depth"], k, p_gb, p_bg, index, delta,
                     depth_range=wl["depth_range"], invalid_frac=wl["invalid"])
    return rgb, dep


def make_tiny_plane(seed: int, modality: str, H: int, W: int, k: int, lost_rows=None,
                    index: int = 10, delta: int = 1) -> Plane:
    """A small plane for oracle/kernel tests; ``lost_rows`` lists lost rows
    (default: a seeded Gilbert-Elliott draw over 4-row slices)."""
    rng = np.random.default_rng(seed)
    if modality == "rgb":
        cur = rgb_frame(rng, H, W)
        refs = _history(rng, cur, k)
    else:
        z = depth_frame(rng, H, W, 500.0, 4000.0)
        refs_z = _history(rng, z, k)
        cur = quantise_depth(z, rng, 0.02)
        refs = np.stack([quantise_depth(r, rng, 0.02) for r in refs_z])
    if lost_rows is None:
        lost = slice_mask(rng, H, W, 0.3, 0.5, slice_rows=4)
    else:
        lost = np.zeros((H, W), dtype=bool)
        lost[list(lost_rows)] = True
    decoded = cur.copy()
    decoded[lost] = 0
    ref_index = np.arange(index - delta - k + 1, index - delta + 1, dtype=np.int64)
    return _plane(refs, ref_index, cur, decoded, lost, index)
