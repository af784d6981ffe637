"""FP8 (E4M3) quantisation as the reduced-precision linear layers use it.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests are the only
callers; the CUDA path never imports it.

The paper runs its model in full precision; the FP8 path is this
repository's reduced-precision variant of the linear layers.  The format is
the OCP 8-bit floating point E4M3: one sign bit, four exponent bits (bias 7),
three mantissa bits; exponent field 0 holds the subnormals m * 2^-9; the
largest finite value is 1.75 * 2^8 = 448 (exponent 15 with mantissa 7 is NaN,
there are no infinities).  Encoding rounds to the nearest representable value,
ties to even mantissa, and saturates magnitudes above 448 to 448.

The scaling rules (per row: the weights' output channels, the activations'
tokens): scale = max|x| / 448, codes = E4M3(x * (448 / max)), both quotients
and the product in float32; an all-zero row keeps scale 1.

Pinned by tests against torch.float8_e4m3fn (all 256 codes decoded, encoding
of in-range values) and by closed forms (448, 2^-6, 2^-9, ties).
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def e4m3_decode(codes: np.ndarray) -> np.ndarray:
    """uint8 codes -> float64 values (NaN for the two NaN codes)."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 0x7).astype(np.float64)
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.exp2(e.astype(np.float64) - 7.0))
    val = np.where((e == 15) & ((c & 7) == 7), np.nan, val)
    return sign * val


def e4m3_encode(x: np.ndarray) -> np.ndarray:
    """float32 (or exactly representable float64) values -> uint8 codes:
    round to nearest, ties to even, saturating to +-448."""
    v = np.asarray(x, dtype=np.float64)
    if np.isnan(v).any():
        raise ValueError("NaN input")
    sign = (v < 0) | ((v == 0) & np.signbit(v))
    a = np.minimum(np.abs(v), E4M3_MAX)
    # binade of a (normal range 2^-6 .. 2^8); below 2^-6 the spacing is 2^-9
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)
    # exact check of the binade (log2 of a float64 may round near powers of 2)
    e = np.where(a < np.exp2(e), e - 1, e)
    e = np.where(a >= np.exp2(e + 1), e + 1, e)
    e = np.clip(e, -6, 8)
    step = np.exp2(e - 3)  # spacing of the representable values in this binade
    q = np.rint(a / step)  # round half to even on the exact quotient
    val = q * step
    val = np.minimum(val, E4M3_MAX)
    # back to fields
    out = np.zeros(v.shape, dtype=np.int64)
    sub = val < 2.0 ** -6
    out = np.where(sub, np.rint(val / 2.0 ** -9).astype(np.int64), out)
    with np.errstate(divide="ignore"):
        en = np.floor(np.log2(np.where(val > 0, val, 1.0)))
    mn = np.rint((val / np.exp2(en) - 1.0) * 8.0).astype(np.int64)
    out = np.where(sub, out, ((en.astype(np.int64) + 7) << 3) | mn)
    out = out | (sign.astype(np.int64) << 7)
    return out.astype(np.uint8)


def quantise_rows(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-row E4M3 codes and scales of a float32 matrix [rows][cols]."""
    x32 = np.asarray(x, dtype=np.float32)
    amax = np.max(np.abs(x32), axis=1)
    scale = np.where(amax > 0, amax / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    with np.errstate(divide="ignore"):
        inv = np.where(amax > 0, np.float32(E4M3_MAX) / np.where(amax > 0, amax, 1), np.float32(1.0))
    inv = inv.astype(np.float32)
    prod = (x32 * inv[:, None]).astype(np.float32)
    return e4m3_encode(prod), scale


def dequantise_rows(codes: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """float64 values codes * scale (per row)."""
    return e4m3_decode(codes) * np.asarray(scale, dtype=np.float64)[:, None]
