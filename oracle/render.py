"""RGB-D unprojection and point splatting: the receiver's rendering of a
recovered RGB-D frame (the pipeline's RGB-D rendering step, Section 5 latency
breakdown; volumetric frames are RGB + depth, Section 2).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests are the only
callers; the CUDA path never imports it.

The paper fixes no camera model; the reading taken: a pinhole depth camera
with intrinsics (fx, fy, cx, cy), pixel (i, j) (column, row) at image
coordinates u = i, v = j; a depth sample d (mm, 0 = no measurement) gives the
point x = (u - cx) d / fx, y = (v - cy) d / fy, z = d with the colour of the
RGB pixel (floor(i W_rgb / W), floor(j H_rgb / H)) (nearest sample when the
two frames differ in size).  Rendering: x' = R x + t, projection with the
target intrinsics u' = fx' x' / z' + cx', v' likewise, pixel = round half to
even; points with z' <= 0 are dropped; each point covers the (2s+1) x (2s+1)
pixels around its pixel; per pixel the smallest z' wins, ties to the smaller
point index (points are numbered row-major over the depth frame).  Output:
RGB (0 where nothing lands) and depth round-half-even(z') clamped to
[0, 65535].

Every float decision is taken in float32, one rounded operation at a time, in
the order written above (products and sums of R x + t left to right), so a
float32 implementation that rounds each step the same way agrees bit for bit.
Pinned by tests: the identity pose reproduces the input frame exactly, a pure
translation along z shifts depth by the translation, a rotation by pi about
the optical axis mirrors the frame, and hand-worked occlusion, tie and
resampling cases on tiny frames.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def unproject(depth: np.ndarray, K) -> tuple[np.ndarray, np.ndarray]:
    """Points [N][3] (float32) of the valid depth samples and their flat pixel indices."""
    fx, fy, cx, cy = (f32(v) for v in K)
    H, W = depth.shape
    jj, ii = np.nonzero(depth)
    idx = (jj * W + ii).astype(np.int64)
    order = np.argsort(idx, kind="stable")
    jj, ii, idx = jj[order], ii[order], idx[order]
    d = depth[jj, ii].astype(f32)
    x = ((ii.astype(f32) - cx) * d) / fx
    y = ((jj.astype(f32) - cy) * d) / fy
    return np.stack([x.astype(f32), y.astype(f32), d], axis=1), idx


def render(rgb: np.ndarray, depth: np.ndarray, K_src, R, t, K_dst, out_hw, splat: int = 0):
    """(out_rgb [H'][W'][3] uint8, out_depth [H'][W'] uint16)."""
    H, W = depth.shape
    Hr, Wr = rgb.shape[:2]
    Ho, Wo = out_hw
    P, idx = unproject(depth, K_src)
    R = np.asarray(R, f32).reshape(3, 3)
    t = np.asarray(t, f32)
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    X = ((R[0, 0] * x + R[0, 1] * y).astype(f32) + R[0, 2] * z).astype(f32) + t[0]
    Y = ((R[1, 0] * x + R[1, 1] * y).astype(f32) + R[1, 2] * z).astype(f32) + t[1]
    Z = ((R[2, 0] * x + R[2, 1] * y).astype(f32) + R[2, 2] * z).astype(f32) + t[2]
    X, Y, Z = X.astype(f32), Y.astype(f32), Z.astype(f32)
    fx, fy, cx, cy = (f32(v) for v in K_dst)
    keep = Z > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        u = ((fx * X).astype(f32) / Z).astype(f32) + cx
        v = ((fy * Y).astype(f32) / Z).astype(f32) + cy
    u, v = u.astype(f32), v.astype(f32)
    keep &= np.isfinite(u) & np.isfinite(v) & (np.abs(u) < 1e9) & (np.abs(v) < 1e9)
    pu = np.rint(np.where(keep, u, 0)).astype(np.int64)
    pv = np.rint(np.where(keep, v, 0)).astype(np.int64)
    # Every (point, covered pixel) pair, then per pixel the smallest (z', index).
    pts = np.nonzero(keep)[0]
    cand_pix, cand_z, cand_k = [], [], []
    for dv in range(-splat, splat + 1):
        for du in range(-splat, splat + 1):
            a, b = pv[pts] + dv, pu[pts] + du
            ok = (a >= 0) & (a < Ho) & (b >= 0) & (b < Wo)
            cand_pix.append(a[ok] * Wo + b[ok])
            cand_z.append(Z[pts[ok]].astype(np.float64))
            cand_k.append(pts[ok])
    pix = np.concatenate(cand_pix) if cand_pix else np.zeros(0, np.int64)
    cz = np.concatenate(cand_z) if cand_z else np.zeros(0)
    ck = np.concatenate(cand_k) if cand_k else np.zeros(0, np.int64)
    order = np.lexsort((idx[ck], cz, pix))  # by pixel, then z', then point index
    pix, ck = pix[order], ck[order]
    first = np.ones(pix.size, bool)
    first[1:] = pix[1:] != pix[:-1]
    best_i = np.full(Ho * Wo, -1, np.int64)
    best_i[pix[first]] = ck[first]
    best_i = best_i.reshape(Ho, Wo)
    out_rgb = np.zeros((Ho, Wo, 3), np.uint8)
    out_d = np.zeros((Ho, Wo), np.uint16)
    hit = best_i >= 0
    k = best_i[hit]
    src = idx[k]
    sj, si = src // W, src % W
    rj = (sj * Hr) // H
    ri = (si * Wr) // W
    out_rgb[hit] = rgb[rj, ri]
    out_d[hit] = np.clip(np.rint(Z[k].astype(np.float64)), 0, 65535).astype(np.uint16)
    return out_rgb, out_d
