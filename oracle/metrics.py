"""Frame-quality metrics the paper evaluates with: SSIM and PSNR (Section 5,
Metrics: SSIM and PSNR of reconstructed against original frames; the depth
loss also carries an SSIM term, Section 3.4.2).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests are the only
callers; the CUDA path never imports it.

The paper cites SSIM and PSNR without parameters; the reading taken is the
original SSIM definition: local statistics under a normalised 11 x 11 Gaussian
window of standard deviation 1.5, K1 = 0.01, K2 = 0.03, C1 = (K1 L)^2,
C2 = (K2 L)^2 with L the data range, the SSIM map over the positions where the
window lies inside the frame ("valid"), averaged; a multi-channel frame
averages its channels' SSIM.  PSNR = 10 log10(L^2 / MSE) with the MSE over every
sample of every channel.  All in float64.

Pinned by tests against direct summation over each window (tiny frames),
closed forms (identical frames, constant frames, a single-sample error) and
symmetry.
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
K1, K2 = 0.01, 0.03


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """Normalised 1-D Gaussian taps; the 2-D window is their outer product."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(x * x) / (2.0 * sigma * sigma))
    return g / g.sum()


def _filter_valid(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable 'valid' correlation of a 2-D array with the window g x g."""
    n = g.size
    H, W = img.shape
    rows = np.zeros((H, W - n + 1))
    for i in range(n):
        rows += g[i] * img[:, i:i + W - n + 1]
    out = np.zeros((H - n + 1, W - n + 1))
    for i in range(n):
        out += g[i] * rows[i:i + H - n + 1, :]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray, data_range: float) -> np.ndarray:
    """SSIM at every valid window position of two single-channel frames."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    g = gaussian_window()
    mx, my = _filter_valid(x, g), _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    c1 = (K1 * data_range) ** 2
    c2 = (K2 * data_range) ** 2
    return ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))


def ssim(x: np.ndarray, y: np.ndarray, data_range: float) -> float:
    """Mean SSIM; [H, W] or [H, W, C] (channels averaged)."""
    x = np.asarray(x)
    y = np.asarray(y)
    if x.ndim == 2:
        return float(ssim_map(x, y, data_range).mean())
    return float(np.mean([ssim_map(x[..., c], y[..., c], data_range).mean() for c in range(x.shape[-1])]))


def mse(x: np.ndarray, y: np.ndarray) -> float:
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    return float(np.mean(d * d))


def psnr(x: np.ndarray, y: np.ndarray, data_range: float) -> float:
    m = mse(x, y)
    return float("inf") if m == 0 else float(10.0 * np.log10(data_range * data_range / m))
