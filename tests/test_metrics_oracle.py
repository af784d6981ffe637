"""Pins of the SSIM / PSNR oracle (oracle/metrics.py): direct summation over
every window, closed forms, invariants."""
import numpy as np
import pytest

from oracle import metrics as Mx


def brute_ssim(x, y, L):
    """SSIM straight from its definition: for every window position, the
    Gaussian-weighted means, variances and covariance summed term by term."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    g = Mx.gaussian_window()
    w2 = np.outer(g, g)
    n = g.size
    H, W = x.shape
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for r in range(H - n + 1):
        for c in range(W - n + 1):
            mx = my = sxx = syy = sxy = 0.0
            for i in range(n):
                for j in range(n):
                    a, b, w = x[r + i, c + j], y[r + i, c + j], w2[i, j]
                    mx += w * a
                    my += w * b
            for i in range(n):
                for j in range(n):
                    a, b, w = x[r + i, c + j], y[r + i, c + j], w2[i, j]
                    sxx += w * (a - mx) ** 2
                    syy += w * (b - my) ** 2
                    sxy += w * (a - mx) * (b - my)
            vals.append(((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2)))
    return float(np.mean(vals))


def test_window_is_normalised_gaussian():
    g = Mx.gaussian_window()
    assert g.size == 11 and abs(g.sum() - 1) < 1e-15
    assert np.allclose(g, g[::-1])
    # ratio of neighbouring taps of a Gaussian with sigma 1.5
    assert abs(g[6] / g[5] - np.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


@pytest.mark.parametrize("L", [255.0, 65535.0])
def test_ssim_matches_direct_summation(L):
    rng = np.random.default_rng(3)
    x = rng.integers(0, int(L) + 1, (15, 17)).astype(np.float64)
    y = np.clip(x + rng.normal(0, L / 20, x.shape), 0, L).round()
    assert abs(Mx.ssim(x, y, L) - brute_ssim(x, y, L)) < 1e-12


def test_ssim_closed_forms():
    rng = np.random.default_rng(4)
    x = rng.integers(0, 256, (20, 20)).astype(np.float64)
    assert abs(Mx.ssim(x, x, 255) - 1.0) < 1e-12
    assert abs(Mx.ssim(x, 255 - x, 255) - Mx.ssim(255 - x, x, 255)) < 1e-12  # symmetry
    # constant frames a and b: only the luminance term remains
    a, b, L = 100.0, 140.0, 255.0
    c1 = (0.01 * L) ** 2
    got = Mx.ssim(np.full((12, 12), a), np.full((12, 12), b), L)
    assert abs(got - (2 * a * b + c1) / (a * a + b * b + c1)) < 1e-12
    # channels are averaged
    rgb_x = rng.integers(0, 256, (14, 14, 3)).astype(np.float64)
    rgb_y = rgb_x.copy()
    rgb_y[..., 1] = 0
    per = [Mx.ssim(rgb_x[..., c], rgb_y[..., c], 255) for c in range(3)]
    assert abs(Mx.ssim(rgb_x, rgb_y, 255) - np.mean(per)) < 1e-15


def test_psnr_closed_form():
    x = np.zeros((10, 10), np.uint8)
    y = x.copy()
    y[3, 4] = 10
    # one sample off by 10 in 100: MSE = 1
    assert abs(Mx.psnr(x, y, 255) - 10 * np.log10(255 ** 2)) < 1e-12
    assert Mx.psnr(x, x, 255) == float("inf")
