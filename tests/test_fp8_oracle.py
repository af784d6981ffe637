"""Pins of the E4M3 quantisation oracle (oracle/fp8.py) against torch's
float8_e4m3fn conversions and closed forms of the OCP E4M3 format."""
import numpy as np
import pytest
import torch

from oracle import fp8


def test_decode_all_codes_matches_torch():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = fp8.e4m3_decode(codes)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(got[ok], ref[ok])
    assert np.isnan(got).sum() == 2  # 0x7F and 0xFF


def test_encode_matches_torch_in_range():
    rng = np.random.default_rng(0)
    mags = np.exp2(rng.uniform(-12, np.log2(448.0), 200000))
    x = (mags * rng.choice([-1.0, 1.0], mags.size)).astype(np.float32)
    # exact ties and every representable value
    reps = fp8.e4m3_decode(np.arange(256, dtype=np.uint8))
    reps = reps[np.isfinite(reps)]
    x = np.concatenate([x, reps.astype(np.float32), np.float32([0.0, -0.0])])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = fp8.e4m3_encode(x)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("value,code", [
    (448.0, 0x7E), (500.0, 0x7E), (1e6, 0x7E), (-448.0, 0xFE), (-1e6, 0xFE),
    (2.0 ** -6, 0x08), (2.0 ** -9, 0x01), (2.0 ** -10, 0x00),  # half the smallest subnormal: tie to 0
    (3 * 2.0 ** -10, 0x02),  # 1.5 subnormal steps: tie to the even 2
    (1.0, 0x38), (-1.0, 0xB8), (1.0 + 1 / 16, 0x38), (1.0 + 3 / 16, 0x3A), (1.75 * 2 ** 8, 0x7E),
    (1.0 + 1 / 16 + 1e-6, 0x39)])
def test_encode_closed_forms(value, code):
    assert int(fp8.e4m3_encode(np.float64(value))) == code


def test_quantise_rows_rule():
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (64, 96)).astype(np.float32)
    x[3] = 0
    x[5] *= 1e-4
    q, s = fp8.quantise_rows(x)
    assert s[3] == 1.0 and not q[3].any()
    amax = np.abs(x).max(axis=1)
    nz = amax > 0
    np.testing.assert_array_equal(s[nz], (amax[nz] / np.float32(448)).astype(np.float32))
    # each row's largest magnitude lands on +-448
    big = np.abs(x).argmax(axis=1)
    assert set(int(v) & 0x7F for v in q[np.arange(64)[nz], big[nz]]) == {0x7E}
    deq = fp8.dequantise_rows(q, s)
    # relative error of a normal E4M3 value is at most 2^-4; subnormals: half a 2^-9 step
    err = np.abs(deq - x)
    bound = np.maximum(np.abs(x) * 2.0 ** -4, s[:, None] * 2.0 ** -10) * (1 + 1e-6)
    assert (err <= bound).all()
