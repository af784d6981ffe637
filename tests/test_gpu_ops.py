"""Step-level parity of the CUDA kernels (through the C ABI) against the FP64
oracle, element by element, at sizes that span several tiles and a ragged
tail.  bf16 paths are compared with the oracle evaluated on the same
bf16-rounded operands, so the tolerance only has to cover accumulation order
and output rounding."""
import numpy as np
import pytest
import torch

import synth
from oracle import revo_oracle as O

pytestmark = pytest.mark.gpu

R = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global R
    import paper_2604_27441_b300 as mod
    mod.lib()
    R = mod
    yield
    assert R.take_device_error() == 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------------ linear

SHAPES = [(300, 256, 192, 128), (1000, 768, 768, 256), (517, 384, 128, 256), (5120, 1152, 1536, 128),
          (3600, 2304, 768, 0), (1, 64, 64, 128), (129, 3072, 768, 256)]


@pytest.mark.parametrize("M,N,K,bn", SHAPES)
@pytest.mark.parametrize("epi", [0, 1, 2, 3])
def test_linear_bf16_tcgen05(M, N, K, bn, epi):
    seed = M * 7 + N + K
    A = bf16(synth.normal(seed, (M, K)))
    W = bf16(synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K)))
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(f64(A), f64(W), b.astype(np.float64))
    if epi == 2:
        ref = O.gelu(ref)
    out_dtype = torch.float32 if epi in (0, 3) else torch.bfloat16
    base = synth.normal(seed + 3, (M, N)) if epi == 3 else np.zeros((M, N), np.float32)
    out = torch.from_numpy(base).to(out_dtype).cuda()
    R.op_linear(R.BF16, epi, A.cuda(), W.cuda(), dev(b), out, M, N, K, bn)
    torch.cuda.synchronize()
    got = f64(out)
    if epi == 3:
        ref = ref + base
    if out_dtype == torch.float32:
        np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-4)
    else:
        np.testing.assert_allclose(got, ref, rtol=8e-3, atol=8e-3)


PAIR_SHAPES = [(300, 256, 192), (1000, 768, 768), (517, 384, 128), (3600, 3072, 768), (1, 64, 64), (129, 2304, 768),
               (256, 512, 256), (5000, 1536, 384)]


@pytest.mark.parametrize("M,N,K", PAIR_SHAPES)
@pytest.mark.parametrize("epi", [0, 1, 2, 3])
def test_linear_bf16_cta_pair_tiles(M, N, K, epi):
    """256-row tiles on a CTA pair (tcgen05.mma.cta_group::2): the oracle's
    values, and bit for bit the single-CTA tile of the same width (same
    float32 dot products, same K order, same epilogue)."""
    seed = M * 3 + N * 5 + K
    A = bf16(synth.normal(seed, (M, K))).cuda()
    W = bf16(synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K))).cuda()
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(f64(A), f64(W), b.astype(np.float64))
    if epi == 2:
        ref = O.gelu(ref)
    out_dtype = torch.float32 if epi in (0, 3) else torch.bfloat16
    base = synth.normal(seed + 3, (M, N)) if epi == 3 else np.zeros((M, N), np.float32)
    if epi == 3:
        ref = ref + base
    for width in (128, 256):
        if width > N:
            continue
        outs = []
        for tile in (width, width | R.TILE_PAIR):
            out = torch.from_numpy(base).to(out_dtype).cuda()
            R.op_linear(R.BF16, epi, A, W, dev(b), out, M, N, K, tile)
            torch.cuda.synchronize()
            outs.append(out)
        got = f64(outs[1])
        if out_dtype == torch.float32:
            np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-4)
        else:
            np.testing.assert_allclose(got, ref, rtol=8e-3, atol=8e-3)
        assert torch.equal(outs[0], outs[1]), f"width {width}: pair tile differs from the single tile"
    assert R.take_device_error() == 0


# 192-wide tiles (float32 epilogues): N = 768 and 384 split evenly, 320 and
# 224 leave a ragged last tile (N % 192 != 0), M spans several row tiles and a
# ragged tail; (3600, 768, 3072) is fc2 of an encoder block.
@pytest.mark.gpu
@pytest.mark.parametrize("M,N,K", [(300, 768, 192), (3600, 768, 3072), (517, 384, 128), (129, 320, 256),
                                   (1, 224, 64)])
@pytest.mark.parametrize("epi", [0, 3])
def test_linear_bf16_192_wide_tiles(M, N, K, epi):
    """The 192-column tile: the oracle's values, and bit for bit the 128- and
    256-column tiles (same float32 dot products in the same K order)."""
    seed = M * 7 + N * 3 + K
    A = bf16(synth.normal(seed, (M, K))).cuda()
    W = bf16(synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K))).cuda()
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(f64(A), f64(W), b.astype(np.float64))
    base = synth.normal(seed + 3, (M, N)) if epi == 3 else np.zeros((M, N), np.float32)
    if epi == 3:
        ref = ref + base
    outs = {}
    for tile in (192, 128, 256):
        if tile > N:
            continue
        out = torch.from_numpy(base).cuda()
        R.op_linear(R.BF16, epi, A, W, dev(b), out, M, N, K, tile)
        torch.cuda.synchronize()
        outs[tile] = out
    np.testing.assert_allclose(f64(outs[192]), ref, rtol=1e-4, atol=2e-4)
    for tile, out in outs.items():
        assert torch.equal(out, outs[192]), f"192-wide tile differs from the {tile}-wide tile"
    assert R.take_device_error() == 0


@pytest.mark.parametrize("M,N,K", [(300, 256, 192), (1000, 768, 768), (77, 96, 24)])
@pytest.mark.parametrize("epi", [0, 2, 3])
def test_linear_fp32_simt(M, N, K, epi):
    seed = M + N * 3 + K
    A = synth.normal(seed, (M, K))
    W = synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K))
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(A.astype(np.float64), W.astype(np.float64), b.astype(np.float64))
    if epi == 2:
        ref = O.gelu(ref)
    base = synth.normal(seed + 3, (M, N)) if epi == 3 else np.zeros((M, N), np.float32)
    out = dev(base)
    R.op_linear(R.FP32, epi, dev(A), dev(W), dev(b), out, M, N, K)
    torch.cuda.synchronize()
    if epi == 3:
        ref = ref + base
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5, atol=2e-5)


# --------------------------------------------------------------- layernorm

@pytest.mark.parametrize("M,D", [(333, 768), (1000, 384), (1, 192)])
@pytest.mark.parametrize("out_bf16", [0, 1])
def test_layernorm(M, D, out_bf16):
    x = synth.normal(M + D, (M, D), 3.0) + 0.5
    g = 1 + synth.normal(M + D + 1, (D,), 0.1)
    b = synth.normal(M + D + 2, (D,), 0.1)
    out = torch.zeros((M, D), dtype=torch.bfloat16 if out_bf16 else torch.float32, device="cuda")
    R.op_layernorm(dev(x), dev(g), dev(b), out, M, D, out_bf16)
    torch.cuda.synchronize()
    ref = O.layer_norm(x.astype(np.float64), g.astype(np.float64), b.astype(np.float64))
    if out_bf16:
        np.testing.assert_allclose(f64(out), ref, rtol=8e-3, atol=8e-3)
    else:
        np.testing.assert_allclose(f64(out), ref, rtol=0, atol=5e-5)


# --------------------------------------------------------------------- fp8

from oracle import fp8 as F8  # noqa: E402


@pytest.mark.parametrize("rows,cols", [(300, 768), (1, 384), (1000, 3072), (77, 128)])
def test_quantize_rows_e4m3_bit_exact(rows, cols):
    """Codes and scales equal the oracle's on the same float32 input: the
    scale and the scaled value are float32 operations on both sides, the
    rounding to E4M3 is the format's."""
    x = synth.normal(rows + cols, (rows, cols), 2.0)
    x[rows // 2] = 0.0
    x[-1, :7] = [1e-7, -3e-6, 5e3, -5e3, 0.0, 1.0, 448.0]
    q = torch.zeros((rows, cols), dtype=torch.uint8, device="cuda")
    sc = torch.zeros(rows, dtype=torch.float32, device="cuda")
    R.op_quantize_rows_e4m3(dev(x), rows, cols, q, sc)
    torch.cuda.synchronize()
    q_ref, s_ref = F8.quantise_rows(x)
    np.testing.assert_array_equal(sc.cpu().numpy(), s_ref)
    np.testing.assert_array_equal(q.cpu().numpy(), q_ref)


@pytest.mark.parametrize("M,D", [(333, 768), (1000, 384), (1, 128)])
def test_layernorm_e4m3(M, D):
    """Dequantised codes are within one E4M3 rounding (2^-4 relative, or half a
    subnormal step) of the FP64 LayerNorm, plus the float32 LN error."""
    x = synth.normal(M + D, (M, D), 3.0) + 0.5
    g = 1 + synth.normal(M + D + 1, (D,), 0.1)
    b = synth.normal(M + D + 2, (D,), 0.1)
    q = torch.zeros((M, D), dtype=torch.uint8, device="cuda")
    sc = torch.zeros(M, dtype=torch.float32, device="cuda")
    R.op_layernorm_e4m3(dev(x), dev(g), dev(b), q, sc, M, D)
    torch.cuda.synchronize()
    ref = O.layer_norm(x.astype(np.float64), g.astype(np.float64), b.astype(np.float64))
    s = sc.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(s, np.abs(ref).max(axis=1) / 448.0, rtol=1e-5)
    deq = F8.dequantise_rows(q.cpu().numpy(), s)
    bound = np.maximum(np.abs(ref) * 2.0 ** -4, s[:, None] * 2.0 ** -10) * (1 + 1e-3) + 5e-5
    assert (np.abs(deq - ref) <= bound).all()


# ------------------------------------------- residual Linear + LayerNorm

@pytest.mark.parametrize("M,N,K", [(1, 384, 384), (127, 768, 768), (300, 384, 1536), (1000, 768, 3072),
                                   (4100, 768, 768), (1300, 320, 256)])
@pytest.mark.parametrize("tile", [128, 256, 128 | 0x1000, 256 | 0x1000])
@pytest.mark.parametrize("fp8", [False, True])
def test_linear_resid_ln_equals_separate_launches(M, N, K, tile, fp8):
    """The LayerNorm fused into the residual GEMM's epilogue (the CTA that adds
    a row block's last column tile normalises the block) gives exactly what
    the residual Linear then the standalone LayerNorm give: the same x, bit for
    bit, and the same bf16 values or E4M3 codes and scales; and x and the
    LayerNorm agree with the oracle (x + A W^T + b, then LN; eps 1e-6)."""
    if (tile & 0xFFF) == 256 and N < 256:
        tile = (tile & 0x1000) | 128
    A = bf16(synth.normal(M + N, (M, K), 1.0))
    W = bf16(synth.normal(M + N + 1, (N, K), 1.0 / np.sqrt(K)))
    b = synth.normal(M + N + 2, (N,), 0.1)
    x0 = synth.normal(M + N + 3, (M, N), 2.0) + 0.25
    g = 1 + synth.normal(M + N + 4, (N,), 0.1)
    beta = synth.normal(M + N + 5, (N,), 0.1)
    Ad, Wd, bd, gd, betad = A.cuda(), W.cuda(), dev(b), dev(g), dev(beta)
    x_sep, x_fused = dev(x0), dev(x0)
    if fp8:
        h_sep = torch.zeros((M, N), dtype=torch.uint8, device="cuda")
        h_fused = torch.full((M, N), 0x7F, dtype=torch.uint8, device="cuda")
        s_sep = torch.zeros(M, dtype=torch.float32, device="cuda")
        s_fused = torch.full((M,), -1.0, dtype=torch.float32, device="cuda")
    else:
        h_sep = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
        h_fused = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
        s_sep = s_fused = None
    R.op_linear(R.BF16, 3, Ad, Wd, bd, x_sep, M, N, K, tile)
    if fp8:
        R.op_layernorm_e4m3(x_sep, gd, betad, h_sep, s_sep, M, N)
    else:
        R.op_layernorm(x_sep, gd, betad, h_sep, M, N, 1)
    R.op_linear_resid_ln(Ad, Wd, bd, x_fused, M, N, K, gd, betad, h_fused, s_fused, fp8, tile)
    # A second call on the same buffers: the row-block counters start from zero again.
    x_again, h_again = dev(x0), torch.empty_like(h_fused)
    s_again = torch.empty_like(s_fused) if fp8 else None
    R.op_linear_resid_ln(Ad, Wd, bd, x_again, M, N, K, gd, betad, h_again, s_again, fp8, tile)
    torch.cuda.synchronize()
    assert torch.equal(x_fused, x_sep) and torch.equal(x_again, x_sep)
    assert torch.equal(h_fused.view(torch.uint8) if not fp8 else h_fused,
                       h_sep.view(torch.uint8) if not fp8 else h_sep)
    assert torch.equal(h_again.view(torch.uint8) if not fp8 else h_again,
                       h_sep.view(torch.uint8) if not fp8 else h_sep)
    if fp8:
        assert torch.equal(s_fused, s_sep) and torch.equal(s_again, s_sep)
    x_ref = x0.astype(np.float64) + O.linear(f64(A), f64(W), b.astype(np.float64))
    np.testing.assert_allclose(f64(x_fused), x_ref, rtol=1e-5, atol=2e-4)
    ln_ref = O.layer_norm(x_ref, g.astype(np.float64), beta.astype(np.float64))
    if fp8:
        s = s_fused.cpu().numpy().astype(np.float64)
        deq = F8.dequantise_rows(h_fused.cpu().numpy(), s)
        bound = np.maximum(np.abs(ln_ref) * 2.0 ** -4, s[:, None] * 2.0 ** -10) * (1 + 1e-3) + 2e-4
        assert (np.abs(deq - ln_ref) <= bound).all()
    else:
        np.testing.assert_allclose(f64(h_fused), ln_ref, rtol=8e-3, atol=8e-3)


@pytest.mark.parametrize("M,N,K,bn", [(300, 256, 768, 128), (1000, 2304, 768, 256), (517, 1536, 384, 256),
                                      (3600, 3072, 768, 0), (1, 64, 128, 128), (129, 384, 384, 128)])
@pytest.mark.parametrize("epi", [1, 2])
def test_linear_fp8_tcgen05(M, N, K, bn, epi):
    """E4M3 operands decode exactly, so the oracle multiplies the decoded
    values (times the row and channel scales) in float64; the tolerance
    covers float32 accumulation and the bf16 output rounding."""
    seed = M * 5 + N + K
    a_codes, a_scale = F8.quantise_rows(synth.normal(seed, (M, K), 1.5))
    w_codes, w_scale = F8.quantise_rows(synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K)))
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(F8.dequantise_rows(a_codes, a_scale), F8.dequantise_rows(w_codes, w_scale), b.astype(np.float64))
    if epi == 2:
        ref = O.gelu(ref)
    out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    R.op_linear_fp8(epi, dev(a_codes), dev(a_scale), dev(w_codes), dev(w_scale), dev(b), out, M, N, K, bn)
    torch.cuda.synchronize()
    np.testing.assert_allclose(f64(out), ref, rtol=8e-3, atol=8e-3)


@pytest.mark.parametrize("M,N,K", [(300, 256, 768), (1000, 2304, 768), (3600, 3072, 768), (1, 64, 128),
                                   (517, 1536, 384)])
@pytest.mark.parametrize("epi", [1, 2])
def test_linear_fp8_cta_pair_tiles(M, N, K, epi):
    """E4M3 pair tiles: the oracle's values and the single tile's bits."""
    seed = M * 11 + N + K
    a_codes, a_scale = F8.quantise_rows(synth.normal(seed, (M, K), 1.5))
    w_codes, w_scale = F8.quantise_rows(synth.normal(seed + 1, (N, K), 1.0 / np.sqrt(K)))
    b = synth.normal(seed + 2, (N,), 0.1)
    ref = O.linear(F8.dequantise_rows(a_codes, a_scale), F8.dequantise_rows(w_codes, w_scale), b.astype(np.float64))
    if epi == 2:
        ref = O.gelu(ref)
    args = [dev(a_codes), dev(a_scale), dev(w_codes), dev(w_scale), dev(b)]
    for width in (128, 256):
        if width > N:
            continue
        outs = []
        for tile in (width, width | R.TILE_PAIR):
            out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
            R.op_linear_fp8(epi, *args[:5], out, M, N, K, tile)
            torch.cuda.synchronize()
            outs.append(out)
        np.testing.assert_allclose(f64(outs[1]), ref, rtol=8e-3, atol=8e-3)
        assert torch.equal(outs[0], outs[1])
    assert R.take_device_error() == 0


# --------------------------------------------------------------- attention

def _oracle_segments(qkv, heads, seg):
    out = np.zeros((qkv.shape[0], qkv.shape[1] // 3))
    for a, b in zip(seg[:-1], seg[1:]):
        if b > a:
            out[a:b] = O.attention(qkv[a:b], heads)
    return out


ATT_CASES = [((0, 300, 1000), 2), ((0, 5, 5, 133, 900), 3), ((0, 3600), 12), ((0, 128, 256), 1),
             ((0, 900, 1800, 2700), 6)]


_ATT_ORACLE = {}


def check_attention_bf16(got, qkv64, heads, seg, cache_key=None):
    """Checks a bf16 attention output against the FP64 oracle on the same
    bf16-rounded q, k, v, with tolerances derived from the kernel's roundings:
    P = exp(...) rounded to bf16 before the PV product (relative error <= 2^-8
    per weight, so |error| <= 2^-8 sum_j a_ij |v_j| with a = softmax), and the
    output rounded to bf16 (<= 2^-8 |O|); plus 2^-12 sum_j a_ij |v_j| for the
    float32 accumulations.  Element by element within that bound, and over the
    whole output and each long segment a relative RMS error below 4e-3 (the
    roundings give ~2e-3; one dropped 128-key tile at N = 3600 gives ~0.2, a 10%
    error in the softmax scale ~0.1)."""
    D = qkv64.shape[1] // 3
    if cache_key is None or cache_key not in _ATT_ORACLE:
        absv = qkv64.copy()
        absv[:, 2 * D:] = np.abs(absv[:, 2 * D:])
        ref_av = (_oracle_segments(qkv64, heads, seg), _oracle_segments(absv, heads, seg))
        if cache_key is not None:
            _ATT_ORACLE[cache_key] = ref_av
    else:
        ref_av = _ATT_ORACLE[cache_key]
    ref, av = ref_av
    bound = 2.0 ** -8 * av + 2.0 ** -8 * np.abs(ref) + 2.0 ** -12 * av + 1e-6
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float(err[bad].max()), float(bound[bad].min()))

    def rel_rms(a, b):
        return float(np.sqrt(np.mean((a - b) ** 2)) / max(np.sqrt(np.mean(b ** 2)), 1e-30))
    assert rel_rms(got, ref) < 4e-3, rel_rms(got, ref)
    for a, b in zip(seg[:-1], seg[1:]):
        if b - a >= 64:
            assert rel_rms(got[a:b], ref[a:b]) < 4e-3, (a, b, rel_rms(got[a:b], ref[a:b]))


@pytest.mark.parametrize("split_tail", [False, True])
@pytest.mark.parametrize("seg,heads", ATT_CASES + [((0, 900), 12), ((0, 10800), 2), ((0, 129, 385, 3600), 12),
                                                   ((0, 4320, 5600, 5856), 4)])
def test_attention_bf16_tcgen05(seg, heads, split_tail):
    """One CTA per (head, 256 queries) unit; with split_tail the units of a
    segment's last, partly filled wave are cut into key ranges merged by a
    second kernel.  The cases cover every unit cut (N = 900, 48
    units), whole waves plus a cut tail (N = 3600: 148 whole + 32 cut in 4),
    nothing cut (N = 10800 with 2 heads), units whose second query tile is
    empty (lengths 129, 256 + 16, ...) and segments of mixed lengths in one
    launch."""
    M, D = seg[-1], 64 * heads
    qkv = bf16(synth.normal(M + heads, (M, 3 * D)))
    out = torch.zeros((M, D), dtype=torch.bfloat16, device="cuda")
    R.op_attention(R.BF16, qkv.cuda(), out, M, D, heads, seg, split_tail=split_tail)
    torch.cuda.synchronize()
    check_attention_bf16(f64(out), f64(qkv), heads, seg, cache_key=(tuple(seg), heads))
    assert R.take_device_error() == 0


@pytest.mark.parametrize("seg,queries,heads", [((0, 3600), [(2400, 3600)], 6), ((0, 900, 1800), [(600, 900), (1500, 1800)], 6),
                                               ((0, 300, 1000), [(0, 17), (700, 1000)], 2)])
def test_attention_bf16_query_rows(seg, queries, heads):
    """Queries restricted to some rows of each segment (the last decoder block
    keeps the final slot's rows only): those rows equal the oracle's full
    attention there; every other output row is left untouched."""
    M, D = seg[-1], 64 * heads
    qkv = bf16(synth.normal(M + 3 * heads, (M, 3 * D)))
    out = torch.full((M, D), 7.0, dtype=torch.bfloat16, device="cuda")
    R.op_attention(R.BF16, qkv.cuda(), out, M, D, heads, seg, queries=queries)
    torch.cuda.synchronize()
    got = f64(out)
    rows = np.zeros(M, bool)
    for a, b in queries:
        rows[a:b] = True
    assert (got[~rows] == 7.0).all()
    full = got.copy()
    ref = _oracle_segments(f64(qkv), heads, seg)
    full[~rows] = ref[~rows]   # rows outside the queries compared as exact
    check_attention_bf16(full, f64(qkv), heads, seg)
    assert R.take_device_error() == 0


@pytest.mark.parametrize("split_tail", [False, True])
def test_attention_segment_alone_equals_in_a_batch(split_tail):
    """A segment's work split depends on its length only: its output inside a
    launch with other segments is bit for bit its output alone (with and
    without the tail cut)."""
    heads, D = 12, 768
    lens = (3600, 900, 10800, 4320)
    seg = np.concatenate([[0], np.cumsum(lens)]).tolist()
    M = seg[-1]
    qkv = bf16(synth.normal(77, (M, 3 * D))).cuda()
    out = torch.zeros((M, D), dtype=torch.bfloat16, device="cuda")
    R.op_attention(R.BF16, qkv, out, M, D, heads, seg, split_tail=split_tail)
    for a, b in zip(seg[:-1], seg[1:]):
        alone = torch.zeros((b - a, D), dtype=torch.bfloat16, device="cuda")
        R.op_attention(R.BF16, qkv[a:b].contiguous(), alone, b - a, D, heads, [0, b - a], split_tail=split_tail)
        torch.cuda.synchronize()
        assert torch.equal(alone, out[a:b]), (a, b)
    assert R.take_device_error() == 0


def _reference_ladder_qkv(M, heads, seed):
    """q, k, v (bf16 values) whose scores climb in steps the kernel's softmax
    must follow by moving its reference.  Head 0: query rows r % 3 == 0 have
    q[0] = 16, rows r % 3 == 1 have q[0] = 8 (lanes of one warp differ), the
    others 0; key dimension 0 is 0 except at a few keys, so with the scale
    log2(e)/8 a row with q[0] = 16 sees scores (log2 units) of about 69 at key
    50 (block 0, keys 32..63 of the block: above the first 32 keys' maximum by
    far more than 57), 138.5 at key 140 (block 1, keys 0..31), 207.7 at key 300
    (block 2, keys 32..63), 271.2 at key 420 (block 3, keys 32..63: 63 above,
    kept as is), then 277 and 268 at keys 460 and 455 (block 3, keys 64..127:
    the reference moves while keys 32..63's P is already in TMEM, and key 420
    keeps a 2^-6 share).  Values of the ladder keys are distinct."""
    D = 64 * heads
    a = synth.normal(seed, (M, 3 * D)).astype(np.float32)
    a[:, 0] = np.where(np.arange(M) % 3 == 0, 16.0, np.where(np.arange(M) % 3 == 1, 8.0, 0.0))
    a[:, D] = 0.0
    for key, b, vv in ((50, 24.0, 3.0), (140, 48.0, -2.0), (300, 72.0, 1.5), (420, 94.0, -3.0), (455, 93.0, 2.5),
                       (460, 96.0, 4.0)):
        if key < M:
            a[key, D] = b
            a[key, 2 * D:2 * D + 64] = vv
    return bf16(a)


@pytest.mark.parametrize("split_tail", [False, True])
@pytest.mark.parametrize("seg,heads", [((0, 1000), 2), ((0, 600, 1600), 2), ((0, 3600), 12)])
def test_attention_bf16_reference_moves(seg, heads, split_tail):
    """Scores that climb by more than 57 (log2 units) past a row's reference,
    in each group of keys of a block and in the first block: the kernel moves
    the reference, scales what it holds by an exact power of two, and the
    output stays within the bf16-derived bound of the FP64 oracle (also with
    the tail cut, whose parts start mid-segment)."""
    M, D = seg[-1], 64 * heads
    qkv = _reference_ladder_qkv(M, heads, 91 + M)
    out = torch.zeros((M, D), dtype=torch.bfloat16, device="cuda")
    R.op_attention(R.BF16, qkv.cuda(), out, M, D, heads, seg, split_tail=split_tail)
    torch.cuda.synchronize()
    got = f64(out)
    assert np.isfinite(got).all()
    check_attention_bf16(got, f64(qkv), heads, seg)
    assert R.take_device_error() == 0


@pytest.mark.parametrize("seg,heads", ATT_CASES[:2] + [((0, 700), 4)])
def test_attention_fp32_simt(seg, heads):
    M, D = seg[-1], 64 * heads
    qkv = synth.normal(M * 3 + heads, (M, 3 * D))
    out = torch.zeros((M, D), dtype=torch.float32, device="cuda")
    R.op_attention(R.FP32, dev(qkv), out, M, D, heads, seg)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), _oracle_segments(qkv.astype(np.float64), heads, seg),
                               rtol=0, atol=2e-5)


# --------------------------------------------------- assemble / statistics

@pytest.mark.parametrize("modality,k", [("rgb", 5), ("depth", 5), ("rgb", 1), ("depth", 3)])
@pytest.mark.parametrize("out_bf16", [0, 1])
def test_assemble(modality, k, out_bf16):
    H, W, T, p = 48, 80, 2, 16
    pl = synth.make_tiny_plane(k * 11 + len(modality), modality, H, W, k)
    C = 3 if modality == "rgb" else 1
    if modality == "rgb":
        frames = np.stack([O.normalise_rgb(f) for f in pl.refs] + [O.normalise_rgb(pl.decoded)])
        mu_sigma = None
        pitch = W * 3
    else:
        mu, sg = O.depth_stats(pl.refs[-1])
        frames = np.stack([O.normalise_depth(f, mu, sg) for f in pl.refs] + [O.normalise_depth(pl.decoded, mu, sg)])
        mu_sigma = dev(np.array([mu, sg], np.float32))
        pitch = W * 2
    ref = O.tubelets(frames, T, p)
    refs_d = [dev(f) for f in pl.refs]
    out = torch.zeros(ref.shape, dtype=torch.bfloat16 if out_bf16 else torch.float32, device="cuda")
    R.op_assemble(C, k, T, p, H, W, refs_d, dev(pl.decoded), pitch, mu_sigma, out, out_bf16)
    torch.cuda.synchronize()
    if out_bf16:
        np.testing.assert_allclose(f64(out), ref, rtol=8e-3, atol=1e-6)
    else:
        np.testing.assert_allclose(f64(out), ref, rtol=2e-6, atol=2e-6)


def pitched(frame, pad, offset):
    """A frame copied into rows of len(row) + pad bytes, starting `offset` bytes
    into a device buffer (rows and base then lack 8/16-byte alignment)."""
    rows = np.ascontiguousarray(frame).view(np.uint8).reshape(frame.shape[0], -1)
    H, rb = rows.shape
    pitch = rb + pad
    buf = np.zeros(offset + H * pitch + 16, np.uint8)
    for y in range(H):
        buf[offset + y * pitch: offset + y * pitch + rb] = rows[y]
    t = dev(buf)
    return t[offset:], pitch


@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_assemble_unaligned_rows(modality):
    """Frames whose rows are not 8/16-byte aligned take the kernel's scalar
    loads; the tokens are the same as from aligned frames."""
    H, W, T, p, k = 48, 80, 2, 16, 3
    pl = synth.make_tiny_plane(77 + len(modality), modality, H, W, k)
    C = 3 if modality == "rgb" else 1
    if modality == "rgb":
        frames = np.stack([O.normalise_rgb(f) for f in pl.refs] + [O.normalise_rgb(pl.decoded)])
        mu_sigma = None
    else:
        mu, sg = O.depth_stats(pl.refs[-1])
        frames = np.stack([O.normalise_depth(f, mu, sg) for f in pl.refs] + [O.normalise_depth(pl.decoded, mu, sg)])
        mu_sigma = dev(np.array([mu, sg], np.float32))
    ref = O.tubelets(frames, T, p)
    offset = 4 if modality == "rgb" else 2
    pad = 4 if modality == "rgb" else 6
    refs_d, pitch = zip(*[pitched(f, pad, offset) for f in pl.refs])
    cur_d, pitch_c = pitched(pl.decoded, pad, offset)
    assert len(set(pitch)) == 1 and pitch[0] == pitch_c
    out = torch.zeros(ref.shape, dtype=torch.float32, device="cuda")
    R.op_assemble(C, k, T, p, H, W, list(refs_d), cur_d, pitch_c, mu_sigma, out, 0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(f64(out), ref, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_blend_unaligned_rows(modality):
    """Decoded / output rows and the head not 16-byte aligned: scalar paths,
    same bit-exact codes."""
    H, W, p = 32, 48, 16
    C = 3 if modality == "rgb" else 1
    pl = synth.make_tiny_plane(H * W + 5, modality, H, W, 1)
    Hp, Wp = H // p, W // p
    head = synth.normal(H + W, (Hp * Wp, C * p * p), 1.5 if modality == "rgb" else 0.8)
    y = O.untubelet_frame(head.astype(np.float64), C, 1, p, Hp, Wp, 0).astype(np.float32)
    if modality == "rgb":
        codes = O.quantise_rgb(O.denormalise_rgb(y, np.float32), np.float32)
        ms = None
    else:
        mu, sg = 2500.0, 700.0
        codes = O.quantise_depth(O.denormalise_depth(y, mu, sg, np.float32), np.float32)
        ms = dev(np.array([mu, sg], np.float32))
    expect = O.blend(pl.decoded, O.unpack_mask(pl.mask, W), codes)
    offset = 4 if modality == "rgb" else 2
    dec_d, pitch = pitched(pl.decoded, 4, offset)
    out_d, _ = pitched(np.zeros_like(pl.decoded), 4, offset)
    head_buf = dev(np.concatenate([np.zeros(1, np.float32), head.ravel()]))[1:]  # 4 bytes past a 16-byte boundary
    R.op_blend(C, p, H, W, head_buf, dec_d, pitch, dev(pl.mask), pl.mask.shape[1], ms, out_d, pitch)
    torch.cuda.synchronize()
    rows = out_d.cpu().numpy()[: H * pitch].reshape(H, pitch)[:, : W * (3 if modality == "rgb" else 2)]
    got = rows.copy().view(np.uint8 if modality == "rgb" else np.uint16).reshape(pl.decoded.shape)
    np.testing.assert_array_equal(got, expect)


@pytest.mark.parametrize("case", ["synthetic", "zeros", "constant", "two_values"])
def test_depth_stats(case):
    if case == "synthetic":
        _, dep = synth.make_request(3003, "1280x720+640x576")
        d = dep.refs[-1]
    elif case == "zeros":
        d = np.zeros((480, 640), np.uint16)
    elif case == "constant":
        d = np.full((240, 320), 1234, np.uint16)
        d[::7, ::5] = 0
    else:
        d = np.zeros((16, 64), np.uint16)
        d[:, ::2] = 1000
        d[:, 1::4] = 3000
    H, W = d.shape
    ms = torch.zeros(2, dtype=torch.float32, device="cuda")
    scratch = torch.zeros(R.depth_stats_scratch_bytes(), dtype=torch.uint8, device="cuda")
    for _ in range(2):   # the scratch is reused: the second call must give the same answer
        R.op_depth_stats(dev(d), H, W, W * 2, ms, scratch)
        torch.cuda.synchronize()
        mu, sg = O.depth_stats(d)
        got = ms.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, [mu, sg], rtol=2e-6, atol=0)


@pytest.mark.parametrize("D,hp,wp,taus", [(768, 15, 20, (5, 3, 1)), (384, 45, 80, (7, 5, 3)), (192, 2, 3, (1,)),
                                         (192, 2, 300, (4, 2)), (192, 260, 3, (1,))])
def test_position_embedding(D, hp, wp, taus):
    """Up to 256 patch rows and columns the row and column parts come from a
    table, larger grids compute them per element; both against the oracle
    (grids whose slot size is not a multiple of the kernel's 8-token runs
    included)."""
    S = len(taus)
    x = torch.zeros((S * hp * wp, D), dtype=torch.float32, device="cuda")
    R.op_add_position(x, S, hp, wp, D, list(taus))
    torch.cuda.synchronize()
    np.testing.assert_allclose(x.cpu().numpy(), O.position_embedding(list(taus), hp, wp, D), rtol=0, atol=2e-5)


@pytest.mark.parametrize("D,K,hp,wp,taus", [(768, 1536, 15, 20, (5, 3, 1)), (384, 768, 45, 80, (7, 5, 3)),
                                           (192, 64, 2, 3, (0,)), (192, 128, 2, 300, (4, 2)),
                                           (384, 256, 3, 5, (1000, 64, 63)), (768, 768, 1, 129, (70000,))])
@pytest.mark.parametrize("tile", [128, 192, 256, 128 | 0x1000, 256 | 0x1000])
def test_linear_with_position_embedding_equals_separate_launches(D, K, hp, wp, taus, tile):
    """The position embedding added in the embedding GEMM's epilogue (table
    values below 256, per-element sincosf beyond: a 300-column grid, temporal
    distances 1000 and 70000) gives the same floats as the Linear then
    op_add_position, bit for bit, and the sum agrees with the oracle."""
    S = len(taus)
    M = S * hp * wp
    A = bf16(synth.normal(M + D, (M, K), 1.0))
    W = bf16(synth.normal(M + D + 1, (D, K), 1.0 / np.sqrt(K)))
    b = synth.normal(M + D + 2, (D,), 0.1)
    Ad, Wd, bd = A.cuda(), W.cuda(), dev(b)
    sep = torch.empty((M, D), dtype=torch.float32, device="cuda")
    fused = torch.full((M, D), float("nan"), dtype=torch.float32, device="cuda")
    R.op_linear(R.BF16, 0, Ad, Wd, bd, sep, M, D, K, tile)
    R.op_add_position(sep, S, hp, wp, D, list(taus))
    R.op_linear_pe(Ad, Wd, bd, fused, S, hp, wp, D, K, list(taus), tile)
    torch.cuda.synchronize()
    assert torch.equal(fused.view(torch.int32), sep.view(torch.int32))
    ref = O.linear(f64(A), f64(W), b.astype(np.float64)) + O.position_embedding(list(taus), hp, wp, D)
    # float32 pos * w_i is off by up to pos * 2^-24 (relative), and sin / cos
    # have slope <= 1: the embedding's own error grows with the position.
    np.testing.assert_allclose(f64(fused), ref, rtol=1e-5, atol=1e-4 + max(max(taus), hp, wp) * 2.0 ** -23)


# -------------------------------------------------------------------- blend

@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_batched_assemble_and_blend_equal_single_launches(modality):
    """One launch for several requests of different sizes (the forward's form)
    gives bit for bit what one launch per request gives."""
    C, k, T, p = (3, 5, 2, 16) if modality == "rgb" else (1, 5, 2, 16)
    sizes = [(48, 80), (32, 128), (64, 64)]
    assemble_jobs, blend_jobs, singles = [], [], []
    for i, (H, W) in enumerate(sizes):
        pl = synth.make_tiny_plane(500 + i, modality, H, W, k)
        pitch = W * (3 if C == 3 else 2)
        refs = [dev(f) for f in pl.refs]
        cur = dev(pl.decoded)
        ms = dev(np.array([1800.0 + i, 600.0], np.float32)) if C == 1 else None
        S, Hp, Wp = (k + 1) // T, H // p, W // p
        tok_b = torch.zeros((S * Hp * Wp, T * C * p * p), dtype=torch.bfloat16, device="cuda")
        tok_s = torch.zeros_like(tok_b)
        R.op_assemble(C, k, T, p, H, W, refs, cur, pitch, ms, tok_s, 1)
        assemble_jobs.append(dict(height=H, width=W, frames=refs + [cur], pitch_bytes=pitch, mu_sigma=ms, out=tok_b))
        head = dev(synth.normal(900 + i, (Hp * Wp, C * p * p)))
        mask = dev(pl.mask)
        shape = pl.decoded.shape
        odt = torch.uint8 if C == 3 else torch.int16
        out_b, out_s = torch.zeros(shape, dtype=odt, device="cuda"), torch.zeros(shape, dtype=odt, device="cuda")
        val_b = torch.zeros(shape, dtype=torch.float32, device="cuda")
        val_s = torch.zeros_like(val_b)
        R.op_blend(C, p, H, W, head, cur, pitch, mask, pl.mask.shape[1], ms, out_s, pitch, val_s)
        blend_jobs.append(dict(height=H, width=W, head=head, decoded=cur, pitch_bytes=pitch, mask=mask,
                               mask_pitch_words=pl.mask.shape[1], mu_sigma=ms, out=out_b, out_pitch=pitch,
                               values=val_b))
        singles.append((tok_b, tok_s, out_b, out_s, val_b, val_s, refs, cur, head, mask, ms))
    R.op_assemble_batch(C, k, T, assemble_jobs, 1)
    R.op_blend_batch(C, blend_jobs)
    torch.cuda.synchronize()
    for tok_b, tok_s, out_b, out_s, val_b, val_s, *_ in singles:
        assert torch.equal(tok_b, tok_s)
        assert torch.equal(out_b, out_s)
        assert torch.equal(val_b, val_s)


@pytest.mark.parametrize("unaligned", [False, True])
@pytest.mark.parametrize("k,T", [(5, 2), (3, 1)])
@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_embed_batch_equals_assemble_and_linear_pe(modality, k, T, unaligned):
    """The implicit-GEMM tubelet embedding of a batch of requests of different
    sizes (no token matrix: the GEMM's producer warps read the frames) against
    the assemble kernel's bf16 tokens through revo_op_linear_pe per request:
    the same operands and epilogue, so depth is equal bit for bit; RGB takes its
    K blocks with the three channel blocks of a pixel group together, the same
    float32 sums in another order (24 block sums re-associated: within 1e-5).  The batch spans
    several 128-row tiles with a ragged last one; one request's temporal
    distance lies beyond the embedding table; with `unaligned` every frame row
    starts off the 8/16-byte grid (the narrow-load path)."""
    C = 3 if modality == "rgb" else 1
    N, p = 768, 16
    K = T * C * p * p
    S = (k + 1) // T
    sizes = [(48, 80), (160, 224), (32, 128), (64, 64)]
    rng = np.random.default_rng(17 + k + T + C)
    W = bf16(synth.normal(4242 + K, (N, K), 1.0 / np.sqrt(K))).cuda()
    b = dev(synth.normal(4243, (N,), 0.1))
    jobs, taus, refs_out = [], [], []
    for i, (H, Wd) in enumerate(sizes):
        pl = synth.make_tiny_plane(610 + 7 * i + k, modality, H, Wd, k)
        frames = list(pl.refs) + [pl.decoded]
        if unaligned:
            pf = [pitched(f, 4 if C == 3 else 6, 4 if C == 3 else 2) for f in frames]
            fr, pitch = [x[0] for x in pf], pf[0][1]
        else:
            fr, pitch = [dev(f) for f in frames], Wd * (3 if C == 3 else 2)
        ms = dev(np.array([1500.0 + 50 * i, 700.0 - 30 * i], np.float32)) if C == 1 else None
        ts = [int(x) for x in rng.integers(1, 9, S)]
        if i == 1:
            ts[0] = 300  # beyond the 256-row embedding table
        Hp, Wp = H // p, Wd // p
        tok = torch.zeros((S * Hp * Wp, K), dtype=torch.bfloat16, device="cuda")
        R.op_assemble(C, k, T, p, H, Wd, fr[:k], fr[k], pitch, ms, tok, 1)
        want = torch.zeros((S * Hp * Wp, N), dtype=torch.float32, device="cuda")
        R.op_linear_pe(tok, W, b, want, S, Hp, Wp, N, K, ts, 256)
        jobs.append(dict(height=H, width=Wd, frames=fr, pitch_bytes=pitch, mu_sigma=ms))
        taus.append(ts)
        refs_out.append(want)
    M = sum(t.shape[0] for t in refs_out)
    assert M > 3 * 128 and M % 128
    out = torch.full((M, N), 7.0, dtype=torch.float32, device="cuda")
    R.op_embed_batch(C, k, T, jobs, taus, W, b, out, N)
    torch.cuda.synchronize()
    want = torch.cat(refs_out)
    if C == 1:
        assert torch.equal(out, want)
    else:
        np.testing.assert_allclose(f64(out), f64(want), rtol=1e-5, atol=2e-5)
    assert R.take_device_error() == 0


@pytest.mark.parametrize("modality,H,W", [("rgb", 48, 80), ("depth", 64, 48), ("rgb", 240, 320)])
def test_blend_codes_bit_exact(modality, H, W):
    """Received pixels are copied bit for bit; lost pixels carry the float32
    de-normalise + round-half-even + clamp code exactly."""
    C, p = (3, 16) if modality == "rgb" else (1, 16)
    pl = synth.make_tiny_plane(H + W, modality, H, W, 1)
    Hp, Wp = H // p, W // p
    head = synth.normal(H * W, (Hp * Wp, C * p * p), 1.5 if modality == "rgb" else 0.8)
    y = O.untubelet_frame(head.astype(np.float64), C, 1, p, Hp, Wp, 0).astype(np.float32)  # [C, H, W]
    if modality == "rgb":
        vals = O.denormalise_rgb(y, np.float32)
        codes = O.quantise_rgb(vals, np.float32)
        ms = None
        pitch = W * 3
    else:
        mu, sg = 2500.0, 700.0
        vals = O.denormalise_depth(y, mu, sg, np.float32)
        codes = O.quantise_depth(vals, np.float32)
        ms = dev(np.array([mu, sg], np.float32))
        pitch = W * 2
    expect = O.blend(pl.decoded, O.unpack_mask(pl.mask, W), codes)
    out = torch.zeros(pl.decoded.shape, dtype=torch.uint8 if modality == "rgb" else torch.int16, device="cuda")
    values = torch.zeros(vals.shape, dtype=torch.float32, device="cuda")
    R.op_blend(C, p, H, W, dev(head), dev(pl.decoded), pitch, dev(pl.mask), pl.mask.shape[1], ms, out, pitch,
               values)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint8 if modality == "rgb" else np.uint16)
    np.testing.assert_array_equal(got, expect)
    np.testing.assert_array_equal(got[~pl.lost], pl.decoded[~pl.lost])
    np.testing.assert_array_equal(values.cpu().numpy(), vals)


# ------------------------------------------------------------ frame metrics

from oracle import metrics as MX  # noqa: E402


@pytest.mark.parametrize("kind,H,W", [("rgb", 240, 320), ("rgb", 37, 53), ("depth", 480, 640), ("depth", 11, 11),
                                      ("rgb", 720, 1280)])
def test_frame_metrics_ssim_psnr(kind, H, W):
    """SSIM (mean over the valid window positions, channels averaged) and PSNR
    against the float64 oracle: |dSSIM| <= 2e-5, |dPSNR| <= 1e-3 dB."""
    rng = np.random.default_rng(H * W)
    if kind == "rgb":
        x = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
        y = np.clip(x.astype(np.int32) + rng.integers(-20, 21, x.shape), 0, 255).astype(np.uint8)
        L, C, sb = 255.0, 3, 1
        tx, ty = dev(x), dev(y)
    else:
        x = rng.integers(500, 4001, (H, W), dtype=np.uint16)
        y = np.clip(x.astype(np.int32) + rng.integers(-60, 61, x.shape), 0, 65535).astype(np.uint16)
        L, C, sb = 65535.0, 1, 2
        tx, ty = dev(x.view(np.int16)), dev(y.view(np.int16))
    scratch = torch.zeros(R.frame_metrics_scratch_bytes(H, W, C) // 4 + 1, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float32, device="cuda")
    R.op_frame_metrics(tx, ty, H, W, C, sb, L, scratch, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert abs(got[0] - MX.ssim(x, y, L)) <= 2e-5
    assert abs(got[1] - MX.mse(x, y)) <= 1e-5 * MX.mse(x, y)
    assert abs(got[2] - MX.psnr(x, y, L)) <= 1e-3
    # identical frames: SSIM 1, PSNR infinite; a second call gives the same bits
    R.op_frame_metrics(tx, tx, H, W, C, sb, L, scratch, out)
    torch.cuda.synchronize()
    same = out.cpu().numpy()
    assert abs(same[0] - 1.0) < 1e-6 and same[1] == 0 and np.isinf(same[2])
    R.op_frame_metrics(tx, ty, H, W, C, sb, L, scratch, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), got.astype(np.float32))


# ---------------------------------------------------------------------- fec

from oracle import fec as FEC  # noqa: E402

_GF_TABLE = None


def gf_table():
    """256 x 256 products from the oracle's field multiplication (built once)."""
    global _GF_TABLE
    if _GF_TABLE is None:
        _GF_TABLE = np.array([[FEC.gf_mul(a, b) for b in range(256)] for a in range(256)], np.uint8)
    return _GF_TABLE


def oracle_parity(data, r):
    """The oracle's parity rows, evaluated with its product table (vectorised)."""
    T = gf_table()
    n = data.shape[0]
    C = FEC.cauchy(n, r)
    out = np.zeros((r, data.shape[1]), np.uint8)
    for i in range(r):
        for j in range(n):
            out[i] ^= T[C[i][j]][data[j]]
    return out


@pytest.mark.parametrize("n,r,S", [(8, 4, 1200), (84, 42, 1200), (170, 85, 64), (1, 0, 4), (255, 1, 1004),
                                    (3, 253, 12)])
def test_fec_encode_decode(n, r, S):
    """Parity bit-exact against the oracle; every data packet rebuilt bit for
    bit from random n-subsets of the n + r packets (all parity, no parity,
    mixed)."""
    rng = np.random.default_rng(n * 1000 + r)
    data = rng.integers(0, 256, (n, S), dtype=np.uint8)
    parity = torch.zeros((max(r, 1), S), dtype=torch.uint8, device="cuda")
    d_data = dev(data)
    R.fec_encode(n, r, S, d_data, parity)
    torch.cuda.synchronize()
    if r > 0:
        np.testing.assert_array_equal(parity.cpu().numpy()[:r], oracle_parity(data, r))
    shards = np.concatenate([data, parity.cpu().numpy()[:r]])
    scratch = torch.zeros(max(R.fec_decode_scratch_bytes(n), 1), dtype=torch.uint8, device="cuda")
    subsets = [list(range(n))]
    if r > 0:
        subsets.append(sorted(rng.choice(n + r, n, replace=False).tolist()))
        subsets.append(list(range(max(0, n - r), n + r))[-n:] if r >= n else list(range(r, n + r)))
        subsets.append(rng.permutation(n + r)[:n].tolist())  # unsorted order
    for present in subsets:
        out = torch.zeros((n, S), dtype=torch.uint8, device="cuda")
        R.fec_decode(n, r, S, present, dev(shards[present]), out, scratch)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), data)


# ------------------------------------------------------------------- render

from oracle import render as RD  # noqa: E402


def _rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay), np.cos(az), np.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return (Rz @ Ry @ Rx).astype(np.float32)


@pytest.mark.parametrize("case", ["identity", "turn", "shift", "splat2", "sizes", "upscale"])
def test_render_rgbd_bit_exact(case):
    """Unprojection + splatting against the oracle, bit for bit (the same
    float32 steps, nearest-z with index ties)."""
    rgb, dep = synth.make_request(4242, "640x480")
    depth = dep.clean.copy()
    depth[::7, ::5] = 0  # holes
    color = rgb.clean
    H, W = depth.shape
    K = (525.0, 525.0, 319.5, 239.5)
    rot, t, Kd, out_hw, s = np.eye(3, dtype=np.float32), (0.0, 0.0, 0.0), K, (H, W), 0
    if case == "turn":
        rot, t = _rot(0.05, -0.12, 0.02), (40.0, -25.0, 120.0)
    elif case == "shift":
        t = (0.0, 0.0, -300.0)
    elif case == "splat2":
        rot, t, s = _rot(0.0, 0.2, 0.0), (150.0, 0.0, 0.0), 2
    elif case == "sizes":
        rgb2, _ = synth.make_request(4243, "1280x720+640x576")
        color = rgb2.clean  # 1280x720 colour over the 640x480 depth
        rot, t = _rot(0.0, -0.08, 0.0), (-60.0, 10.0, 0.0)
    elif case == "upscale":  # twice the resolution: 3 x 3 splats close the gaps
        Kd, out_hw, s = (1050.0, 1050.0, 639.5, 359.5), (720, 1280), 1
    ref_rgb, ref_d = RD.render(color, depth, K, rot, t, Kd, out_hw, splat=s)
    nbytes = R.render_scratch_bytes(*out_hw)
    assert nbytes == out_hw[0] * out_hw[1] * 8
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out_rgb = torch.zeros((*out_hw, 3), dtype=torch.uint8, device="cuda")
    out_d = torch.zeros(out_hw, dtype=torch.int16, device="cuda")
    R.render_rgbd(dev(color), dev(depth.view(np.int16)), K, rot, t, Kd, out_hw, s, scratch, out_rgb, out_d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_d.cpu().numpy().view(np.uint16), ref_d)
    np.testing.assert_array_equal(out_rgb.cpu().numpy(), ref_rgb)
    assert (ref_d > 0).mean() > 0.3  # the view actually shows the scene


# ------------------------------------------------------------ bounded waits

def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """A wait that nothing completes gives up after its limit, records its
    code in the device error word and returns; the next kernels run normally."""
    assert R.take_device_error() == 0
    R.op_wait_selftest(2_000_000)  # about 1 ms of SM clocks
    torch.cuda.synchronize()
    assert R.take_device_error() == 5
    assert R.take_device_error() == 0  # taking the word clears it
    M, D = 64, 192
    x = synth.normal(9, (M, D))
    out = torch.zeros((M, D), dtype=torch.float32, device="cuda")
    R.op_layernorm(dev(x), dev(np.ones(D, np.float32)), dev(np.zeros(D, np.float32)), out, M, D, 0)
    torch.cuda.synchronize()
    ref = O.layer_norm(x.astype(np.float64), np.ones(D), np.zeros(D))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=5e-5)
    with pytest.raises(R.RevoError):
        R.op_wait_selftest(10)  # below the accepted range: rejected on the host
