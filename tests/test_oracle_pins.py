"""Pins of the FP64 oracle against things other than itself.

Each step of the oracle is checked against an independent float64 library
routine (torch.nn.functional / torch.nn modules), against brute-force
direct summation on tiny inputs, against closed forms, or against
invariants of the method (Section 3.4, Appendix B.1, B.3).
"""
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import synth
from oracle import revo_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
torch.set_num_threads(min(8, os.cpu_count() or 1))


def _t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------- tubelets --

@pytest.mark.parametrize("C", [1, 3])
def test_tubelet_embedding_is_conv3d(C):
    """Tubelet embedding (App. B.3) == Conv3d with kernel = stride = (T, p, p)."""
    rng = np.random.default_rng(1)
    T, p, F_, H, W, D = 2, 4, 6, 8, 12, 5
    frames = rng.normal(size=(F_, C, H, W))
    w = rng.normal(size=(D, T * C * p * p))
    b = rng.normal(size=D)
    ours = O.linear(O.tubelets(frames, T, p), w, b)
    conv_w = w.reshape(D, T, C, p, p).transpose(0, 2, 1, 3, 4)     # (t,c,y,x) -> [D, C, T, p, p]
    ref = F.conv3d(_t(frames).permute(1, 0, 2, 3)[None], _t(conv_w), _t(b), stride=(T, p, p))
    ref = ref[0].permute(1, 2, 3, 0).reshape(-1, D).numpy()          # (s, ty, tx) token order
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("C", [1, 3])
def test_head_unpatchify_is_conv_transpose3d(C):
    """Pixel head + un-patchify of the last slot == ConvTranspose3d, frame t = T-1."""
    rng = np.random.default_rng(2)
    T, p, Hp, Wp, Dd = 2, 4, 3, 2, 7
    tok = rng.normal(size=(Hp * Wp, Dd))
    w = rng.normal(size=(T * C * p * p, Dd))
    b = rng.normal(size=T * C * p * p)
    ours = O.untubelet_frame(O.linear(tok, w, b), C, T, p, Hp, Wp, T - 1)
    ct_w = w.reshape(T, C, p, p, Dd).transpose(4, 1, 0, 2, 3)          # [Dd, C, T, p, p]
    x = _t(tok).reshape(Hp, Wp, Dd).permute(2, 0, 1)[None, :, None]   # [1, Dd, 1, Hp, Wp]
    ref = F.conv_transpose3d(x, _t(ct_w), stride=(T, p, p))[0, :, T - 1].numpy()
    ref = ref + np.tile(b.reshape(T, C, p, p)[T - 1], (1, Hp, Wp))
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


def test_tubelet_roundtrip_brute_force():
    """Brute-force index check of the (s, ty, tx) x (t, c, y, x) layout."""
    rng = np.random.default_rng(3)
    T, p, F_, C, H, W = 2, 2, 4, 3, 4, 6
    fr = rng.normal(size=(F_, C, H, W))
    tok = O.tubelets(fr, T, p)
    Hp, Wp = H // p, W // p
    for s in range(F_ // T):
        for ty in range(Hp):
            for tx in range(Wp):
                n = (s * Hp + ty) * Wp + tx
                for t in range(T):
                    for c in range(C):
                        for y in range(p):
                            for x in range(p):
                                kk = ((t * C + c) * p + y) * p + x
                                assert tok[n, kk] == fr[s * T + t, c, ty * p + y, tx * p + x]


# ----------------------------------------------------------- layer pieces --

def test_layer_norm_matches_torch():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(17, 48)) * 3 + 1
    g, b = rng.normal(size=48), rng.normal(size=48)
    ref = F.layer_norm(_t(x), (48,), _t(g), _t(b), eps=1e-6).numpy()
    np.testing.assert_allclose(O.layer_norm(x, g, b), ref, rtol=0, atol=1e-12)


def test_layer_norm_invariants():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(9, 64)) * 5 - 2
    y = O.layer_norm(x, np.ones(64), np.zeros(64))
    np.testing.assert_allclose(y.mean(axis=1), 0, atol=1e-13)
    var = x.var(axis=1)
    np.testing.assert_allclose(y.var(axis=1), var / (var + 1e-6), rtol=1e-12)


def test_gelu_matches_torch_and_closed_forms():
    x = np.linspace(-8, 8, 1001)
    np.testing.assert_allclose(O.gelu(x), F.gelu(_t(x)).numpy(), rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.gelu(x) - O.gelu(-x), x, atol=1e-14)     # x Phi(x) + x Phi(-x) = x
    assert O.gelu(np.array([0.0]))[0] == 0.0
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert abs(O.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-14


def _brute_attention(q, k, v, heads):
    N, D = q.shape
    dh = D // heads
    out = np.zeros((N, D))
    for h in range(heads):
        for i in range(N):
            s = [sum(q[i, h * dh + d] * k[j, h * dh + d] for d in range(dh)) / math.sqrt(dh) for j in range(N)]
            m = max(s)
            e = [math.exp(x - m) for x in s]
            z = sum(e)
            for d in range(dh):
                out[i, h * dh + d] = sum(e[j] / z * v[j, h * dh + d] for j in range(N))
    return out


def test_attention_brute_force_and_sdpa():
    rng = np.random.default_rng(6)
    N, D, H = 7, 8, 2
    qkv = rng.normal(size=(N, 3 * D)) * 2
    ours = O.attention(qkv, H)
    q, k, v = qkv[:, :D], qkv[:, D:2 * D], qkv[:, 2 * D:]
    np.testing.assert_allclose(ours, _brute_attention(q, k, v, H), rtol=0, atol=1e-12)
    qt = _t(q).reshape(N, H, D // H).transpose(0, 1)
    kt = _t(k).reshape(N, H, D // H).transpose(0, 1)
    vt = _t(v).reshape(N, H, D // H).transpose(0, 1)
    ref = F.scaled_dot_product_attention(qt, kt, vt).transpose(0, 1).reshape(N, D).numpy()
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


def test_softmax_rows_sum_to_one():
    s = np.random.default_rng(7).normal(size=(5, 300)) * 30
    np.testing.assert_allclose(O.softmax_rows(s).sum(axis=1), 1.0, atol=1e-14)


def test_attention_permutation_equivariant():
    rng = np.random.default_rng(8)
    qkv = rng.normal(size=(11, 3 * 12))
    perm = rng.permutation(11)
    np.testing.assert_allclose(O.attention(qkv[perm], 3), O.attention(qkv, 3)[perm], atol=1e-13)


def _torch_block(w, prefix, d, heads, mlp):
    layer = torch.nn.TransformerEncoderLayer(d, heads, dim_feedforward=mlp, dropout=0.0, activation="gelu",
                                             layer_norm_eps=1e-6, batch_first=True, norm_first=True,
                                             dtype=torch.float64)
    with torch.no_grad():
        layer.norm1.weight.copy_(_t(w[prefix + "ln1.g"]))
        layer.norm1.bias.copy_(_t(w[prefix + "ln1.b"]))
        layer.self_attn.in_proj_weight.copy_(_t(w[prefix + "qkv.w"]))
        layer.self_attn.in_proj_bias.copy_(_t(w[prefix + "qkv.b"]))
        layer.self_attn.out_proj.weight.copy_(_t(w[prefix + "proj.w"]))
        layer.self_attn.out_proj.bias.copy_(_t(w[prefix + "proj.b"]))
        layer.norm2.weight.copy_(_t(w[prefix + "ln2.g"]))
        layer.norm2.bias.copy_(_t(w[prefix + "ln2.b"]))
        layer.linear1.weight.copy_(_t(w[prefix + "fc1.w"]))
        layer.linear1.bias.copy_(_t(w[prefix + "fc1.b"]))
        layer.linear2.weight.copy_(_t(w[prefix + "fc2.w"]))
        layer.linear2.bias.copy_(_t(w[prefix + "fc2.b"]))
    return layer.train(False)


def test_block_matches_torch_transformer_layer():
    """Pre-LN block with exact GELU == torch.nn.TransformerEncoderLayer(norm_first=True)."""
    cfg = synth.tiny(3, enc_dim=32, enc_heads=4)
    w = {n: a.astype(np.float64) for n, a in synth.weights(cfg, seed=11).items()}
    x = np.random.default_rng(9).normal(size=(13, 32))
    layer = _torch_block(w, "enc.0.", 32, 4, 128)
    with torch.no_grad():
        ref = layer(_t(x)[None])[0].numpy()
    np.testing.assert_allclose(O.block(x, w, "enc.0.", 4), ref, rtol=0, atol=1e-11)


# --------------------------------------------------------- whole network --

def _torch_forward(w, cfg, frames, taus):
    """The same network assembled from torch float64 modules: Conv3d tubelet
    embedding, TransformerEncoderLayer blocks, LayerNorm, Linear, and a
    ConvTranspose3d pixel head."""
    F_, C, H, W = frames.shape
    T, p = cfg.tubelet, cfg.patch
    Hp, Wp = H // p, W // p
    D, Dd, K = cfg.enc_dim, cfg.dec_dim, cfg.token_dim
    conv_w = w["patch_embed.w"].reshape(D, T, C, p, p).transpose(0, 2, 1, 3, 4)
    x = F.conv3d(_t(frames).permute(1, 0, 2, 3)[None], _t(conv_w), _t(w["patch_embed.b"]), stride=(T, p, p))
    x = x[0].permute(1, 2, 3, 0).reshape(-1, D)
    x = x + _t(O.position_embedding(taus, Hp, Wp, D))
    with torch.no_grad():
        for i in range(cfg.enc_depth):
            x = _torch_block(w, f"enc.{i}.", D, cfg.enc_heads, cfg.mlp_ratio * D)(x[None])[0]
        x = F.layer_norm(x, (D,), _t(w["enc_norm.g"]), _t(w["enc_norm.b"]), eps=1e-6)
        x = F.linear(x, _t(w["enc2dec.w"]), _t(w["enc2dec.b"])) + _t(O.position_embedding(taus, Hp, Wp, Dd))
        for i in range(cfg.dec_depth):
            x = _torch_block(w, f"dec.{i}.", Dd, cfg.dec_heads, cfg.mlp_ratio * Dd)(x[None])[0]
        x = F.layer_norm(x, (Dd,), _t(w["dec_norm.g"]), _t(w["dec_norm.b"]), eps=1e-6)
    S = F_ // T
    last = x[(S - 1) * Hp * Wp:].reshape(Hp, Wp, Dd).permute(2, 0, 1)[None, :, None]
    ct_w = w["head.w"].reshape(T, C, p, p, Dd).transpose(4, 1, 0, 2, 3)
    y = F.conv_transpose3d(last, _t(ct_w), stride=(T, p, p))[0, :, T - 1].numpy()
    return y + np.tile(w["head.b"].reshape(T, C, p, p)[T - 1], (1, Hp, Wp))


@pytest.mark.parametrize("C,k", [(3, 1), (1, 3), (3, 5)])
def test_forward_matches_torch_modules(C, k):
    cfg = synth.tiny(C, k=k, enc_depth=2, dec_depth=2, enc_dim=24, dec_dim=12)
    w = {n: a.astype(np.float64) for n, a in synth.weights(cfg, seed=5).items()}
    frames = np.random.default_rng(10).normal(size=(k + 1, C, 8, 12))
    taus = O.temporal_distances(np.arange(10 - k, 10), 10, cfg.tubelet)
    np.testing.assert_allclose(O.forward(w, cfg, frames, taus), _torch_forward(w, cfg, frames, taus),
                               rtol=0, atol=1e-11)


def _brute_forward(w, cfg, frames, taus):
    """Direct-summation forward in pure Python loops (tiny sizes only)."""
    F_, C, H, W = frames.shape
    T, p = cfg.tubelet, cfg.patch
    Hp, Wp, S = H // p, W // p, F_ // T

    def lin(x, name):
        Wm, b = w[name + ".w"], w[name + ".b"]
        return [[b[o] + sum(Wm[o][i] * row[i] for i in range(len(row))) for o in range(len(b))] for row in x]

    def ln(x, name):
        g, b = w[name + ".g"], w[name + ".b"]
        out = []
        for row in x:
            m = sum(row) / len(row)
            v = sum((a - m) ** 2 for a in row) / len(row)
            out.append([(a - m) / math.sqrt(v + 1e-6) * g[i] + b[i] for i, a in enumerate(row)])
        return out

    def pe(d):
        part = d // 3
        def sc(pos):
            half = part // 2
            return [math.sin(pos * 10000 ** (-2 * i / part)) for i in range(half)] + \
                   [math.cos(pos * 10000 ** (-2 * i / part)) for i in range(half)]
        return [sc(taus[s]) + sc(r) + sc(c) for s in range(S) for r in range(Hp) for c in range(Wp)]

    def blk(x, pre, heads):
        d = len(x[0])
        dh = d // heads
        h = ln(x, pre + "ln1")
        qkv = lin(h, pre + "qkv")
        n = len(x)
        att = [[0.0] * d for _ in range(n)]
        for hh in range(heads):
            for i in range(n):
                s = [sum(qkv[i][hh * dh + e] * qkv[j][d + hh * dh + e] for e in range(dh)) / math.sqrt(dh)
                     for j in range(n)]
                m = max(s)
                ex = [math.exp(a - m) for a in s]
                z = sum(ex)
                for e in range(dh):
                    att[i][hh * dh + e] = sum(ex[j] / z * qkv[j][2 * d + hh * dh + e] for j in range(n))
        pr = lin(att, pre + "proj")
        x = [[x[i][e] + pr[i][e] for e in range(d)] for i in range(n)]
        h = lin(ln(x, pre + "ln2"), pre + "fc1")
        h = [[0.5 * a * (1 + math.erf(a / math.sqrt(2))) for a in row] for row in h]
        f2 = lin(h, pre + "fc2")
        return [[x[i][e] + f2[i][e] for e in range(d)] for i in range(n)]

    toks = []
    for s in range(S):
        for ty in range(Hp):
            for tx in range(Wp):
                toks.append([frames[s * T + t, c, ty * p + y, tx * p + xx]
                             for t in range(T) for c in range(C) for y in range(p) for xx in range(p)])
    x = lin(toks, "patch_embed")
    x = [[a + b for a, b in zip(r1, r2)] for r1, r2 in zip(x, pe(cfg.enc_dim))]
    for i in range(cfg.enc_depth):
        x = blk(x, f"enc.{i}.", cfg.enc_heads)
    x = lin(ln(x, "enc_norm"), "enc2dec")
    x = [[a + b for a, b in zip(r1, r2)] for r1, r2 in zip(x, pe(cfg.dec_dim))]
    for i in range(cfg.dec_depth):
        x = blk(x, f"dec.{i}.", cfg.dec_heads)
    y = lin(ln(x, "dec_norm"), "head")
    out = np.zeros((C, H, W))
    for ty in range(Hp):
        for tx in range(Wp):
            v = y[(S - 1) * Hp * Wp + ty * Wp + tx]
            for c in range(C):
                for yy in range(p):
                    for xx in range(p):
                        out[c, ty * p + yy, tx * p + xx] = v[(((T - 1) * C + c) * p + yy) * p + xx]
    return out


def test_forward_brute_force_tiny():
    cfg = synth.tiny(1, k=3, patch=2, enc_dim=6, enc_heads=2, dec_dim=6, dec_heads=2)
    w = {n: a.astype(np.float64) for n, a in synth.weights(cfg, seed=3).items()}
    frames = np.random.default_rng(12).normal(size=(4, 1, 4, 4))
    taus = [3, 1]
    np.testing.assert_allclose(O.forward(w, cfg, frames, taus), _brute_forward(w, cfg, frames, taus),
                               rtol=0, atol=1e-12)


# ------------------------------------------------------ embedding / shapes --

def test_sincos_closed_form():
    np.testing.assert_array_equal(O.sincos(0.0, 8), [0, 0, 0, 0, 1, 1, 1, 1])
    v = O.sincos(1.0, 4)   # w = [1, 10000^(-1/2) = 0.01]
    np.testing.assert_allclose(v, [math.sin(1), math.sin(0.01), math.cos(1), math.cos(0.01)], atol=1e-16)


def test_position_embedding_is_resolution_consistent():
    small = O.position_embedding([4, 2, 0], 15, 20, 48).reshape(3, 15, 20, 48)
    big = O.position_embedding([4, 2, 0], 30, 40, 48).reshape(3, 30, 40, 48)
    np.testing.assert_array_equal(small, big[:, :15, :20])


def test_temporal_distances():
    assert O.temporal_distances([95, 96, 97, 98, 99], 100, 2) == [5, 3, 1]
    assert O.temporal_distances([95, 96, 97, 98, 99], 102, 2) == [7, 5, 3]
    assert O.temporal_distances([9], 10, 2) == [1]


def test_golden_token_and_parameter_counts():
    g = json.load(open(os.path.join(GOLDEN, "shapes.json")))
    for key, n in g["tokens"].items():
        H, W = map(int, key.split("x"))
        assert synth.RGB.tokens(H, W) == n
    for name, cfg in (("rgb", synth.RGB), ("depth", synth.DEPTH)):
        total = sum(int(np.prod(s)) for s in synth.param_shapes(cfg).values())
        assert total == g["params"][name]
    enc = sum(int(np.prod(s)) for n, s in synth.param_shapes(synth.RGB).items() if n.startswith("enc.0."))
    dec = sum(int(np.prod(s)) for n, s in synth.param_shapes(synth.RGB).items() if n.startswith("dec.0."))
    assert enc == g["encoder_block_params"] and dec == g["decoder_block_params"]


# ------------------------------------------------------- normalise / blend --

def test_rgb_normalisation_closed_form():
    f = np.array([[[0, 255, 128]]], dtype=np.uint8)
    v = O.normalise_rgb(f)[:, 0, 0]
    np.testing.assert_allclose(v, [(0 - 0.485) / 0.229, (1 - 0.456) / 0.224, (128 / 255 - 0.406) / 0.225],
                               atol=1e-15)


def test_depth_stats_closed_forms():
    assert O.depth_stats(np.zeros((4, 4), np.uint16)) == (0.0, 1.0)
    f = np.full((4, 4), 1000, np.uint16)
    f[0, 0] = 0
    assert O.depth_stats(f) == (1000.0, 1.0)
    g = np.array([[1000, 3000, 0, 1000, 3000]], np.uint16)
    assert O.depth_stats(g) == (2000.0, 1000.0)


def test_rgb_denormalise_inverts_normalise_for_every_code():
    """De-normalisation is the inverse of the input normalisation: for every
    uint8 code, on a frame whose height, width and channel count all differ,
    normalise then de-normalise gives the code / 255 in [H, W, 3] layout.  A
    swapped mean and std, a division in place of the product, or a transposed
    axis fails here."""
    codes = np.arange(256, dtype=np.uint8)
    rng = np.random.default_rng(31)
    f = rng.permutation(np.concatenate([codes, codes, codes, codes[:12]]))[:4 * 5 * 3 * 13].reshape(4 * 13, 5, 3)
    f = np.ascontiguousarray(f[:20]).astype(np.uint8)      # [20, 5, 3]: H != W != C
    for frame in (f, np.ascontiguousarray(np.broadcast_to(codes[:, None, None], (256, 2, 3)))):
        y = O.normalise_rgb(frame)
        assert y.shape == (3,) + frame.shape[:2]
        np.testing.assert_allclose(O.denormalise_rgb(y), frame / 255.0, rtol=0, atol=1e-15)


def test_rgb_denormalise_closed_forms():
    """y = 0 gives each channel's mean, y = 1 its mean plus its deviation, at
    every pixel of the [H, W, 3] result (ImageNet statistics)."""
    mean, std = np.array([0.485, 0.456, 0.406]), np.array([0.229, 0.224, 0.225])
    z = O.denormalise_rgb(np.zeros((3, 2, 7)))
    o = O.denormalise_rgb(np.ones((3, 2, 7)))
    assert z.shape == (2, 7, 3)
    np.testing.assert_allclose(z, np.broadcast_to(mean, (2, 7, 3)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(o, np.broadcast_to(mean + std, (2, 7, 3)), rtol=0, atol=1e-15)
    # one channel at a time: channel c of y lands in the last axis at c
    for c in range(3):
        y = np.zeros((3, 2, 7))
        y[c] = 1.0
        want = mean.copy()
        want[c] += std[c]
        np.testing.assert_allclose(O.denormalise_rgb(y), np.broadcast_to(want, (2, 7, 3)), rtol=0, atol=1e-15)


def test_depth_normalise_closed_forms_and_inverse():
    """(d - mu) / sigma with a non-trivial (mu, sigma): d = mu -> 0,
    d = mu + sigma -> 1, d = 0 (no measurement) -> -mu / sigma; de-normalising
    gives the millimetres back for every code of a range, in [H, W] layout."""
    mu, sigma = 1234.5, 321.25
    d = np.array([[1234, 1235, 0], [1555, 1556, 913]], np.uint16)
    y = O.normalise_depth(d, mu, sigma)
    assert y.shape == (1, 2, 3)
    np.testing.assert_allclose(y[0, 1, 0], (1555 - mu) / sigma, atol=1e-15)
    np.testing.assert_allclose(y[0, 0, 2], -mu / sigma, atol=1e-15)
    e = np.array([[mu, mu + sigma, mu - sigma]])
    np.testing.assert_allclose(O.normalise_depth(e, mu, sigma)[0], [[0.0, 1.0, -1.0]], atol=1e-15)
    np.testing.assert_allclose(O.denormalise_depth(np.array([[[0.0, 1.0, -2.0]]]), mu, sigma),
                               [[mu, mu + sigma, mu - 2 * sigma]], atol=1e-12)
    codes = np.arange(0, 65536, 7, dtype=np.uint16)[:9000].reshape(90, 100)
    back = O.denormalise_depth(O.normalise_depth(codes, mu, sigma), mu, sigma)
    assert back.shape == codes.shape
    np.testing.assert_allclose(back, codes.astype(np.float64), rtol=0, atol=1e-10)


def _constant_output_weights(cfg, head_bias):
    """Weights whose network output is head_bias at every pixel, whatever the
    input: every matrix and every LayerNorm gain is zero (each LayerNorm then
    outputs its shift, zero), so the pixel head sees zeros and adds its bias."""
    w = synth.weights(cfg, seed=3)
    for n in w:
        w[n] = np.zeros_like(w[n])
    w["head.b"] = np.full_like(w["head.b"], head_bias)
    return w


@pytest.mark.parametrize("head_bias", [0.0, 1.0, -0.5])
def test_recover_depth_statistics_come_from_the_newest_reference(head_bias):
    """recover() normalises depth with the statistics of the newest reference
    (the last clean frame), not of the current frame or an older reference.
    With a network whose normalised output is the constant y, every recovered
    depth is y * sigma + mu of that frame: here mu = 2000, sigma = 1000 (half
    the valid pixels at 1000 mm, half at 3000, zeros excluded), while the
    current frame and the older references have mean 500 (sigma floored to 1)."""
    cfg = synth.tiny(1, k=3)
    w = _constant_output_weights(cfg, head_bias)
    H, W = 8, 12
    old = np.full((H, W), 500, np.uint16)
    newest = np.zeros((H, W), np.uint16)
    newest[:, 0::2] = 1000
    newest[:, 1::2] = 3000
    newest[0, :4] = 0
    newest[1, :2] = 0   # zeros are excluded; 46 pixels of each value remain
    refs = np.stack([old, old, newest])
    decoded = np.full((H, W), 500, np.uint16)
    lost = np.zeros((H, W), bool)
    lost[:4] = True
    decoded[lost] = 0
    codes, values = O.recover("depth", w, cfg, refs, [7, 8, 9], decoded, synth.pack_mask(lost), 10)
    np.testing.assert_allclose(values, np.full((H, W), head_bias * 1000.0 + 2000.0), rtol=0, atol=1e-9)
    np.testing.assert_array_equal(codes[lost], np.full(lost.sum(), round(head_bias * 1000 + 2000), np.uint16))
    np.testing.assert_array_equal(codes[~lost], decoded[~lost])


@pytest.mark.parametrize("head_bias", [0.0, 1.0])
def test_recover_rgb_denormalises_per_channel(head_bias):
    """recover() for RGB: a constant normalised output y gives y std_c + mean_c
    in channel c of every pixel (ImageNet statistics), whatever the frames."""
    cfg = synth.tiny(3, k=1)
    w = _constant_output_weights(cfg, head_bias)
    pl = synth.make_tiny_plane(9, "rgb", 8, 12, 1, lost_rows=[2, 3])
    _, values = O.recover("rgb", w, cfg, pl.refs, pl.ref_index, pl.decoded, pl.mask, pl.index)
    want = np.array([0.485, 0.456, 0.406]) + head_bias * np.array([0.229, 0.224, 0.225])
    np.testing.assert_allclose(values, np.broadcast_to(want, (8, 12, 3)), rtol=0, atol=1e-14)


def test_quantisation_round_half_even_and_clamp():
    v = np.array([0.5, 1.5, 2.5, -3.0, 300.0, 254.5]) / 255.0
    np.testing.assert_array_equal(O.quantise_rgb(v * 255.0 / 255.0), [0, 2, 2, 0, 255, 254])
    np.testing.assert_array_equal(O.quantise_depth(np.array([1000.5, 1001.5, -1.0, 65535.7, 70000.0])),
                                  [1000, 1002, 0, 65535, 65535])


def test_mask_pack_unpack_roundtrip():
    rng = np.random.default_rng(13)
    lost = rng.random((5, 70)) < 0.3
    words = synth.pack_mask(lost)
    assert words.shape == (5, 3) and words.dtype == np.uint32
    np.testing.assert_array_equal(O.unpack_mask(words, 70), lost)
    # bit x % 32 of word x // 32, LSB first
    one = np.zeros((1, 40), bool)
    one[0, 33] = True
    assert synth.pack_mask(one)[0, 1] == 2


# ------------------------------------------------------- end-to-end shape --

@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_all_received_passes_through_bit_exact(modality):
    C = 3 if modality == "rgb" else 1
    cfg = synth.tiny(C, k=3)
    w = synth.weights(cfg, seed=1)
    pl = synth.make_tiny_plane(4, modality, 8, 12, 3, lost_rows=[])
    codes, _ = O.recover(modality, w, cfg, pl.refs, pl.ref_index, pl.decoded, pl.mask, pl.index)
    assert codes.dtype == pl.decoded.dtype
    np.testing.assert_array_equal(codes, pl.decoded)


@pytest.mark.parametrize("modality", ["rgb", "depth"])
def test_received_pixels_unchanged_lost_pixels_recovered(modality):
    C = 3 if modality == "rgb" else 1
    cfg = synth.tiny(C, k=3)
    w = synth.weights(cfg, seed=1)
    pl = synth.make_tiny_plane(5, modality, 8, 12, 3, lost_rows=[0, 1, 2, 3])
    codes, values = O.recover(modality, w, cfg, pl.refs, pl.ref_index, pl.decoded, pl.mask, pl.index)
    np.testing.assert_array_equal(codes[~pl.lost], pl.decoded[~pl.lost])
    q = O.quantise_rgb(values) if modality == "rgb" else O.quantise_depth(values)
    np.testing.assert_array_equal(codes[pl.lost], q[pl.lost])
    assert values.shape[:2] == pl.decoded.shape[:2]


def _frames(C, k, H, W, seed=14):
    return np.random.default_rng(seed).normal(size=(k + 1, C, H, W))


def test_receptive_field_without_blocks_is_one_patch():
    """With no transformer block, a current-frame pixel only reaches its own patch."""
    cfg = synth.tiny(1, k=1, enc_depth=0, dec_depth=0)
    w = synth.weights(cfg, seed=2)
    fr = _frames(1, 1, 8, 12)
    y0 = O.forward(w, cfg, fr, [1])
    fr2 = fr.copy()
    fr2[-1, 0, 5, 6] += 1.0            # patch (1, 1) with p = 4
    diff = np.abs(O.forward(w, cfg, fr2, [1]) - y0)[0] > 0
    expect = np.zeros((8, 12), bool)
    expect[4:8, 4:8] = True
    np.testing.assert_array_equal(diff, expect)


def test_receptive_field_with_attention_is_global():
    cfg = synth.tiny(1, k=3, enc_depth=1, dec_depth=0)
    w = synth.weights(cfg, seed=2)
    fr = _frames(1, 3, 8, 12)
    y0 = O.forward(w, cfg, fr, [3, 1])
    fr2 = fr.copy()
    fr2[0, 0, 1, 1] += 1.0             # oldest reference frame: reaches output only through attention
    assert (np.abs(O.forward(w, cfg, fr2, [3, 1]) - y0) > 0).all()


def test_temporal_distance_changes_output():
    """Section 3.4.1: the embedding carries the reference-target distance, so the
    same references at another distance give another reconstruction."""
    cfg = synth.tiny(3, k=3)
    w = synth.weights(cfg, seed=2)
    fr = _frames(3, 3, 8, 12)
    a = O.forward(w, cfg, fr, O.temporal_distances([7, 8, 9], 10, 2))
    b = O.forward(w, cfg, fr, O.temporal_distances([7, 8, 9], 12, 2))
    assert np.abs(a - b).max() > 1e-6


def test_gilbert_elliott_stationary_rate():
    rng = np.random.default_rng(15)
    for rate in (0.05, 0.2, 0.4):
        lost = np.concatenate([synth.gilbert_elliott(rng, 1000, synth.p_gb_for_rate(rate), 0.5)
                               for _ in range(40)])
        assert abs(lost.mean() - rate) < 0.025
