"""The C-ABI library builds, loads, exports every symbol include/revo.h
declares, and validates arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import paper_2604_27441_b300 as R
from paper_2604_27441_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(R.LIB_PATH):
        B.build()
    return R.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "revo.h")).read()
    return sorted(set(re.findall(r"^REVO_API\s+[\w\s\*]*?\b(revo_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_four_recovery_calls():
    syms = declared_symbols()
    for name in ("revo_recover_create", "revo_recover_submit", "revo_recover_poll", "revo_recover_destroy"):
        assert name in syms
    assert len(syms) >= 16


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_config_default_is_the_vit_b_reading(lib):
    cfg = R.config()
    assert (cfg.k, cfg.tubelet, cfg.patch) == (5, 2, 16)
    assert (cfg.enc_dim, cfg.enc_depth, cfg.enc_heads) == (768, 12, 12)
    assert (cfg.dec_dim, cfg.dec_depth, cfg.dec_heads, cfg.mlp_ratio) == (384, 4, 6, 4)
    assert cfg.precision == R.BF16 and cfg.max_batch == 1 and cfg.lanes == 1


def test_struct_layouts_match_the_header(lib, tmp_path):
    """The binding's ctypes structs have the C compiler's sizes and offsets."""
    src = tmp_path / "layout.c"
    fields = {"revo_config": R.Config, "revo_plane": R.Plane, "revo_request": R.Request, "revo_result": R.Result,
              "revo_stats": R.Stats, "revo_intrinsics": R.Intrinsics, "revo_pose": R.Pose}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "revo.h"', "int main(void) {"]
    for cname, py in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                check=True).stdout.split("\n") if line)
    for cname, py in fields.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_null_arguments_are_rejected_before_any_device_work(lib):
    assert lib.revo_op_linear(R.FP32, 0, None, None, None, None, 4, 4, 8, 0, None) == R.REVO_EINVAL
    assert lib.revo_op_layernorm(None, None, None, None, 4, 8, 0, None) == R.REVO_EINVAL
    seg = (C.c_int * 2)(0, 4)
    assert lib.revo_op_attention(R.FP32, None, None, 4, 64, 1, seg, None, None, 1, 0, None) == R.REVO_EINVAL
    assert lib.revo_op_attention(R.FP32, 1, 1, 4, 96, 1, seg, None, None, 1, 0, None) == R.REVO_EINVAL  # width 96
    qb, qe = (C.c_int * 1)(0), (C.c_int * 1)(5)   # query rows past the segment end
    assert lib.revo_op_attention(R.FP32, 1, 1, 4, 64, 1, seg, qb, qe, 1, 0, None) == R.REVO_EINVAL
    assert lib.revo_op_attention(R.FP32, 1, 1, 4, 64, 1, seg, qb, None, 1, 0, None) == R.REVO_EINVAL
    assert lib.revo_op_depth_stats(None, 4, 4, 8, None, None, None) == R.REVO_EINVAL
    assert "bad argument" in R.last_error() or R.last_error()
    h = C.c_void_p()
    assert lib.revo_recover_create(None, C.byref(h)) == R.REVO_EINVAL
    assert lib.revo_recover_submit(None, None, None) == R.REVO_EINVAL
    assert lib.revo_recover_poll(None, 1, 0, None) == R.REVO_EINVAL
    assert lib.revo_recover_stats(None, None) == R.REVO_EINVAL
    assert lib.revo_fec_encode(0, 1, 8, None, 8, None, 8, None) == R.REVO_EINVAL
    assert lib.revo_fec_encode(200, 100, 8, 1, 8, 1, 8, None) == R.REVO_EINVAL  # n + r > 256
    assert lib.revo_fec_encode(4, 2, 6, 1, 8, 1, 8, None) == R.REVO_EINVAL     # packet not a multiple of 4
    dup = (C.c_int * 2)(0, 0)
    assert lib.revo_fec_decode(2, 1, 8, dup, 1, 8, 1, 8, 1, None) == R.REVO_EINVAL
    assert lib.revo_op_frame_metrics(None, 8, None, 8, 4, 4, 1, 1, 255.0, None, None, None) == R.REVO_EINVAL
    jobs = (R.AssembleJob * 1)()
    jobs[0].height, jobs[0].width, jobs[0].pitch_bytes = 32, 32, 96
    taus = (C.c_int * 8)()
    emb = lib.revo_op_embed_batch
    assert emb(3, 5, 2, 1, None, taus, 1, None, 1, 768, None) == R.REVO_EINVAL       # no jobs
    assert emb(3, 5, 3, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 768, None) == R.REVO_EINVAL  # T = 3
    assert emb(3, 4, 2, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 768, None) == R.REVO_EINVAL  # k + 1 odd
    assert emb(3, 5, 2, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 700, None) == R.REVO_EINVAL  # N % 192
    assert emb(2, 5, 2, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 768, None) == R.REVO_EINVAL  # 2 channels
    assert emb(3, 5, 2, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 768, None) == R.REVO_EINVAL  # no frames
    jobs[0].width = 40  # not a multiple of 16
    for f in range(6):
        jobs[0].frames[f] = 16
    assert emb(3, 5, 2, 1, C.cast(jobs, C.c_void_p), taus, 1, None, 1, 768, None) == R.REVO_EINVAL
    lib.revo_recover_destroy(None)


def test_bad_config_is_rejected(lib):
    cfg = R.config(max_batch=0)
    h = C.c_void_p()
    assert lib.revo_recover_create(C.byref(cfg), C.byref(h)) == R.REVO_EINVAL
    assert h.value is None
    cfg = R.config()  # no weights
    assert lib.revo_recover_create(C.byref(cfg), C.byref(h)) == R.REVO_EINVAL


def test_depth_stats_scratch_is_small(lib):
    n = R.depth_stats_scratch_bytes()
    assert 0 < n < 64 * 1024


def test_binding_refuses_non_contiguous_buffers():
    import numpy as np
    a = np.zeros((4, 6, 3), np.uint8)
    assert R.ptr(a) == a.ctypes.data
    with pytest.raises(ValueError):
        R.ptr(a.transpose(1, 0, 2))


def test_synthetic_frames_are_row_major():
    import synth
    rgb, dep = synth.make_request(1, "320x240")
    for pl in (rgb, dep, synth.make_tiny_plane(5, "rgb", 48, 80, 5)):
        for name in ("refs", "decoded", "mask", "clean", "lost"):
            assert getattr(pl, name).flags["C_CONTIGUOUS"], name


@pytest.mark.parametrize("shape,channels,seed", [
    (dict(k=1, tubelet=2, enc_dim=192, enc_depth=1, enc_heads=3, dec_dim=192, dec_depth=1, dec_heads=3), 3, 0),
    (dict(k=3, tubelet=1, enc_dim=384, enc_depth=2, enc_heads=6, dec_dim=192, dec_depth=1, dec_heads=3), 1, 7),
    (dict(), 3, 0), (dict(), 1, 1), (dict(), 3, 2 ** 40 + 5)])
def test_seeded_random_init_equals_the_synthetic_weights(shape, channels, seed):
    """revo_init_weights (C++, host) draws exactly the weights the Python side
    draws for the same shape and seed (NumPy's PCG64 seeded through
    SeedSequence, uniform doubles rounded to float32): bit for bit, so a
    context created from a seed alone computes the same network the oracle
    is given.  ViT-B shapes included (94 M parameters)."""
    import numpy as np
    import synth
    cfg = R.config(**shape)
    mc = synth.ModelConfig(channels=channels, k=cfg.k, tubelet=cfg.tubelet, patch=cfg.patch, enc_dim=cfg.enc_dim,
                           enc_depth=cfg.enc_depth, enc_heads=cfg.enc_heads, dec_dim=cfg.dec_dim,
                           dec_depth=cfg.dec_depth, dec_heads=cfg.dec_heads, mlp_ratio=cfg.mlp_ratio)
    want = synth.flatten(synth.weights(mc, seed=seed))
    got = R.init_weights(cfg, channels, seed)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_init_weights_rejects_a_wrong_count():
    import numpy as np
    cfg = R.config()
    out = np.empty(10, np.float32)
    assert R.lib().revo_init_weights(C.byref(cfg), 3, 0, out.ctypes.data, 10) == R.REVO_EINVAL
