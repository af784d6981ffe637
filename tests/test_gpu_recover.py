"""End-to-end parity of revo_recover_create/submit/poll/destroy with the FP64
oracle on seeded synthetic RGB-D frames.

Tolerances on the de-normalised float outputs (every pixel of the network
output, before the blend):
  FP32 path: max |error| <= 1e-4 on [0, 1] RGB and <= 1 mm on depth;
  BF16 and FP8 paths: PSNR >= 45 dB on [0, 1] RGB and on depth / 65535, max
             depth error <= 8 mm.
Blended codes: received pixels bit-exact; a lost pixel's code differs from the
oracle's by at most floor(|float error| * scale) + 1 and is equal wherever the
oracle's value is farther than the observed error from a rounding boundary.
"""
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


SMALL = dict(k=5, tubelet=2, patch=16, enc_dim=192, enc_depth=2, enc_heads=3, dec_dim=192, dec_depth=1,
             dec_heads=3, mlp_ratio=4)
VITB = dict(k=5, tubelet=2, patch=16, enc_dim=768, enc_depth=12, enc_heads=12, dec_dim=384, dec_depth=4,
            dec_heads=6, mlp_ratio=4)


def model_cfg(shape, C):
    return synth.ModelConfig(channels=C, k=shape["k"], tubelet=shape["tubelet"], patch=shape["patch"],
                             enc_dim=shape["enc_dim"], enc_depth=shape["enc_depth"], enc_heads=shape["enc_heads"],
                             dec_dim=shape["dec_dim"], dec_depth=shape["dec_depth"], dec_heads=shape["dec_heads"],
                             mlp_ratio=shape["mlp_ratio"])


_WEIGHTS = {}


def weights(shape, C):
    key = (tuple(sorted(shape.items())), C)
    if key not in _WEIGHTS:
        _WEIGHTS[key] = synth.weights(model_cfg(shape, C), seed=0 if C == 3 else 1)
    return _WEIGHTS[key]


def make_ctx(shape, precision, max_hw, max_batch=1, lanes=1, max_streams=4, use_graphs=0, autotune=0):
    w_rgb = synth.flatten(weights(shape, 3))
    w_dep = synth.flatten(weights(shape, 1))
    cfg = R.config(**shape, precision=precision, max_height=max_hw[0], max_width=max_hw[1], max_batch=max_batch,
                   lanes=lanes, max_streams=max_streams, use_graphs=use_graphs, autotune=autotune)
    return R.Context(cfg, w_rgb, w_dep)


def push_refs(ctx, sid, rgb, dep, on_device=True):
    keep = []
    for j in range(rgb.refs.shape[0]):
        fr, fd = rgb.refs[j], dep.refs[j]
        if on_device:
            fr, fd = torch.from_numpy(fr).cuda(), torch.from_numpy(fd.view(np.int16)).cuda()
        keep += [fr, fd]
        req = R.request(sid, int(rgb.ref_index[j]), R.RGB | R.DEPTH | R.CLEAN, on_device=on_device,
                        rgb=(fr, rgb.height, rgb.width), depth=(fd, dep.height, dep.width))
        ctx.poll(ctx.submit(req))
    return keep


class Outputs:
    def __init__(self, rgb, dep, on_device=True):
        self.on_device = on_device
        if on_device:
            self.rgb_in = torch.from_numpy(rgb.decoded).cuda()
            self.dep_in = torch.from_numpy(dep.decoded.view(np.int16)).cuda()
            self.rgb_mask = torch.from_numpy(rgb.mask.view(np.int32)).cuda()
            self.dep_mask = torch.from_numpy(dep.mask.view(np.int32)).cuda()
            self.rgb_out = torch.zeros(rgb.decoded.shape, dtype=torch.uint8, device="cuda")
            self.dep_out = torch.zeros(dep.decoded.shape, dtype=torch.int16, device="cuda")
            self.rgb_val = torch.zeros(rgb.decoded.shape, dtype=torch.float32, device="cuda")
            self.dep_val = torch.zeros(dep.decoded.shape, dtype=torch.float32, device="cuda")
        else:
            self.rgb_in, self.dep_in = rgb.decoded, dep.decoded
            self.rgb_mask, self.dep_mask = rgb.mask, dep.mask
            self.rgb_out = np.zeros(rgb.decoded.shape, np.uint8)
            self.dep_out = np.zeros(dep.decoded.shape, np.uint16)
            self.rgb_val = np.zeros(rgb.decoded.shape, np.float32)
            self.dep_val = np.zeros(dep.decoded.shape, np.float32)

    def request(self, sid, rgb, dep):
        return R.request(sid, rgb.index, R.RGB | R.DEPTH, on_device=self.on_device,
                         rgb=(self.rgb_in, rgb.height, rgb.width), rgb_mask=self.rgb_mask,
                         depth=(self.dep_in, dep.height, dep.width), depth_mask=self.dep_mask,
                         rgb_out=self.rgb_out, depth_out=self.dep_out, rgb_values=self.rgb_val,
                         depth_values=self.dep_val)

    def numpy(self):
        def cv(t):
            return t.cpu().numpy() if isinstance(t, torch.Tensor) else t
        return (cv(self.rgb_out), cv(self.dep_out).view(np.uint16), cv(self.rgb_val), cv(self.dep_val))


def run(ctx, sid, rgb, dep, on_device=True):
    keep = push_refs(ctx, sid, rgb, dep, on_device)
    o = Outputs(rgb, dep, on_device)
    res = ctx.poll(ctx.submit(o.request(sid, rgb, dep)))
    assert res.status == R.REVO_OK
    del keep
    return o.numpy()


_ORACLE = {}


def oracle(shape, rgb, dep, key):
    if key not in _ORACLE:
        out = []
        for mod, pl, C in (("rgb", rgb, 3), ("depth", dep, 1)):
            out.append(O.recover(mod, weights(shape, C), model_cfg(shape, C), pl.refs, pl.ref_index, pl.decoded,
                                 pl.mask, pl.index))
        _ORACLE[key] = out
    return _ORACLE[key]


def psnr(err, peak):
    mse = float(np.mean(np.square(err)))
    return np.inf if mse == 0 else 10 * np.log10(peak * peak / mse)


def check(precision, got, ref, rgb, dep, report=None):
    g_rgb, g_dep, v_rgb, v_dep = got
    (c_rgb, o_rgb), (c_dep, o_dep) = ref
    e_rgb = v_rgb.astype(np.float64) - o_rgb
    e_dep = v_dep.astype(np.float64) - o_dep
    stats = dict(rgb_max=float(np.abs(e_rgb).max()), dep_max_mm=float(np.abs(e_dep).max()),
                 rgb_psnr=psnr(e_rgb, 1.0), dep_psnr=psnr(e_dep / 65535.0, 1.0),
                 rgb_psnr_lost=psnr(e_rgb[rgb.lost], 1.0) if rgb.lost.any() else np.inf)
    if report is not None:
        report.update(stats)
    print(f"parity precision={precision}", {k: round(float(v), 6) for k, v in stats.items()})
    if precision == R.FP32:
        tol_rgb, tol_dep = 1e-4, 1.0
        assert stats["rgb_max"] <= tol_rgb, stats
        assert stats["dep_max_mm"] <= tol_dep, stats
    else:
        tol_rgb, tol_dep = None, 8.0
        assert stats["rgb_psnr"] >= 45.0, stats
        assert stats["dep_psnr"] >= 45.0, stats
        assert stats["dep_max_mm"] <= tol_dep, stats
    # Blended codes.
    for g, c, o, pl, scale, tol in ((g_rgb, c_rgb, o_rgb, rgb, 255.0, e_rgb), (g_dep, c_dep, o_dep, dep, 1.0, e_dep)):
        np.testing.assert_array_equal(g[~pl.lost], pl.decoded[~pl.lost])
        lost = pl.lost if o.ndim == 2 else np.repeat(pl.lost[..., None], o.shape[-1], axis=-1)
        d = np.abs(g.astype(np.int64) - c.astype(np.int64))
        # |rint(v) - rint(o)| <= floor(|v - o|) + 1 for the float values v (GPU) and o (oracle)
        bound = np.floor(np.abs(tol) * scale) + 1
        assert (d[lost] <= bound[lost]).all()
        # away from a rounding boundary (by more than the observed error plus the
        # float32 rounding of the kernel's v * scale) the codes agree exactly
        frac = np.abs((o * scale) - np.floor(o * scale) - 0.5)
        margin = np.abs(tol) * scale + np.abs(o * scale) * 2.0 ** -22 + 1e-6
        safe = lost & (frac > margin)
        np.testing.assert_array_equal(g[safe], c[safe])
    return stats


# ------------------------------------------------------------------ tests

@pytest.mark.parametrize("precision", [0, 1])
def test_small_network_parity(precision):
    rgb, dep = synth.make_request(11, "320x240")
    rgb = synth.make_tiny_plane(21, "rgb", 64, 96, 5)
    dep = synth.make_tiny_plane(22, "depth", 64, 96, 5)
    with make_ctx(SMALL, precision, (64, 96)) as ctx:
        got = run(ctx, 0, rgb, dep)
    check(precision, got, oracle(SMALL, rgb, dep, "small"), rgb, dep)


@pytest.mark.parametrize("pattern", ["none_lost", "all_lost"])
def test_small_network_degenerate_masks(pattern):
    """The mask's two degenerate cases through the whole path: nothing lost
    (every output code is the decoded frame's, bit for bit) and every pixel
    lost (the decoded frame is all zeros and every code is the network's)."""
    H, W = 64, 96
    rows = [] if pattern == "none_lost" else list(range(H))
    rgb = synth.make_tiny_plane(31, "rgb", H, W, 5, lost_rows=rows)
    dep = synth.make_tiny_plane(32, "depth", H, W, 5, lost_rows=rows)
    assert rgb.lost.all() == (pattern == "all_lost") and rgb.lost.any() == (pattern == "all_lost")
    with make_ctx(SMALL, 1, (H, W)) as ctx:
        got = run(ctx, 0, rgb, dep)
    ref = oracle(SMALL, rgb, dep, "small-" + pattern)
    check(1, got, ref, rgb, dep)
    if pattern == "none_lost":
        np.testing.assert_array_equal(got[0], rgb.decoded)
        np.testing.assert_array_equal(got[1], dep.decoded)
    else:
        assert not rgb.decoded.any() and not dep.decoded.any()
        # The oracle's codes for a fully lost frame are its quantised values.
        np.testing.assert_array_equal(ref[0][0], O.quantise_rgb(ref[0][1]))
        np.testing.assert_array_equal(ref[1][0], O.quantise_depth(ref[1][1]))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_vitb_320x240_parity(precision):
    rgb, dep = synth.make_request(1001, "320x240")
    with make_ctx(VITB, precision, (240, 320)) as ctx:
        got = run(ctx, 0, rgb, dep)
    check(precision, got, oracle(VITB, rgb, dep, "320"), rgb, dep)


@pytest.mark.parametrize("precision", [1, 0, 2])
def test_vitb_640x480_parity(precision):
    rgb, dep = synth.make_request(2001, "640x480", loss_rate=0.2)
    with make_ctx(VITB, precision, (480, 640)) as ctx:
        got = run(ctx, 0, rgb, dep)
    check(precision, got, oracle(VITB, rgb, dep, "640"), rgb, dep)


# The 1280x720 RGB + 640x576 depth request shared by the decoupled-size test
# and the mixed batch below (one oracle run serves both).
SEED_720 = 3001


@pytest.mark.parametrize("precision", [1, 2])
def test_vitb_1280x720_rgb_640x576_depth_parity(precision):
    """Decoupled streams at different sizes (Section 3.4.2: a model per
    modality): 1280x720 RGB (N = 10800 tokens) with a 640x576 depth stream
    (N = 4320; 300-5000 mm, 2% invalid zero pixels), 20% bursty slice loss,
    BF16 and FP8 against the FP64 oracle."""
    rgb, dep = synth.make_request(SEED_720, "1280x720+640x576", loss_rate=0.2)
    assert (rgb.height, rgb.width, dep.height, dep.width) == (720, 1280, 576, 640)
    assert (dep.clean == 0).mean() > 0.01
    with make_ctx(VITB, precision, (720, 1280)) as ctx:
        got = run(ctx, 0, rgb, dep)
    check(precision, got, oracle(VITB, rgb, dep, "720"), rgb, dep)


def test_host_buffers_match_device_buffers():
    rgb, dep = synth.make_request(1002, "320x240")
    with make_ctx(VITB, R.BF16, (240, 320)) as ctx:
        a = run(ctx, 0, rgb, dep, on_device=True)
        b = run(ctx, 1, rgb, dep, on_device=False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_batch_result_equals_alone():
    """Requests fused into one launch give exactly what each gives alone."""
    reqs = [synth.make_request(1003, "320x240"), synth.make_request(2003, "640x480", loss_rate=0.1),
            synth.make_request(1004, "320x240")]
    alone = []
    with make_ctx(VITB, R.BF16, (480, 640), max_streams=4) as ctx:
        for sid, (rgb, dep) in enumerate(reqs):
            alone.append(run(ctx, sid, rgb, dep))
    with make_ctx(VITB, R.BF16, (480, 640), max_batch=3, max_streams=4) as ctx:
        keep = [push_refs(ctx, sid, rgb, dep) for sid, (rgb, dep) in enumerate(reqs)]
        outs = [Outputs(rgb, dep) for rgb, dep in reqs]
        # REVO_HOLD on the first two: all three are admitted into one batch
        tickets = []
        for sid, o in enumerate(outs):
            r = o.request(sid, *reqs[sid])
            if sid < 2:
                r.flags |= R.HOLD
            tickets.append(ctx.submit(r))
        sizes = [ctx.poll(t).batch_size for t in tickets]
        del keep
    assert sizes == [3, 3, 3]
    for a, o in zip(alone, outs):
        for x, y in zip(a, o.numpy()):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_replay_equals_plain_launches(precision):
    """With graph replay on, a size pattern runs eagerly, is then captured, then
    replayed; every run reads its own requests' frames, masks and temporal
    distances (new content each time, same sizes) and gives exactly what plain
    launches give.  At BF16 and FP8 the graph path embeds the tubelets with the
    implicit GEMM (frames read in the GEMM's producer) and the plain path with
    the assemble kernel + GEMM: the same operands and K order, so the same
    bits."""
    shape = SMALL if precision == 0 else VITB
    rounds = [[synth.make_request(3000 + 10 * it + j, wl, index=40 + it, delta=1 + (it + j) % 3)
               for j, wl in enumerate(("320x240", "640x480", "320x240"))] for it in range(4)]
    got = {}
    for graphs in (0, 1):
        with make_ctx(shape, precision, (480, 640), max_batch=3, max_streams=3, use_graphs=graphs) as ctx:
            for it, reqs in enumerate(rounds):
                keep = [push_refs(ctx, sid, rgb, dep) for sid, (rgb, dep) in enumerate(reqs)]
                outs = [Outputs(rgb, dep) for rgb, dep in reqs]
                tickets = [ctx.submit(o.request(sid, *reqs[sid])) for sid, o in enumerate(outs)]
                ctx.flush()
                for t in tickets:
                    assert ctx.poll(t).status == R.REVO_OK
                del keep
                got[graphs, it] = [o.numpy() for o in outs]
    for it in range(len(rounds)):
        for a, b in zip(got[0, it], got[1, it]):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
    # the content differs from round to round, so a stale argument table would show
    assert not np.array_equal(got[1, 2][0][0], got[1, 3][0][0])


def test_hold_batches_mixed_sizes_with_autotuned_tiles():
    """REVO_HOLD admits requests without launching; the batch starts when it is
    full.  Tile widths chosen by the autotuner leave every output unchanged (a
    tile width changes which CTA computes an element, not its arithmetic)."""
    reqs = [synth.make_request(SEED_720 if wl.startswith("1280") else 3100 + i, wl, loss_rate=0.2)
            for i, wl in enumerate(("640x480", "320x240", "1280x720+640x576", "320x240"))]
    got = {}
    for tune in (0, 1):
        with make_ctx(VITB, R.BF16, (720, 1280), max_batch=4, max_streams=4, use_graphs=1, autotune=tune) as ctx:
            keep = [push_refs(ctx, sid, rgb, dep) for sid, (rgb, dep) in enumerate(reqs)]
            for rep in range(3):
                outs = [Outputs(rgb, dep) for rgb, dep in reqs]
                tickets = []
                for sid, o in enumerate(outs):
                    r = o.request(sid, *reqs[sid])
                    r.flags |= R.HOLD
                    tickets.append(ctx.submit(r))
                    if sid < len(outs) - 1:
                        assert ctx.stats()["pending"] == sid + 1
                res = [ctx.poll(t) for t in tickets]
                assert all(x.status == R.REVO_OK and x.batch_size == 4 for x in res)
                got[tune, rep] = [o.numpy() for o in outs]
            st = ctx.stats()
            del keep
        assert st["batches"] == 3 and st["pending"] == 0 and st["in_flight"] == 0
        assert st["graphs_captured"] == 2 and st["graph_replays"] == 4  # 2 modalities x (capture, replay)
        assert (st["tuned_shapes"] > 0) == bool(tune)
    for rep in range(3):
        for a, b in zip(got[0, rep], got[1, rep]):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
    # the mixed batch equals the 640x480 request alone
    with make_ctx(VITB, R.BF16, (480, 640)) as ctx:
        alone = run(ctx, 0, *reqs[0])
    for x, y in zip(alone, got[1, 2][0]):
        np.testing.assert_array_equal(x, y)
    # and its 1280x720 + 640x576 member matches the FP64 oracle
    check(R.BF16, got[1, 2][2], oracle(VITB, *reqs[2], "720"), *reqs[2])


@pytest.mark.parametrize("k,T", [(3, 1), (7, 2), (1, 2)])
def test_k_and_tubelet_variants(k, T):
    """Other reference counts and tubelet sizes (the paper's ablation over k
    and T, Section 4 / Appendix B.3) through the same kernels, BF16 against
    the FP64 oracle at 320x240; the graph path (implicit-GEMM embedding over
    k + 1 frames in slots of T) gives the plain path's bits."""
    shape = dict(VITB, k=k, tubelet=T)
    rgb, dep = synth.make_request(1200 + 10 * k + T, "320x240", k=k)
    got = {}
    for graphs in (0, 1):
        with make_ctx(shape, R.BF16, (240, 320), use_graphs=graphs) as ctx:
            got[graphs] = run(ctx, 0, rgb, dep)
    for x, y in zip(got[0], got[1]):
        np.testing.assert_array_equal(x, y)
    check(R.BF16, got[1], oracle(shape, rgb, dep, f"kt{k}{T}"), rgb, dep)


def test_unaligned_current_frame():
    """The current frame read straight from the caller's device buffers at
    addresses that are only 4-byte (RGB) and 2-byte (depth) aligned: the
    implicit-GEMM embedding, the assemble kernel and the blend take their
    narrow-load paths, and the graph path still gives the plain path's bits
    (twice: the eager run and the captured replay)."""
    rgb, dep = synth.make_request(3500, "320x240", loss_rate=0.2)
    got = {}
    for graphs in (0, 1):
        with make_ctx(VITB, R.BF16, (240, 320), use_graphs=graphs) as ctx:
            keep = push_refs(ctx, 0, rgb, dep)
            rbuf = torch.zeros(rgb.decoded.size + 16, dtype=torch.uint8, device="cuda")
            rbuf[4:4 + rgb.decoded.size] = torch.from_numpy(rgb.decoded.reshape(-1)).cuda()
            dbuf = torch.zeros(dep.decoded.size + 8, dtype=torch.int16, device="cuda")
            dbuf[1:1 + dep.decoded.size] = torch.from_numpy(dep.decoded.reshape(-1).view(np.int16)).cuda()
            for rep in range(2):
                o = Outputs(rgb, dep)
                req = o.request(0, rgb, dep)
                req.rgb.data = rbuf.data_ptr() + 4
                req.depth.data = dbuf.data_ptr() + 2
                assert ctx.poll(ctx.submit(req)).status == R.REVO_OK
                got[graphs, rep] = o.numpy()
            del keep
    for rep in range(2):
        for x, y in zip(got[0, rep], got[1, rep]):
            np.testing.assert_array_equal(x, y)
    with make_ctx(VITB, R.BF16, (240, 320)) as ctx:
        aligned = run(ctx, 0, rgb, dep)
    for x, y in zip(aligned, got[1, 1]):
        np.testing.assert_array_equal(x, y)


def test_two_lanes_interleaved_streams():
    reqs = [synth.make_request(1010 + i, "320x240") for i in range(4)]
    alone = []
    with make_ctx(VITB, R.BF16, (240, 320)) as ctx:
        for sid, (rgb, dep) in enumerate(reqs):
            alone.append(run(ctx, sid, rgb, dep))
    with make_ctx(VITB, R.BF16, (240, 320), max_batch=2, lanes=2) as ctx:
        keep = [push_refs(ctx, sid, rgb, dep) for sid, (rgb, dep) in enumerate(reqs)]
        outs = [Outputs(rgb, dep) for rgb, dep in reqs]
        tickets = [ctx.submit(o.request(sid, *reqs[sid])) for sid, o in enumerate(outs)]
        for t in tickets[::-1]:
            assert ctx.poll(t).status == R.REVO_OK
        del keep
    for a, o in zip(alone, outs):
        for x, y in zip(a, o.numpy()):
            np.testing.assert_array_equal(x, y)


def test_frames_in_flight_reuse_batch_resources():
    """Two lanes with two frames in flight and clean-frame pushes in between:
    retired batches hand their events and pinned error words to later ones
    (copy-only batches of clean frames included), and every frame still
    equals the same frame recovered alone, bit for bit."""
    reqs = [synth.make_request(1040 + i, "320x240") for i in range(4)]
    alone = []
    with make_ctx(VITB, R.BF16, (240, 320)) as ctx:
        for sid, (rgb, dep) in enumerate(reqs):
            alone.append(run(ctx, sid, rgb, dep))
    with make_ctx(VITB, R.BF16, (240, 320), lanes=2, use_graphs=1) as ctx:
        keep = [push_refs(ctx, sid, *reqs[sid]) for sid in (0, 1)]
        outs = [Outputs(rgb, dep) for rgb, dep in reqs]
        inflight = []

        def submit(sid):
            inflight.append(ctx.submit(outs[sid].request(sid, *reqs[sid])))
            if len(inflight) == 2:
                assert ctx.poll(inflight.pop(0)).status == R.REVO_OK

        for i in range(6):  # streams 0 and 1 only, two in flight
            submit(i % 2)
        keep += [push_refs(ctx, sid, *reqs[sid]) for sid in (2, 3)]  # copy-only batches while one is in flight
        for i in range(12):
            submit(i % 4)
        while inflight:
            assert ctx.poll(inflight.pop(0)).status == R.REVO_OK
        st = ctx.stats()
        assert st["pending"] == 0 and st["in_flight"] == 0
        del keep
    for a, o in zip(alone, outs):
        for x, y in zip(a, o.numpy()):
            np.testing.assert_array_equal(x, y)


def test_temporal_distance_reaches_the_network():
    """Same references at a larger distance to the target (Section 3.4.1) give
    another output, matching the oracle's."""
    rgb, dep = synth.make_request(1005, "320x240", index=100, delta=3)
    with make_ctx(SMALL, R.FP32, (240, 320)) as ctx:
        got = run(ctx, 0, rgb, dep)
    check(R.FP32, got, oracle(SMALL, rgb, dep, "delta3"), rgb, dep)
    rgb1, dep1 = synth.make_request(1005, "320x240", index=100, delta=1)
    assert not np.array_equal(rgb1.ref_index, rgb.ref_index)


def test_error_statuses():
    rgb, dep = synth.make_request(1006, "320x240")
    with make_ctx(SMALL, R.BF16, (240, 320)) as ctx:
        o = Outputs(rgb, dep)
        with pytest.raises(R.RevoError) as ei:
            ctx.submit(o.request(0, rgb, dep))
        assert ei.value.status == R.REVO_ENOREF
        with pytest.raises(R.RevoError) as ei:
            ctx.poll(12345, 0)
        assert ei.value.status == R.REVO_EINVAL
        keep = push_refs(ctx, 0, rgb, dep)
        small = synth.make_tiny_plane(3, "rgb", 64, 96, 5)
        req = R.request(0, 200, R.RGB, on_device=True, rgb=(o.rgb_in, 64, 96), rgb_mask=o.rgb_mask,
                        rgb_out=o.rgb_out)
        with pytest.raises(R.RevoError) as ei:
            ctx.submit(req)   # frame size differs from the stream's references
        assert ei.value.status == R.REVO_EINVAL
        req = R.request(9, 200, R.RGB, on_device=True, rgb=(o.rgb_in, 240, 320), rgb_mask=o.rgb_mask,
                        rgb_out=o.rgb_out)
        with pytest.raises(R.RevoError) as ei:
            ctx.submit(req)   # stream id beyond max_streams
        assert ei.value.status == R.REVO_EINVAL
        t = ctx.submit(o.request(0, rgb, dep))
        assert ctx.poll(t).status == R.REVO_OK
        del keep, small


def test_weights_from_seed_and_file_equal_the_arrays(tmp_path):
    """A context whose models come from a seed (revo_init_weights' random
    initialisation) or from flat float32 files computes exactly what the same
    weights passed as arrays give."""
    rgb, dep = synth.make_tiny_plane(31, "rgb", 64, 96, 5), synth.make_tiny_plane(32, "depth", 64, 96, 5)
    with make_ctx(SMALL, R.BF16, (64, 96)) as ctx:
        want = run(ctx, 0, rgb, dep)
    cfg = R.config(**SMALL, precision=R.BF16, max_height=64, max_width=96, max_streams=4, seed=0, random_init=3)
    with R.Context(cfg) as ctx:
        got_seed = run(ctx, 0, rgb, dep)
    paths = []
    for C, seed in ((3, 0), (1, 1)):
        p = tmp_path / f"w{C}.bin"
        synth.flatten(weights(SMALL, C)).tofile(p)
        paths.append(str(p))
    cfg = R.config(**SMALL, precision=R.BF16, max_height=64, max_width=96, max_streams=4,
                   rgb_weights_path=paths[0], depth_weights_path=paths[1])
    with R.Context(cfg) as ctx:
        got_file = run(ctx, 0, rgb, dep)
    for a, b, c in zip(want, got_seed, got_file):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)


def test_autotune_cache_file_round_trip(tmp_path):
    """With autotune on, create times every GEMM shape and writes the cache
    file; a second context reads it and times nothing; both give the same
    outputs as a context without tuning (a tile choice never changes results)."""
    cache = str(tmp_path / "tiles.txt")
    rgb, dep = synth.make_request(1020, "320x240")
    outs, tuned = [], []
    for tune, path in ((0, None), (1, cache), (1, cache)):
        kw = dict(autotune_cache=path) if path else {}
        cfg = R.config(**VITB, precision=R.BF16, max_height=240, max_width=320, max_streams=2, autotune=tune, **kw)
        with R.Context(cfg, synth.flatten(weights(VITB, 3)), synth.flatten(weights(VITB, 1))) as ctx:
            outs.append(run(ctx, 0, rgb, dep))
            st = ctx.stats()
            tuned.append((st["tuned_shapes"], st["tuned_timed"]))
        if tune:
            lines = open(cache).read().splitlines()
            assert lines[0].startswith("revo-autotune 1 sm_10")
            assert len(lines) - 1 == st["tuned_shapes"] > 0
    assert tuned[0][0] == 0 and tuned[1][0] == tuned[2][0]
    assert tuned[1][1] == tuned[1][0] and tuned[2][1] == 0   # the second context timed nothing
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            np.testing.assert_array_equal(x, y)


def test_serial_models_equal_concurrent_models():
    """serial_models runs a batch's RGB forward before its depth forward
    instead of beside it: the outputs are the same bit for bit."""
    reqs = [synth.make_request(1030 + i, "320x240") for i in range(3)]
    got = {}
    for serial in (0, 1):
        cfg = R.config(**VITB, precision=R.BF16, max_height=240, max_width=320, max_streams=3, max_batch=3,
                       serial_models=serial)
        with R.Context(cfg, synth.flatten(weights(VITB, 3)), synth.flatten(weights(VITB, 1))) as ctx:
            keep = [push_refs(ctx, sid, rgb, dep) for sid, (rgb, dep) in enumerate(reqs)]
            outs = [Outputs(rgb, dep) for rgb, dep in reqs]
            tickets = []
            for sid, o in enumerate(outs):
                r = o.request(sid, *reqs[sid])
                r.flags |= R.HOLD if sid < 2 else 0
                tickets.append(ctx.submit(r))
            assert all(ctx.poll(t).batch_size == 3 for t in tickets)
            got[serial] = [o.numpy() for o in outs]
            del keep
    for a, b in zip(got[0], got[1]):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
