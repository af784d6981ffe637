#!/usr/bin/env python
"""Benchmark of the ReVo neural loss-recovery hot path on B300.

One step = recovery of one corrupted RGB-D frame (640x480 RGB uint8 +
640x480 depth uint16, batch 1): tubelet assembly + normalisation, the ViT-B
encoder-decoder forward of both modality models (run concurrently on two CUDA
streams), the pixel head and the masked blend, through the library's C ABI
(revo_recover_submit + revo_recover_poll).  Four conference streams, one per
Gilbert-Elliott slice-loss rate (5/10/20/40 %), each with five clean
references resident on the device, take turns.  Random-init weights and
seeded synthetic frames.  Two frames are kept in flight (--in-flight, one
lane each), as a receiver serving several conference streams would: each
frame is still its own batch-1 launch, and its latency (submit -> poll) is
reported against the 33 ms frame budget.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle, same metric

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "recovered RGB-D frames/s + p99 latency, BF16/FP8 vs FP32, at ≥45 dB vs FP64 oracle"
UNIT = "frames/s"
WORKLOAD = "640x480"
H, W = 480, 640
LOSS_RATES = (0.05, 0.10, 0.20, 0.40)
VITB = dict(k=5, tubelet=2, patch=16, enc_dim=768, enc_depth=12, enc_heads=12, dec_dim=384, dec_depth=4,
            dec_heads=6, mlp_ratio=4)
FRAME_BUDGET_MS = 33.0
PRECISIONS = {"bf16": lambda R: R.BF16, "fp32": lambda R: R.FP32, "fp8": lambda R: R.FP8}
DTYPE_NAMES = {"bf16": "bf16", "fp32": "f32", "fp8": "e4m3 (encoder fc1; per-token x per-channel scales) + bf16"}
# DRAM bytes (read + write) of one attn_tc_kernel launch at N = 3600, 12 heads,
# from an ncu capture of the current kernel version (None once it changes).
ATTN_DRAM_BYTES_PER_LAUNCH = 16629760


def run_pipelined(R, ctx, req_list, n: int, depth: int, start: int = 0):
    """Submits requests start .. start+n-1 (cycling through req_list) keeping
    up to `depth` in flight, polls each in submission order; returns the
    per-frame latencies (ms, submit -> poll return) and the kernel launches."""
    import collections
    q = collections.deque()
    lat, launches = [], 0

    def retire():
        nonlocal launches
        tk, ts = q.popleft()
        res = ctx.poll(tk)
        if res.status != R.REVO_OK:
            raise RuntimeError(f"recovery failed: {R.STATUS_NAMES.get(res.status)} {R.last_error()}")
        lat.append((time.perf_counter() - ts) * 1e3)
        launches += res.kernel_launches

    for i in range(n):
        q.append((ctx.submit(req_list[(start + i) % len(req_list)]), time.perf_counter()))
        if len(q) >= depth:
            retire()
    while q:
        retire()
    return lat, launches


def workload_config(world: int, seq_len: int) -> dict:
    """The headline workload, as both arms name it in `config`."""
    return {"workload": f"{WORKLOAD} RGB uint8 + {WORKLOAD} depth uint16, batch 1, "
                        "loss 5/10/20/40% (4 streams in turn)",
            "model": "ViT-B enc-dec (768x12 / 384x4), k=5, T=2, p=16", "global_batch": world,
            "seq_len": seq_len, "parallelism": f"replicas x{world}"}


def flops_per_model(C: int, h: int, w: int) -> dict:
    """Algorithmic FLOPs of one forward (2 per multiply-add), exact savings applied:
    the pixel head runs on the target frame's rows of the last slot only."""
    k, T, p, D, L, Dd, Ld, r = 5, 2, 16, 768, 12, 384, 4, 4
    P = (h // p) * (w // p)
    N = (k + 1) // T * P
    Kt = T * C * p * p
    lin = 2 * N * Kt * D
    lin += L * 2 * N * (3 * D * D + D * D + 2 * r * D * D)
    lin += 2 * N * D * Dd
    lin += Ld * 2 * N * (3 * Dd * Dd + Dd * Dd + 2 * r * Dd * Dd)
    lin += 2 * P * Dd * (C * p * p)
    attn_enc = 4 * N * N * D
    attn_dec = 4 * N * N * Dd
    return dict(N=N, linear=lin, attn_enc_per_block=attn_enc, attn=L * attn_enc + Ld * attn_dec,
                total=lin + L * attn_enc + Ld * attn_dec)


def peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- ranks --
# One process per GPU; the recovery path shards by conference stream with no
# exchange, so ranks only meet for barriers and the max of their timings.

def rank_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_max(v: float, world: int) -> float:
    """Max of a scalar over ranks (CUDA tensor under NCCL, CPU under gloo)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps_per_rank: int, max_seconds: float, world: int) -> float:
    """Frames/s of the whole job: every rank's frames over the slowest rank's time."""
    return world * steps_per_rank / max_seconds


# --------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle arm --

def oracle_rgb_sample(seed: int = 2002):
    """Times the FP64 oracle recovering the RGB plane of one 640x480 frame (the
    bounded sample); returns (seconds, the oracle's values, the plane)."""
    import synth
    from oracle import revo_oracle as O
    rgb, _ = synth.make_request(seed, WORKLOAD, loss_rate=0.2)
    w = synth.weights(synth.RGB, seed=0)
    t0 = time.perf_counter()
    codes, values = O.recover("rgb", w, synth.RGB, rgb.refs, rgb.ref_index, rgb.decoded, rgb.mask, rgb.index)
    return time.perf_counter() - t0, values, rgb


def cpu_baseline(seconds_rgb: float) -> dict:
    f_rgb = flops_per_model(3, H, W)["total"]
    f_dep = flops_per_model(1, H, W)["total"]
    per_frame = seconds_rgb * (f_rgb + f_dep) / f_rgb
    return {"value": 1.0 / per_frame, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle recovering the RGB plane of one {WORKLOAD} frame "
                      f"({seconds_rgb:.1f} s), scaled to an RGB-D frame by the FLOP ratio "
                      f"{(f_rgb + f_dep) / f_rgb:.3f}"}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import revo_oracle as O
    import synth
    # Each step: one oracle encoder block of the RGB model on the token count
    # of a 320x240 frame (N = 900; a bounded sample, ~0.3-0.5 s on 8 cores, so
    # the default 210 steps end within minutes); a 640x480 RGB-D frame costs
    # `blocks_per_frame` such blocks by FLOP count.  At N = 900 the attention
    # share is smaller than at N = 3600, where the oracle's per-FLOP speed is
    # lower (softmax), so the scaled figure favours the CPU.
    fr = flops_per_model(3, H, W)
    fd = flops_per_model(1, H, W)
    N, D = flops_per_model(3, 240, 320)["N"], 768
    block_flops = 2 * N * (3 * D * D + D * D + 8 * D * D) + 4 * N * N * D
    blocks_per_frame = (fr["total"] + fd["total"]) / block_flops
    cfg = synth.RGB
    w = {n: a.astype(np.float64) for n, a in synth.weights(cfg, seed=0).items() if n.startswith("enc.0.")}
    x = synth.normal(7, (N, D)).astype(np.float64)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.block(x, w, "enc.0.", cfg.enc_heads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per_frame = statistics.mean(times) * blocks_per_frame
    value = 1.0 / per_frame
    sample = (f"per step one FP64 oracle encoder block at N={N} tokens; an RGB-D frame = "
              f"{blocks_per_frame:.2f} such blocks by FLOP count")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(1, flops_per_model(3, H, W)["N"]),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# -------------------------------------------------------------- our arm --

def elementwise_roofline(R, torch, stream) -> dict:
    """The HBM-bound stages alone at the largest frame of the workloads (1280x720
    RGB): the fused unpack + normalise + tubelet gather (assemble) and the
    de-normalise + masked blend.  L2 is flushed (a 256 MB write, then a read of
    it) before every timed launch; achieved = algorithmic bytes / CUDA-event
    time."""
    Hh, Ww, k, T, p = 720, 1280, 5, 2, 16
    frame = Hh * Ww * 3
    refs = [torch.randint(0, 256, (Hh, Ww, 3), dtype=torch.uint8, device="cuda") for _ in range(k)]
    cur = torch.randint(0, 256, (Hh, Ww, 3), dtype=torch.uint8, device="cuda")
    P = (Hh // p) * (Ww // p)
    tokens = torch.empty(((k + 1) // T * P, T * 3 * p * p), dtype=torch.bfloat16, device="cuda")
    head = torch.randn((P, 3 * p * p), device="cuda")
    mask = torch.randint(-2 ** 31, 2 ** 31 - 1, (Hh, (Ww + 31) // 32), dtype=torch.int32, device="cuda")
    out = torch.empty((Hh, Ww, 3), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_sum = torch.zeros((), dtype=torch.int64, device="cuda")
    stats = torch.zeros(2, device="cuda")

    def timed(fn, reps=10):
        tot = 0.0
        for i in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                # Evict the operands: write a buffer larger than L2, then read
                # it, so the lines left in L2 are clean and the timed launch
                # does not pay for writing back the flush's dirty lines.
                flush.fill_(i & 255)
                flush_sum.copy_(flush.view(torch.int64).sum())
                e0.record(stream)
                fn()
                e1.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                tot += e0.elapsed_time(e1) * 1e3
        return tot / reps

    us_a = timed(lambda: R.op_assemble(3, k, T, p, Hh, Ww, refs, cur, Ww * 3, stats, tokens, 1, stream=stream))
    us_b = timed(lambda: R.op_blend(3, p, Hh, Ww, head, cur, Ww * 3, mask, (Ww + 31) // 32, stats, out, Ww * 3,
                                    stream=stream))
    bytes_a = (k + 1) * frame + tokens.numel() * 2
    bytes_b = head.numel() * 4 + frame + mask.numel() * 4 + frame
    hbm = peaks().get("hbm_gbs")
    mk = lambda us, b: {"us": us, "bytes": b, "gbs": b / us / 1e3,  # noqa: E731
                        "frac_of_measured_hbm": (b / us / 1e3 / hbm) if hbm else None}
    return {"assemble_rgb_1280x720": mk(us_a, bytes_a), "blend_rgb_1280x720": mk(us_b, bytes_b),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if hbm else None}


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2604_27441_b300 as R
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        rank_barrier(world)

    def max_over_ranks(v: float) -> float:
        return rank_max(v, world)

    precision = PRECISIONS[args.precision](R)
    stream = torch.cuda.Stream()
    w_rgb = synth.flatten(synth.weights(synth.RGB, seed=0))
    w_dep = synth.flatten(synth.weights(synth.DEPTH, seed=1))
    depth = max(1, min(8, args.in_flight))  # frames in flight, one lane each
    cfg = R.config(**VITB, precision=precision, device=local, max_height=H, max_width=W, max_streams=8,
                   max_batch=1, lanes=depth, use_graphs=0 if args.no_graphs else 1, autotune=1)
    ctx = R.Context(cfg, w_rgb, w_dep, stream=stream)

    # Four conference streams (one per loss rate), references pushed once.
    reqs = [synth.make_request(2000 + 100 * rank + i, WORKLOAD, loss_rate=r) for i, r in enumerate(LOSS_RATES)]
    keep = []
    dev_req, host_req, dev_bufs = [], [], []
    for sid, (rgb, dep) in enumerate(reqs):
        for j in range(rgb.refs.shape[0]):
            fr = torch.from_numpy(rgb.refs[j]).cuda()
            fd = torch.from_numpy(dep.refs[j].view(np.int16)).cuda()
            keep += [fr, fd]
            ctx.poll(ctx.submit(R.request(sid, int(rgb.ref_index[j]), R.RGB | R.DEPTH | R.CLEAN, on_device=True,
                                          rgb=(fr, H, W), depth=(fd, H, W))))
        d = dict(ri=torch.from_numpy(rgb.decoded).cuda(), di=torch.from_numpy(dep.decoded.view(np.int16)).cuda(),
                 rm=torch.from_numpy(rgb.mask.view(np.int32)).cuda(), dm=torch.from_numpy(dep.mask.view(np.int32)).cuda(),
                 ro=torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda"),
                 do=torch.zeros((H, W), dtype=torch.int16, device="cuda"),
                 rv=torch.zeros((H, W, 3), dtype=torch.float32, device="cuda"))
        keep.append(d)
        dev_bufs.append(d)
        dev_req.append(R.request(sid, rgb.index, R.RGB | R.DEPTH, on_device=True, rgb=(d["ri"], H, W),
                                 rgb_mask=d["rm"], depth=(d["di"], H, W), depth_mask=d["dm"], rgb_out=d["ro"],
                                 depth_out=d["do"], rgb_values=d["rv"] if sid == 2 else None))
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        h = dict(ri=pin(rgb.decoded), di=pin(dep.decoded.view(np.int16)), rm=pin(rgb.mask.view(np.int32)),
                 dm=pin(dep.mask.view(np.int32)), ro=torch.zeros((H, W, 3), dtype=torch.uint8).pin_memory(),
                 do=torch.zeros((H, W), dtype=torch.int16).pin_memory())
        keep.append(h)
        host_req.append(R.request(sid, rgb.index, R.RGB | R.DEPTH, on_device=False, rgb=(h["ri"], H, W),
                                  rgb_mask=h["rm"], depth=(h["di"], H, W), depth_mask=h["dm"], rgb_out=h["ro"],
                                  depth_out=h["do"]))
    h2d = H * W * 3 + H * W * 2 + 2 * H * ((W + 31) // 32) * 4
    d2h = H * W * 3 + H * W * 2

    run_pipelined(R, ctx, dev_req, args.warmup, depth)
    torch.cuda.synchronize()
    barrier()

    # Timed region: device-resident inputs and outputs.
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, launches = [], 0
    # REVO_PROFILE_RANGE=1 marks the timed region for a profiler started with
    # --profile-from-start off (it changes nothing else).
    mark = os.environ.get("REVO_PROFILE_RANGE") == "1"
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        if mark:
            torch.cuda.profiler.start()
        # With `depth` frames in flight the other lanes run on the context's
        # own streams: the end event is recorded once every frame has been
        # polled (complete), so the span covers all of them.
        start.record(stream)
        lat, launches = run_pipelined(R, ctx, dev_req, args.steps, depth)
        end.record(stream)
        torch.cuda.synchronize()
        if mark:
            torch.cuda.profiler.stop()
        barrier()
    dev_s = start.elapsed_time(end) / 1e3
    dev_s_max = max_over_ranks(dev_s)
    value = whole_job_rate(args.steps, dev_s_max, world)
    clocks = clk.summary()

    # End to end: host (pinned) buffers, copies inside the timed region, host clock.
    run_pipelined(R, ctx, host_req, 2 * depth, depth)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    run_pipelined(R, ctx, host_req, args.steps, depth)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # Dominant kernel, timed alone on the same stream with CUDA events: the
    # tcgen05 flash attention of one encoder block at N = 3600 tokens.
    fl = flops_per_model(3, H, W)
    N, D = fl["N"], 768
    roof = None
    if precision != R.FP32:
        qkv = (torch.randn((N, 3 * D), device="cuda") * 1.0).to(torch.bfloat16)
        out = torch.empty((N, D), dtype=torch.bfloat16, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(3):
                R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record(stream)
            for _ in range(reps):
                R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream)
            e1.record(stream)
            e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(3):
                R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream, split_tail=True)
            e2.record(stream)
            for _ in range(reps):
                R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream, split_tail=True)
            e3.record(stream)
        torch.cuda.synchronize()
        per_launch = e0.elapsed_time(e1) / 1e3 / reps
        split_us = e2.elapsed_time(e3) * 1e3 / reps
        pk = peaks()
        peak = pk.get("bf16_tflops")
        achieved = fl["attn_enc_per_block"] / per_launch / 1e12
        roof = {"kernel": "attn_tc_kernel (tcgen05 flash attention, N=3600, 12 heads x 64)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None, "traffic": ATTN_DRAM_BYTES_PER_LAUNCH,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone)" if peak else None,
                "flops_per_launch": fl["attn_enc_per_block"], "us_per_launch": per_launch * 1e6,
                "note": "the form the step runs (RGB and depth in flight together: no tail split); alone, with "
                        "the last wave's key ranges split over idle SMs (REVO_ATTN_SPLIT_TAIL)",
                "alone_split_tail": {"us_per_launch": split_us,
                                     "achieved": fl["attn_enc_per_block"] / (split_us * 1e-6) / 1e12,
                                     "frac": (fl["attn_enc_per_block"] / (split_us * 1e-6) / 1e12 / peak)
                                     if peak else None}}
        assert R.take_device_error() == 0

    elementwise = elementwise_roofline(R, torch, stream) if rank == 0 else None

    # Quality of the timed configuration against the FP64 oracle (RGB plane of the
    # 20 %-loss stream) + the CPU baseline from the same oracle run.
    quality, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        secs, o_vals, pl = oracle_rgb_sample()
        cpu = cpu_baseline(secs)
        # stream 2 carries the 20 %-loss frame the oracle recovered (same seed)
        err = dev_bufs[2]["rv"].cpu().numpy().astype(np.float64) - o_vals
        mse = float(np.mean(err * err))
        quality = {"rgb_psnr_db_vs_fp64": 10 * np.log10(1.0 / mse) if mse > 0 else float("inf"),
                   "rgb_max_abs_err": float(np.abs(err).max()), "gate_db": 45.0}

    # The other precisions on the same four streams and the same device buffers
    # (each in a context of its own), device-timed, with the same quality check:
    # the FP32 batch-1 path is the one the reduced-precision paths must beat.
    compare = {}
    if world == 1 and not args.no_compare:
        for name in sorted(PRECISIONS):
            if name == args.precision:
                continue
            c2 = R.Context(R.config(**VITB, precision=PRECISIONS[name](R), device=local, max_height=H, max_width=W,
                                    max_streams=8, max_batch=1, lanes=depth, use_graphs=0 if args.no_graphs else 1,
                                    autotune=1),
                           w_rgb, w_dep, stream=stream)
            for sid, (rgb, dep) in enumerate(reqs):
                for j in range(rgb.refs.shape[0]):
                    fr = torch.from_numpy(rgb.refs[j]).cuda()
                    fd = torch.from_numpy(dep.refs[j].view(np.int16)).cuda()
                    keep += [fr, fd]
                    c2.poll(c2.submit(R.request(sid, int(rgb.ref_index[j]), R.RGB | R.DEPTH | R.CLEAN,
                                                on_device=True, rgb=(fr, H, W), depth=(fd, H, W))))
            n2 = 6 if name == "fp32" else 40
            run_pipelined(R, c2, dev_req, 4, depth)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_pipelined(R, c2, dev_req, n2, depth)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            entry = {"frames_per_s": n2 / sec, "ms_per_step": sec * 1e3 / n2, "steps": n2, "batch": 1,
                     "in_flight": depth}
            c2.poll(c2.submit(dev_req[2]))
            if quality is not None:
                err = dev_bufs[2]["rv"].cpu().numpy().astype(np.float64) - o_vals
                mse = float(np.mean(err * err))
                entry["rgb_psnr_db_vs_fp64"] = 10 * np.log10(1.0 / mse) if mse > 0 else float("inf")
                entry["rgb_max_abs_err"] = float(np.abs(err).max())
            compare[name] = entry
            c2.close()
        if "fp32" in compare:
            compare["speedup_vs_fp32_batch1"] = value / compare["fp32"]["frames_per_s"]

    if rank == 0:
        lat_s = sorted(lat)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[args.precision],
            "data": "synthetic (seeded RGB-D frames, Gilbert-Elliott slice loss, random-init ViT-B weights)",
            "config": {**workload_config(world, fl["N"]),
                       "in_flight": depth, "lanes": depth,
                       "launch": "kernels" if args.no_graphs else "CUDA graph replay per request-size pattern, "
                                 "autotuned GEMM tile widths",
                       "l2": "working set > L2: bf16 weights of both models (0.37 GB) stream every step"},
            "latency_ms": {"p50": float(np.percentile(lat_s, 50)), "p99": float(np.percentile(lat_s, 99)),
                           "budget": FRAME_BUDGET_MS},
            "flops_per_step": flops_per_model(3, H, W)["total"] + flops_per_model(1, H, W)["total"],
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "cpu_baseline": cpu, "quality": quality, "precisions": compare, "elementwise": elementwise,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------ mixed sizes / serving --

# The 16-participant resolution mix: 6 x 320x240, 6 x 640x480, 4 x (1280x720
# RGB + 640x576 depth), interleaved so the first n streams keep the proportions.
MIX16 = ["320x240", "640x480", "1280x720+640x576", "320x240", "640x480", "1280x720+640x576", "320x240",
         "640x480", "1280x720+640x576", "320x240", "640x480", "1280x720+640x576", "320x240", "640x480",
         "320x240", "640x480"]


def request_flops(workload: str) -> float:
    import synth
    wl = synth.WORKLOADS[workload]
    (hr, wr), (hd, wd) = wl["rgb"], wl["depth"]
    return flops_per_model(3, hr, wr)["total"] + flops_per_model(1, hd, wd)["total"]


class StreamIO:
    """One conference stream's buffers: k clean references pushed once, then a
    few corrupted frames (seeded, same size) to recover in turn."""

    def __init__(self, R, torch, ctx, sid, workload, seed, loss_rate, frames, on_device, p_gb=None, k=5):
        import synth
        self.R, self.sid, self.workload = R, sid, workload
        self.reqs, self.keep, self.planes = [], [], []
        self.on_device = on_device
        for f in range(frames):
            kw = dict(loss_rate=loss_rate) if loss_rate is not None else {}
            rgb, dep = synth.make_request(seed + 7919 * f, workload, index=100 + f, k=k, **kw)
            self.planes.append((rgb, dep))
        rgb0, dep0 = self.planes[0]
        self.shape = ((rgb0.height, rgb0.width), (dep0.height, dep0.width))
        self.push_refs(ctx, rgb0, dep0)
        self.cleans = []
        for rgb, dep in self.planes:
            self.reqs.append(self._request(torch, rgb, dep))
            self.cleans.append(self._clean(torch, rgb, dep))

    def _buf(self, torch, a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.cuda() if self.on_device else t.pin_memory()

    def push_refs(self, ctx, rgb, dep):
        R = self.R
        import torch
        for j in range(rgb.refs.shape[0]):
            fr = torch.from_numpy(rgb.refs[j]).cuda()
            fd = torch.from_numpy(dep.refs[j].view(np.int16)).cuda()
            self.keep += [fr, fd]
            ctx.poll(ctx.submit(R.request(self.sid, int(rgb.ref_index[j]), R.RGB | R.DEPTH | R.CLEAN, on_device=True,
                                          rgb=(fr, rgb.height, rgb.width), depth=(fd, dep.height, dep.width))))

    def _request(self, torch, rgb, dep):
        R = self.R
        (hr, wr), (hd, wd) = self.shape
        b = dict(ri=self._buf(torch, rgb.decoded), di=self._buf(torch, dep.decoded.view(np.int16)),
                 rm=self._buf(torch, rgb.mask.view(np.int32)), dm=self._buf(torch, dep.mask.view(np.int32)),
                 ro=self._buf(torch, np.zeros((hr, wr, 3), np.uint8)),
                 do=self._buf(torch, np.zeros((hd, wd), np.int16)))
        self.keep.append(b)
        return R.request(self.sid, rgb.index, R.RGB | R.DEPTH, on_device=self.on_device, rgb=(b["ri"], hr, wr),
                         rgb_mask=b["rm"], depth=(b["di"], hd, wd), depth_mask=b["dm"], rgb_out=b["ro"],
                         depth_out=b["do"])

    def _clean(self, torch, rgb, dep):
        R = self.R
        (hr, wr), (hd, wd) = self.shape
        b = dict(ci=self._buf(torch, rgb.clean), cd=self._buf(torch, dep.clean.view(np.int16)))
        self.keep.append(b)
        return R.request(self.sid, rgb.index, R.RGB | R.DEPTH | R.CLEAN, on_device=self.on_device,
                         rgb=(b["ci"], hr, wr), depth=(b["cd"], hd, wd))

    def clean_request(self, i):
        """An intact frame of this stream (it enters the reference history)."""
        return self.cleans[i % len(self.cleans)]


def run_mixed(args) -> None:
    """The batched mixed-resolution launch: 16 participant streams (6 x 320x240,
    6 x 640x480, 4 x 1280x720 RGB + 640x576 depth), independent Gilbert-Elliott
    loss per stream, all 16 frames admitted into one batch per step (one graph
    replay per modality, autotuned GEMM tiles).  Beside it, the same 16 frames
    recovered one per launch (batch 1) in the same context."""
    import torch

    import paper_2604_27441_b300 as R
    import synth

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    precision = PRECISIONS[args.precision](R)
    cfg = R.config(**VITB, precision=precision, max_height=720, max_width=1280, max_streams=16, max_batch=16,
                   lanes=1, use_graphs=0 if args.no_graphs else 1, autotune=1)
    ctx = R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                    synth.flatten(synth.weights(synth.DEPTH, seed=1)), stream=stream)
    streams = [StreamIO(R, torch, ctx, sid, wl, 4000 + sid, None, 1, True) for sid, wl in enumerate(MIX16)]
    flops = sum(request_flops(wl) for wl in MIX16)

    def batched_step():
        ts = [ctx.submit(_with_flag(R, s.reqs[0], R.HOLD if i < len(streams) - 1 else 0))
              for i, s in enumerate(streams)]
        res = [ctx.poll(t) for t in ts]
        assert all(r.status == R.REVO_OK for r in res), R.last_error()
        return res

    def single_step():
        return [ctx.poll(ctx.submit(s.reqs[0])) for s in streams]

    out = {}
    for name, fn in (("batched", batched_step), ("batch1", single_step)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        steps = max(3, args.steps // 10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            lat, sizes, launches = [], [], 0
            for _ in range(steps):
                res = fn()
                lat += [r.latency_ms for r in res]
                sizes += [r.batch_size for r in res]
                launches += sum(r.kernel_launches for r in res) // max(1, res[0].batch_size) if name == "batched" \
                    else sum(r.kernel_launches for r in res)
            e1.record(stream)
            torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out[name] = {"frames_per_s": len(streams) * steps / sec, "ms_per_step": sec * 1e3 / steps,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_batch": float(np.mean(sizes)), "gpu_launches": launches, "steps": steps,
                     "effective_tflops": flops * steps / sec / 1e12, "clocks": clk.summary()}
    pk = peaks()
    st = ctx.stats()
    ctx.close()
    line = {"metric": METRIC, "value": out["batched"]["frames_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": out["batched"]["steps"], "warmup": args.warmup, "ms_per_step": out["batched"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAMES[args.precision], "data": "synthetic",
            "config": {"workload": "mixed16: 6 x 320x240 + 6 x 640x480 + 4 x (1280x720 RGB + 640x576 depth), "
                                   "one batch of 16 per step", "flops_per_step": flops,
                       "launch": "kernels" if args.no_graphs else "CUDA graph replay, autotuned GEMM tiles"},
            "batched": out["batched"], "batch1": out["batch1"],
            "speedup_vs_batch1": out["batched"]["frames_per_s"] / out["batch1"]["frames_per_s"],
            "tensor_frac_of_measured_sustained": (out["batched"]["effective_tflops"] /
                                                  pk["bf16_tflops_sustained"]) if pk.get("bf16_tflops_sustained")
            else None,
            "context": st}
    print(json.dumps(line), flush=True)


def _with_flag(R, req, extra):
    c = R.Request()
    R.C.memmove(R.C.byref(c), R.C.byref(req), R.C.sizeof(R.Request))
    c.flags |= extra
    return c


def arrival_schedule(n_streams: int, seconds: float, rng, fps: float = 30.0) -> list:
    """(arrival ms, stream, frame number) sorted by time: each stream sends a
    frame every 1000/fps ms from a uniform phase, each frame shifted by
    clip(Poisson(5) - 5, -5, 5) ms."""
    period = 1000.0 / fps
    phase = rng.uniform(0, period, n_streams)
    total = seconds * 1000.0
    events = []
    for sid in range(n_streams):
        n = 0
        while True:
            t = phase[sid] + n * period + float(np.clip(rng.poisson(5) - 5, -5, 5))
            if t > total:
                break
            events.append((t, sid, n))
            n += 1
    events.sort()
    return events


def run_serving(args) -> None:
    """Serving loop: `--streams` conference streams of the mixed resolutions,
    each sending 30 frames/s (uniform phase, per-frame jitter
    clip(Poisson(5) - 5, -5, 5) ms), Gilbert-Elliott slice loss at a per-stream
    rate drawn from 10-30 %, every 30th frame intact (REVO_CLEAN, it refreshes
    the stream's references).  Frames are submitted from pinned host memory as
    they arrive and polled without blocking; latency = submit -> completion seen
    by poll.  The first `--serve-warmup` seconds are not counted."""
    import torch

    import paper_2604_27441_b300 as R

    import synth
    torch.cuda.set_device(0)
    rng = np.random.default_rng(5000 + args.streams)
    precision = PRECISIONS[args.precision](R)
    cfg = R.config(**VITB, precision=precision, max_height=720, max_width=1280, max_streams=args.streams,
                   max_batch=args.max_batch, lanes=args.lanes, use_graphs=0 if args.no_graphs else 1, autotune=1,
                   hbm_budget_bytes=40 << 30)
    ctx = R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                    synth.flatten(synth.weights(synth.DEPTH, seed=1)))
    wls = [MIX16[i % len(MIX16)] for i in range(args.streams)]
    rates = rng.uniform(0.10, 0.30, args.streams)
    streams = [StreamIO(R, torch, ctx, sid, wl, 6000 + sid, float(rates[sid]), 3, False)
               for sid, wl in enumerate(wls)]
    events = arrival_schedule(args.streams, args.seconds, rng)
    outstanding = {}  # ticket -> (sid, arrival ms, flops)
    lat, done_frames, late, eagain, clean = [], 0, 0, 0, 0
    flops_done = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    def now_ms():
        return (time.perf_counter() - t0) * 1e3

    def drain(block_until=None):
        nonlocal done_frames, late, flops_done
        while True:
            for t in list(outstanding):
                r = ctx.poll(t, 0)
                if r is None:
                    continue
                sid, t_arr, fl = outstanding.pop(t)
                if r.status != R.REVO_OK:
                    raise RuntimeError(f"serving request failed: {R.STATUS_NAMES.get(r.status)} {R.last_error()}")
                if t_arr >= args.serve_warmup * 1e3:
                    lat.append(r.latency_ms)
                    done_frames += 1
                    flops_done += fl
                    late += r.latency_ms > FRAME_BUDGET_MS
            if block_until is None or now_ms() >= block_until:
                return
            time.sleep(0.0002)

    with ClockSampler(0) as clk:
        for t_arr, sid, n in events:
            drain(block_until=t_arr)
            s = streams[sid]
            if n % 30 == 29:
                c = s.clean_request(n)
                c.frame_index = 100 + n
                ctx.submit(c)
                clean += 1
                continue
            req = s.reqs[n % len(s.reqs)]
            req.frame_index = 100 + n
            try:
                tk = ctx.submit(req)
            except R.RevoError as e:
                if e.status == R.REVO_EAGAIN:
                    eagain += 1
                    continue
                raise
            outstanding[tk] = (sid, t_arr, request_flops(s.workload))
        while outstanding:
            drain(block_until=now_ms() + 1.0)
        wall = now_ms() - args.serve_warmup * 1e3
    st = ctx.stats()
    ctx.close()
    lat_s = sorted(lat)
    offered = sum(1 for t, _, n in events if t >= args.serve_warmup * 1e3 and n % 30 != 29)
    line = {"metric": METRIC, "value": done_frames / (wall / 1e3), "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAMES[args.precision], "data": "synthetic",
            "config": {"workload": f"serving: {args.streams} streams at 30 fps, resolutions {sorted(set(wls))}",
                       "seconds": args.seconds, "warmup_s": args.serve_warmup, "max_batch": args.max_batch,
                       "lanes": args.lanes, "hbm_budget_gb": 40, "inputs": "pinned host buffers"},
            "latency_ms": {"p50": float(np.percentile(lat_s, 50)) if lat_s else None,
                           "p99": float(np.percentile(lat_s, 99)) if lat_s else None,
                           "max": float(lat_s[-1]) if lat_s else None, "budget": FRAME_BUDGET_MS,
                           "over_budget": late},
            "offered_frames": offered, "recovered_frames": done_frames, "rejected_eagain": eagain,
            "clean_frames": clean, "offered_tflops": sum(request_flops(wls[sid]) for t, sid, n in events
                                                         if t >= args.serve_warmup * 1e3 and n % 30 != 29)
            / (wall / 1e3) / 1e12, "achieved_tflops": flops_done / (wall / 1e3) / 1e12,
            "clocks": clk.summary(), "context": st}
    print(json.dumps(line), flush=True)


def run_kt(args) -> None:
    """Latency per 640x480 RGB-D frame against the number of clean references
    k and the tubelet length T (the paper's ablation over k and T): the same
    kernels at the token counts (k + 1) / T * 1200 each pair gives, batch 1,
    graph replay, device-timed."""
    import torch

    import paper_2604_27441_b300 as R
    import synth

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    precision = PRECISIONS[args.precision](R)
    rows = []
    for k, T in ((1, 1), (1, 2), (3, 1), (3, 2), (5, 1), (5, 2), (7, 1), (7, 2)):
        shape = dict(VITB, k=k, tubelet=T)
        cfgs = [synth.ModelConfig(channels=C, k=k, tubelet=T) for C in (3, 1)]
        ctx = R.Context(R.config(**shape, precision=precision, max_height=H, max_width=W, max_streams=2,
                                 max_batch=1, lanes=1, use_graphs=1, autotune=1),
                        synth.flatten(synth.weights(cfgs[0], seed=0)), synth.flatten(synth.weights(cfgs[1], seed=1)),
                        stream=stream)
        io = StreamIO(R, torch, ctx, 0, WORKLOAD, 7000 + 10 * k + T, 0.2, 1, True, k=k)
        req = io.reqs[0]
        for _ in range(args.warmup):
            ctx.poll(ctx.submit(req))
        torch.cuda.synchronize()
        n = max(10, args.steps // 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            r = ctx.poll(ctx.submit(req))
            assert r.status == R.REVO_OK, R.last_error()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        tokens = (k + 1) // T * (H // 16) * (W // 16)
        rows.append({"k": k, "T": T, "tokens": tokens, "ms_per_frame": ms, "frames_per_s": 1e3 / ms})
        ctx.close()
    print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
                      "dtype": DTYPE_NAMES[args.precision], "data": "synthetic",
                      "config": {"workload": f"k/T sweep, {WORKLOAD} RGB-D, batch 1"}, "rows": rows}), flush=True)


def run_profile_kernel(args) -> None:
    """Launches one kernel of the step at the bench's shape (for ncu captures):
    W warm-up + K timed launches on one stream, CUDA-event timed."""
    import torch

    import paper_2604_27441_b300 as R
    fl = flops_per_model(3, H, W)
    N, D = fl["N"], 768
    stream = torch.cuda.Stream()
    if args.profile_kernel == "attention":
        qkv = torch.randn((N, 3 * D), device="cuda").to(torch.bfloat16)
        out = torch.empty((N, D), dtype=torch.bfloat16, device="cuda")
        launch = lambda: R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream)  # noqa: E731
        flops = fl["attn_enc_per_block"]
    elif args.profile_kernel == "attention_split":
        qkv = torch.randn((N, 3 * D), device="cuda").to(torch.bfloat16)
        out = torch.empty((N, D), dtype=torch.bfloat16, device="cuda")
        launch = lambda: R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream,  # noqa: E731
                                        split_tail=True)
        flops = fl["attn_enc_per_block"]
    elif args.profile_kernel in ("assemble", "blend"):  # the HBM-bound stages at 1280x720 RGB, k = 5, T = 2
        Hh, Ww, k, T, p = 720, 1280, 5, 2, 16
        frames = [torch.randint(0, 256, (Hh, Ww, 3), dtype=torch.uint8, device="cuda") for _ in range(k + 1)]
        P = (Hh // p) * (Ww // p)
        stats = torch.zeros(2, device="cuda")
        if args.profile_kernel == "assemble":
            tokens = torch.empty(((k + 1) // T * P, T * 3 * p * p), dtype=torch.bfloat16, device="cuda")
            launch = lambda: R.op_assemble(3, k, T, p, Hh, Ww, frames[:k], frames[k], Ww * 3, stats,  # noqa: E731
                                           tokens, 1, stream=stream)
            nbytes = (k + 1) * Hh * Ww * 3 + tokens.numel() * 2
        else:
            head = torch.randn((P, 3 * p * p), device="cuda")
            mask = torch.randint(-2 ** 31, 2 ** 31 - 1, (Hh, (Ww + 31) // 32), dtype=torch.int32, device="cuda")
            out = torch.empty((Hh, Ww, 3), dtype=torch.uint8, device="cuda")
            launch = lambda: R.op_blend(3, p, Hh, Ww, head, frames[k], Ww * 3, mask, (Ww + 31) // 32,  # noqa: E731
                                        stats, out, Ww * 3, stream=stream)
            nbytes = head.numel() * 4 + 2 * Hh * Ww * 3 + mask.numel() * 4
        flops = None
    elif args.profile_kernel in ("fc1_fp8", "fc1_fp8_pair"):  # the same fc1 with E4M3 operands
        a = torch.randint(0, 120, (N, D), dtype=torch.uint8, device="cuda")
        w = torch.randint(0, 120, (4 * D, D), dtype=torch.uint8, device="cuda")
        sa = torch.full((N,), 0.01, device="cuda")
        sw = torch.full((4 * D,), 0.01, device="cuda")
        b = torch.zeros(4 * D, device="cuda")
        out = torch.empty((N, 4 * D), dtype=torch.bfloat16, device="cuda")
        tile = 256 | (R.TILE_PAIR if args.profile_kernel == "fc1_fp8_pair" else 0)
        launch = lambda: R.op_linear_fp8(2, a, sa, w, sw, b, out, N, 4 * D, D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    elif args.profile_kernel in ("fc2", "fc2_pair"):  # fc2 of an encoder block: residual f32 += [N, 3072] x [768, 3072]^T
        a = torch.randn((N, 4 * D), device="cuda").to(torch.bfloat16)
        w = (torch.randn((D, 4 * D), device="cuda") / 56).to(torch.bfloat16)
        b = torch.zeros(D, device="cuda")
        out = torch.zeros((N, D), device="cuda")
        tile = 256 | (R.TILE_PAIR if args.profile_kernel == "fc2_pair" else 0)
        launch = lambda: R.op_linear(R.BF16, 3, a, w, b, out, N, D, 4 * D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    else:  # fc1 of an encoder block: [N, 768] x [3072, 768]^T + GELU (fc1_pair: 256-row tiles on CTA pairs)
        a = torch.randn((N, D), device="cuda").to(torch.bfloat16)
        w = (torch.randn((4 * D, D), device="cuda") / 28).to(torch.bfloat16)
        b = torch.zeros(4 * D, device="cuda")
        out = torch.empty((N, 4 * D), dtype=torch.bfloat16, device="cuda")
        tile = 256 | (R.TILE_PAIR if args.profile_kernel == "fc1_pair" else 0)
        launch = lambda: R.op_linear(R.BF16, 2, a, w, b, out, N, 4 * D, D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        launch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        launch()
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / args.steps
    rate = {"tflops": flops / us / 1e6} if flops else {"gbs": nbytes / us / 1e3, "bytes": nbytes}
    print(json.dumps({"kernel": args.profile_kernel, "us_per_launch": us, **rate,
                      "device_error": R.take_device_error()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-kernel", choices=["attention", "attention_split", "fc1", "fc1_pair", "fc1_fp8", "fc1_fp8_pair",
                                                 "fc2", "fc2_pair",
                             "assemble", "blend"],
                    default=None,
                    help="only launch one kernel of the step (for profiler captures)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graphs", action="store_true", help="plain kernel launches instead of graph replay")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precisions")
    ap.add_argument("--workload", choices=["640x480", "mixed16", "serving", "kt"], default="640x480",
                    help="640x480: the headline batch-1 step; mixed16: one batch of 16 mixed-size streams; "
                         "serving: real-time arrivals from --streams streams")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--seconds", type=float, default=30.0)
    ap.add_argument("--serve-warmup", type=float, default=3.0)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--lanes", type=int, default=2)
    ap.add_argument("--in-flight", type=int, default=2,
                    help="headline: batch-1 frames in flight (one lane each); 1 = submit, wait, repeat")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_kernel:
        run_profile_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed16":
        run_mixed(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "kt":
        run_kt(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
