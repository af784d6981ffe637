#!/usr/bin/env python
"""Benchmark of the ReVo neural loss-recovery hot path on B300.

The headline step is the batched mixed-resolution tick: 16 conference
streams (6 x 320x240, 6 x 640x480, 4 x 1280x720 RGB + 640x576 depth), one
corrupted RGB-D frame each with independent Gilbert-Elliott slice loss, all
recovered in one batch per modality (one CUDA-graph replay each, autotuned
GEMM tiles) through the library's C ABI (revo_recover_submit with REVO_HOLD +
revo_recover_poll): tubelet assembly + normalisation, the ViT-B
encoder-decoder forward of both modality models (two CUDA streams), the pixel
head and the masked blend.  `value` = recovered frames/s of that tick (BF16),
inputs resident on the device.  Beside it, in the same JSON line:

  latency_ms   p50/p99 of the real-time serving loop (8 streams x 30 frames/s
               of the same resolution mix, 20 s, pinned host inputs), BF16;
               `serving` has BF16 and FP8
  e2e          the tick with pinned host buffers (every tick's copies inside
               the timing; two ticks in flight on two lanes)
  batch1_640x480  one 640x480 RGB-D frame per launch (two in flight) at BF16,
               FP8 and FP32 -- the FP32 batch-1 path is the one to beat --
               with RGB and depth error against the FP64 oracle
  roofline     the dominant kernel (the tick's batched encoder attention)
  cpu_baseline the FP64 oracle on 320x240 RGB-D frames, scaled to the tick

  python bench.py [--gpus N] [--steps K] [--warmup W]
  python bench.py --impl reference ...   # the FP64 CPU oracle, same metric and workload
  python bench.py --workload 640x480 | serving | kt   # single measurements

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import contextlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "recovered RGB-D frames/s + p99 latency, BF16/FP8 vs FP32, at ≥45 dB vs FP64 oracle"
UNIT = "frames/s"
H, W = 480, 640  # the batch-1 comparison frame
LOSS_RATES = (0.05, 0.10, 0.20, 0.40)
VITB = dict(k=5, tubelet=2, patch=16, enc_dim=768, enc_depth=12, enc_heads=12, dec_dim=384, dec_depth=4,
            dec_heads=6, mlp_ratio=4)
FRAME_BUDGET_MS = 33.0
PRECISIONS = {"bf16": lambda R: R.BF16, "fp32": lambda R: R.FP32, "fp8": lambda R: R.FP8}
DTYPE_NAMES = {"bf16": "bf16", "fp32": "f32",
               "fp8": "e4m3 (RGB model: encoder and decoder qkv + fc1; per-token x per-channel scales) + bf16"}
# The 16-participant resolution mix: 6 x 320x240, 6 x 640x480, 4 x (1280x720
# RGB + 640x576 depth), interleaved so the first n streams keep the proportions.
MIX16 = ["320x240", "640x480", "1280x720+640x576", "320x240", "640x480", "1280x720+640x576", "320x240",
         "640x480", "1280x720+640x576", "320x240", "640x480", "1280x720+640x576", "320x240", "640x480",
         "320x240", "640x480"]
TICK_WORKLOAD = ("mixed16: 16 participant streams (6 x 320x240, 6 x 640x480, 4 x 1280x720 RGB + 640x576 depth), "
                 "independent Gilbert-Elliott slice loss, one batch per modality per step")
# Tile choices are shared by the benchmark's contexts through one cache file
# (each context times only the GEMM shapes the file lacks).
TILE_CACHE = os.path.join(tempfile.gettempdir(), f"revo_tiles_{os.getpid()}.txt")
# DRAM bytes (read + write) of one attn_tc_kernel launch of the tick's batched
# RGB encoder attention, from an ncu capture of the current kernel version
# (None once the kernel changes).
ATTN_DRAM_BYTES_PER_LAUNCH = 330185984 + 89459200


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


def tick_config(world: int) -> dict:
    """The headline workload, as both arms name it in `config`."""
    return {"workload": TICK_WORKLOAD, "model": "ViT-B enc-dec (768x12 / 384x4), k=5, T=2, p=16",
            "global_batch": 16 * world, "seq_len": 10800, "parallelism": f"replicas x{world}"}


def flops_per_model(C: int, h: int, w: int) -> dict:
    """Algorithmic FLOPs of one forward (2 per multiply-add), exact savings applied:
    the last decoder block's queries, proj and MLP and the pixel head run on the
    final slot's P rows only (its keys and values on all N), and the head keeps
    the target frame's outputs only."""
    k, T, p, D, L, Dd, Ld, r = 5, 2, 16, 768, 12, 384, 4, 4
    P = (h // p) * (w // p)
    N = (k + 1) // T * P
    Kt = T * C * p * p
    lin = 2 * N * Kt * D
    lin += L * 2 * N * (3 * D * D + D * D + 2 * r * D * D)
    lin += 2 * N * D * Dd
    lin += (Ld - 1) * 2 * N * (3 * Dd * Dd + Dd * Dd + 2 * r * Dd * Dd)
    lin += 2 * N * 3 * Dd * Dd + 2 * P * (Dd * Dd + 2 * r * Dd * Dd)
    lin += 2 * P * Dd * (C * p * p)
    attn_enc = 4 * N * N * D
    attn_dec = (Ld - 1) * 4 * N * N * Dd + 4 * P * N * Dd
    return dict(N=N, linear=lin, attn_enc_per_block=attn_enc, attn=L * attn_enc + attn_dec,
                total=lin + L * attn_enc + attn_dec)


def request_flops(workload: str) -> float:
    import synth
    wl = synth.WORKLOADS[workload]
    (hr, wr), (hd, wd) = wl["rgb"], wl["depth"]
    return flops_per_model(3, hr, wr)["total"] + flops_per_model(1, hd, wd)["total"]


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


def whole_job_rate(steps_per_rank: int, max_seconds: float, world: int, frames_per_step: int = 1) -> float:
    """Frames/s of the whole job: every rank's frames over the slowest rank's time."""
    return world * steps_per_rank * frames_per_step / max_seconds


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


class SmClockProbe:
    """The SM clock read through NVML (the driver's libnvidia-ml, by ctypes)
    about every millisecond while a short timed region runs (a few ms: too
    short for nvidia-smi's 200 ms samples).  Reads only; gives no samples
    where the library cannot be loaded."""

    NVML_CLOCK_SM = 1

    def __init__(self, gpu_index: int):
        self.gpu, self.samples = gpu_index, []
        self._stop, self._thread, self._lib = threading.Event(), None, None

    def __enter__(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return self
            self._lib = lib
            handle = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(handle)) != 0:
                return self
            clk = ctypes.c_uint()

            def poll():
                while not self._stop.is_set():
                    if lib.nvmlDeviceGetClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(clk)) == 0:
                        self.samples.append(clk.value)
                    time.sleep(0.001)

            self._thread = threading.Thread(target=poll, daemon=True)
            self._thread.start()
        except OSError:
            self._thread = None
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._thread is not None:
            self._thread.join(timeout=1.0)
        if self._lib is not None:
            self._lib.nvmlShutdown()

    def summary(self) -> dict:
        return {"sm_mhz_median": statistics.median(self.samples) if self.samples else None,
                "samples": len(self.samples), "source": "NVML, ~1 ms"}


# ------------------------------------------------------------ oracle arm --
# One oracle measurement serves both CPU figures (the main arm's cpu_baseline
# and the --impl reference arm): seconds per 320x240 RGB-D frame of the FP64
# oracle (both modality models), scaled to the tick by FLOP count.

ORACLE_SAMPLE = "320x240"


def oracle_sample_inputs():
    import synth
    rgb, dep = synth.make_request(1001, ORACLE_SAMPLE)
    return rgb, dep, synth.weights(synth.RGB, seed=0), synth.weights(synth.DEPTH, seed=1)


def oracle_frame_seconds(inputs) -> float:
    """One 320x240 RGB-D frame through the FP64 oracle, as it stands."""
    import synth
    from oracle import revo_oracle as O
    rgb, dep, wr, wd = inputs
    t0 = time.perf_counter()
    O.recover("rgb", wr, synth.RGB, rgb.refs, rgb.ref_index, rgb.decoded, rgb.mask, rgb.index)
    O.recover("depth", wd, synth.DEPTH, dep.refs, dep.ref_index, dep.decoded, dep.mask, dep.index)
    return time.perf_counter() - t0


def oracle_scale() -> tuple[float, float]:
    """(FLOPs of the tick, FLOPs of one oracle sample frame)."""
    return sum(request_flops(wl) for wl in MIX16), request_flops(ORACLE_SAMPLE)


def oracle_tick_rate(seconds_per_frame: float) -> float:
    tick, frame = oracle_scale()
    return len(MIX16) / (seconds_per_frame * tick / frame)


def oracle_sample_text(seconds_per_frame: float, frames: int) -> str:
    tick, frame = oracle_scale()
    return (f"FP64 oracle recovering {frames} whole {ORACLE_SAMPLE} RGB-D frame(s) (both models), "
            f"{seconds_per_frame:.2f} s per frame, scaled to the 16-frame tick by FLOPs ({tick / frame:.1f} such "
            f"frames; the oracle's softmax makes its larger frames slower per FLOP, so the scaled figure favours "
            f"the CPU)")


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inputs = oracle_sample_inputs()
    times = []
    for i in range(args.warmup + args.steps):
        dt = oracle_frame_seconds(inputs)
        if i >= args.warmup:
            times.append(dt)
    per_frame = statistics.mean(times)
    value = oracle_tick_rate(per_frame)
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_frame,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": tick_config(1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: " + oracle_sample_text(per_frame, 1)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# -------------------------------------------------------------- our arm --

def elementwise_roofline(R, torch, stream) -> dict:
    """The HBM-bound stages alone at the largest frame of the workloads (1280x720
    RGB): the fused unpack + normalise + tubelet gather (assemble) and the
    de-normalise + masked blend; the same two over the tick's 16 RGB planes in
    one launch each, and the LayerNorm over the tick's RGB rows.  L2 is flushed
    (a 256 MB write, then a read of it) before every timed launch; achieved =
    algorithmic bytes / CUDA-event time."""
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
    out = {"assemble_rgb_1280x720": mk(us_a, bytes_a), "blend_rgb_1280x720": mk(us_b, bytes_b)}
    del refs, tokens, head
    # The form the tick runs: one launch over the 16 requests' RGB planes.
    import synth
    ajobs, bjobs, keep = [], [], []
    bytes_ta = bytes_tb = 0
    for wl in MIX16:
        hh, ww = synth.WORKLOADS[wl]["rgb"]
        fr = [torch.randint(0, 256, (hh, ww, 3), dtype=torch.uint8, device="cuda") for _ in range(k + 1)]
        pp = (hh // p) * (ww // p)
        tok = torch.empty(((k + 1) // T * pp, T * 3 * p * p), dtype=torch.bfloat16, device="cuda")
        hd = torch.randn((pp, 3 * p * p), device="cuda")
        mk_ = torch.randint(-2 ** 31, 2 ** 31 - 1, (hh, (ww + 31) // 32), dtype=torch.int32, device="cuda")
        o = torch.empty((hh, ww, 3), dtype=torch.uint8, device="cuda")
        keep += [fr, tok, hd, mk_, o]
        ajobs.append(dict(height=hh, width=ww, frames=fr, pitch_bytes=ww * 3, mu_sigma=None, out=tok))
        bjobs.append(dict(height=hh, width=ww, head=hd, decoded=fr[k], pitch_bytes=ww * 3, mask=mk_,
                          mask_pitch_words=(ww + 31) // 32, mu_sigma=None, out=o, out_pitch=ww * 3))
        bytes_ta += (k + 1) * hh * ww * 3 + tok.numel() * 2
        bytes_tb += hd.numel() * 4 + 2 * hh * ww * 3 + mk_.numel() * 4
    # The argument tables are uploaded by the first call; time the second and later.
    R.op_assemble_batch(3, k, T, ajobs, 1, stream=stream)
    R.op_blend_batch(3, bjobs, stream=stream)
    out["assemble_rgb_tick_batch16"] = mk(timed(lambda: R.op_assemble_batch(3, k, T, ajobs, 1, stream=stream)),
                                          bytes_ta)
    out["blend_rgb_tick_batch16"] = mk(timed(lambda: R.op_blend_batch(3, bjobs, stream=stream)), bytes_tb)
    del keep, ajobs, bjobs
    # The LayerNorm over the tick's RGB rows (x float32 in, h bf16 out), the
    # standalone launch the forward runs before qkv and fc1.
    ln, _, bytes_ln = profile_launch(R, torch, "layernorm_tick", stream)
    out["layernorm_rgb_tick_70200x768"] = mk(timed(ln), bytes_ln)
    del ln
    out["peak_source"] = "MEASURED_PEAKS.json hbm_gbs" if hbm else None
    out["note"] = ("single frame: one launch for one 1280x720 plane (launch ramp dominates 16.7 MB); "
                   "tick_batch16: one launch over the 16 requests' RGB planes, as the forward runs them; "
                   "layernorm: one launch over the tick's 70200 RGB rows at D = 768")
    return out


def tick_segments(wl_rgb: bool = True) -> list:
    """Token counts of the tick's RGB (or depth) requests, in MIX16 order."""
    import synth
    out = []
    for wl in MIX16:
        h, w = synth.WORKLOADS[wl]["rgb" if wl_rgb else "depth"]
        out.append(3 * (h // 16) * (w // 16))
    return out


def attention_roofline(R, torch, stream) -> dict:
    """The dominant kernel of the tick, timed alone on the same stream with CUDA
    events: the batched tcgen05 attention of one RGB encoder block over the 16
    requests' token segments (N = 900 x 6, 3600 x 6, 10800 x 4; 12 heads x 64),
    in the form the forward runs (one CTA per unit).  Achieved = 4 N^2 D summed
    over the segments / launch time.  Beside it the same kernel on one 640x480
    request (N = 3600) and its tail-cut form (REVO_ATTN_SPLIT_TAIL).  `clock`:
    the SM clock during the timed launches (NVML), so that runs on different
    boxes can be compared."""
    D, heads = 768, 12
    lens = tick_segments(True)
    seg = np.concatenate([[0], np.cumsum(lens)]).astype(int).tolist()
    M = seg[-1]
    qkv = torch.randn((M, 3 * D), device="cuda").to(torch.bfloat16)
    out = torch.empty((M, D), dtype=torch.bfloat16, device="cuda")

    def timed(fn, reps, probe=None):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with probe if probe is not None else contextlib.nullcontext():
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    flops = sum(4 * n * n * D for n in lens)
    probe = SmClockProbe(torch.cuda.current_device())
    sec = timed(lambda: R.op_attention(R.BF16, qkv, out, M, D, heads, seg, stream=stream), 10, probe)
    N1 = 3600
    f1 = 4 * N1 * N1 * D
    q1, o1 = qkv[:N1].contiguous(), out[:N1]
    sec1 = timed(lambda: R.op_attention(R.BF16, q1, o1, N1, D, heads, [0, N1], stream=stream), 50)
    sec1s = timed(lambda: R.op_attention(R.BF16, q1, o1, N1, D, heads, [0, N1], stream=stream, split_tail=True), 50)
    assert R.take_device_error() == 0
    peak = peaks().get("bf16_tflops")
    tf = lambda f, s: f / s / 1e12  # noqa: E731
    return {"kernel": "attn_tc_kernel + attn_combine_kernel (tcgen05 flash attention; the tick's RGB encoder "
                      "attention: 16 segments, N = 900 x 6 + 3600 x 6 + 10800 x 4, 12 heads x 64)",
            "bound": "tensor", "achieved": tf(flops, sec), "peak": peak, "unit": "TFLOP/s",
            "frac": tf(flops, sec) / peak if peak else None, "traffic": ATTN_DRAM_BYTES_PER_LAUNCH,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone)" if peak else None,
            "flops_per_launch": flops, "us_per_launch": sec * 1e6, "clock": probe.summary(),
            "n3600_alone": {"us_per_launch": sec1 * 1e6, "achieved": tf(f1, sec1),
                            "frac": tf(f1, sec1) / peak if peak else None},
            "n3600_split_tail": {"us_per_launch": sec1s * 1e6, "achieved": tf(f1, sec1s),
                                 "frac": tf(f1, sec1s) / peak if peak else None}}


def tensor_roofline(R, torch, stream) -> dict:
    """The contractions besides attention at the 16-stream tick's sizes, each
    timed alone on the stream with CUDA events (3 warm-up + 10 launches):
    fc1 (GELU), fc2 and proj (residual) over the 70200 RGB rows on CTA pairs,
    fc1 with E4M3 operands, and the tubelet embedding (the Conv3d as an
    implicit GEMM) over the tick's RGB and depth frames.  Achieved = 2 M N K /
    launch time; peak = the measured bf16 burst (E4M3: twice it, the nominal
    ratio).  For fc1, fc2 and proj also the HBM rate of their algorithmic bytes
    (operands read once, the output written once; the residual's float32 x
    read and written) against the measured copy rate: proj (K = 768 into a
    float32 residual) has more bytes per FLOP than the tensor/HBM balance."""
    peak = peaks().get("bf16_tflops")
    hbm = peaks().get("hbm_gbs")
    out = {}
    for name, fp8 in (("fc1_tick", False), ("fc2_tick", False), ("proj_tick", False), ("fc1_fp8_tick", True),
                      ("embed_tick", False), ("embed_tick_depth", False)):
        launch, flops, nbytes = profile_launch(R, torch, name, stream)
        with torch.cuda.stream(stream):
            for _ in range(3):
                launch()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                launch()
            e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / 10
        pk = (2 * peak if fp8 else peak) if peak else None
        out[name] = {"us_per_launch": sec * 1e6, "flops_per_launch": flops, "achieved_tflops": flops / sec / 1e12,
                     "peak_tflops": pk, "frac": flops / sec / 1e12 / pk if pk else None}
        if nbytes:
            out[name].update(bytes_per_launch=nbytes, achieved_gbs=nbytes / sec / 1e9,
                             frac_of_measured_hbm=nbytes / sec / 1e9 / hbm if hbm else None)
        del launch
        torch.cuda.empty_cache()
    assert R.take_device_error() == 0
    out["peak_source"] = ("MEASURED_PEAKS.json bf16_tflops (burst; kernels timed alone); E4M3: 2x; "
                          "hbm_gbs for the byte rates" if peak else None)
    return out


class StreamIO:
    """One conference stream's buffers: k clean references pushed once, then a
    few corrupted frames (seeded, same size) to recover in turn."""

    def __init__(self, R, torch, ctx, sid, workload, seed, loss_rate, frames, on_device, k=5, values=False):
        import synth
        self.R, self.sid, self.workload = R, sid, workload
        self.reqs, self.keep, self.planes, self.bufs = [], [], [], []
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
            self.reqs.append(self._request(torch, rgb, dep, values))
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

    def _request(self, torch, rgb, dep, values):
        R = self.R
        (hr, wr), (hd, wd) = self.shape
        b = dict(ri=self._buf(torch, rgb.decoded), di=self._buf(torch, dep.decoded.view(np.int16)),
                 rm=self._buf(torch, rgb.mask.view(np.int32)), dm=self._buf(torch, dep.mask.view(np.int32)),
                 ro=self._buf(torch, np.zeros((hr, wr, 3), np.uint8)),
                 do=self._buf(torch, np.zeros((hd, wd), np.int16)))
        if values:
            b["rv"] = self._buf(torch, np.zeros((hr, wr, 3), np.float32))
            b["dv"] = self._buf(torch, np.zeros((hd, wd), np.float32))
        self.keep.append(b)
        self.bufs.append(b)
        return R.request(self.sid, rgb.index, R.RGB | R.DEPTH, on_device=self.on_device, rgb=(b["ri"], hr, wr),
                         rgb_mask=b["rm"], depth=(b["di"], hd, wd), depth_mask=b["dm"], rgb_out=b["ro"],
                         depth_out=b["do"], rgb_values=b.get("rv"), depth_values=b.get("dv"))

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

    def io_bytes(self):
        """(host->device, device->host) bytes of one recovery request."""
        (hr, wr), (hd, wd) = self.shape
        h2d = hr * wr * 3 + hd * wd * 2 + 4 * (hr * ((wr + 31) // 32) + hd * ((wd + 31) // 32))
        return h2d, hr * wr * 3 + hd * wd * 2


def _with_flag(R, req, extra):
    c = R.Request()
    R.C.memmove(R.C.byref(c), R.C.byref(req), R.C.sizeof(R.Request))
    c.flags |= extra
    return c


def tick_context(R, precision, stream, graphs=True, lanes=1, serial=0):
    import synth
    cfg = R.config(**VITB, precision=precision, max_height=720, max_width=1280, max_streams=16, max_batch=16,
                   lanes=lanes, use_graphs=1 if graphs else 0, autotune=1, autotune_cache=TILE_CACHE,
                   serial_models=serial)
    return R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                     synth.flatten(synth.weights(synth.DEPTH, seed=1)), stream=stream)


def tick_streams(R, torch, ctx, on_device, base_seed=4000):
    """The 16 streams, each with two request buffers (two ticks in flight)."""
    return [StreamIO(R, torch, ctx, sid, wl, base_seed + sid, None, 2, on_device) for sid, wl in enumerate(MIX16)]


def tick_submit(R, ctx, streams, which=0):
    """Submits the 16 frames (all but the last with REVO_HOLD, so they form one
    batch), from each stream's request buffers `which` (ticks in flight
    together use different ones); returns the tickets."""
    return [ctx.submit(_with_flag(R, s.reqs[which % len(s.reqs)], R.HOLD if i < len(streams) - 1 else 0))
            for i, s in enumerate(streams)]


def tick_poll(R, ctx, tickets):
    res = [ctx.poll(t) for t in tickets]
    if not all(r.status == R.REVO_OK for r in res):
        raise RuntimeError(f"tick failed: {R.last_error()}")
    return res


def tick_once(R, ctx, streams):
    """Submits the 16 frames (all but the last with REVO_HOLD, so they form one
    batch), polls them all."""
    ts = [ctx.submit(_with_flag(R, s.reqs[0], R.HOLD if i < len(streams) - 1 else 0))
          for i, s in enumerate(streams)]
    res = [ctx.poll(t) for t in ts]
    if not all(r.status == R.REVO_OK for r in res):
        raise RuntimeError(f"tick failed: {R.last_error()}")
    return res


def measure_tick(R, torch, ctx, streams, stream, steps, warmup, clock_gpu=None):
    """Device-timed ticks (CUDA events on the context's stream)."""
    for _ in range(warmup):
        tick_once(R, ctx, streams)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, launches = [], 0
    clk = ClockSampler(clock_gpu) if clock_gpu is not None else None
    # REVO_PROFILE_RANGE=1 marks the timed ticks for a profiler started with
    # --profile-from-start off (it changes nothing else).
    mark = os.environ.get("REVO_PROFILE_RANGE") == "1"
    if clk:
        clk.__enter__()
    try:
        torch.cuda.synchronize()
        if mark:
            torch.cuda.profiler.start()
        e0.record(stream)
        # Two ticks in flight: tick i + 1 is submitted before tick i is polled
        # (one lane: its batch queues behind tick i on the same streams), so
        # the device does not wait for the host between ticks.
        inflight = []
        for i in range(steps + 1):
            if i < steps:
                inflight.append(tick_submit(R, ctx, streams, i))
            if len(inflight) == 2 or (i == steps and inflight):
                res = tick_poll(R, ctx, inflight.pop(0))
                lat += [r.latency_ms for r in res]
                launches += res[0].kernel_launches  # every request of the batch reports the batch's launches
        e1.record(stream)
        torch.cuda.synchronize()
        if mark:
            torch.cuda.profiler.stop()
    finally:
        if clk:
            clk.__exit__()
    sec = e0.elapsed_time(e1) / 1e3
    flops = sum(request_flops(wl) for wl in MIX16)
    return {"seconds": sec, "frames_per_s": len(streams) * steps / sec, "ms_per_step": sec * 1e3 / steps,
            "steps": steps, "launches": launches, "tick_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                                       "p99": float(np.percentile(lat, 99))},
            "effective_tflops": flops * steps / sec / 1e12, "clocks": clk.summary() if clk else None}


def measure_tick_e2e(R, torch, precision, graphs, steps, base_seed, serial=0, lanes=1, depth=2):
    """The tick end to end through pinned host buffers, host clock: every
    tick's frame and mask copies in (at submit) and its blended frames out
    (before poll returns) are inside the timed region.  `depth` ticks are in
    flight, as a serving loop runs them: tick i + 1 is submitted before tick
    i is polled, so its input copies overlap tick i's kernels (one lane: two
    lanes measured 295.5 against 301.7 frames/s, two ticks' kernels side by
    side compete for the SMs).  Each stream has two request buffers (ticks
    use them in turn), so no output buffer is borrowed twice."""
    ctx = tick_context(R, precision, None, graphs=graphs, lanes=lanes, serial=serial)
    try:
        streams = tick_streams(R, torch, ctx, False, base_seed)

        def run(n):
            inflight = []
            for i in range(n):
                inflight.append(tick_submit(R, ctx, streams, i))
                if len(inflight) == depth:
                    tick_poll(R, ctx, inflight.pop(0))
            for ts in inflight:
                tick_poll(R, ctx, ts)

        run(4)  # both lanes' graphs captured, tiles from the cache
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(steps)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        h2d = sum(s.io_bytes()[0] for s in streams)
        d2h = sum(s.io_bytes()[1] for s in streams)
    finally:
        ctx.close()
    return sec, h2d, d2h


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


def measure_serving(R, torch, precision, n_streams, seconds, serve_warmup, max_batch=8, lanes=2, graphs=True):
    """Serving loop: n_streams conference streams of the mixed resolutions,
    each sending 30 frames/s (uniform phase, per-frame jitter
    clip(Poisson(5) - 5, -5, 5) ms), Gilbert-Elliott slice loss at a per-stream
    rate drawn from 10-30 %, every 30th frame intact (REVO_CLEAN, it refreshes
    the stream's references).  Frames are submitted from pinned host memory as
    they arrive and polled without blocking; latency = submit -> completion seen
    by poll (and, beside it, from the frame's scheduled arrival: under overload
    submit blocks until a staging slot frees, and that wait counts there).
    Frames arriving in the first serve_warmup seconds are not counted."""
    import synth
    rng = np.random.default_rng(5000 + n_streams)
    cfg = R.config(**VITB, precision=precision, max_height=720, max_width=1280, max_streams=n_streams,
                   max_batch=max_batch, lanes=lanes, use_graphs=1 if graphs else 0, autotune=1,
                   autotune_cache=TILE_CACHE,
                   hbm_budget_bytes=40 << 30)
    ctx = R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                    synth.flatten(synth.weights(synth.DEPTH, seed=1)))
    wls = [MIX16[i % len(MIX16)] for i in range(n_streams)]
    rates = rng.uniform(0.10, 0.30, n_streams)
    streams = [StreamIO(R, torch, ctx, sid, wl, 6000 + sid, float(rates[sid]), 3, False)
               for sid, wl in enumerate(wls)]
    events = arrival_schedule(n_streams, seconds, rng)
    outstanding = {}  # ticket -> (sid, arrival ms, flops)
    lat, lat_arr, done_frames, late, eagain, clean = [], [], 0, 0, 0, 0
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
                if t_arr >= serve_warmup * 1e3:
                    lat.append(r.latency_ms)
                    lat_arr.append(now_ms() - t_arr)
                    done_frames += 1
                    flops_done += fl
                    late += r.latency_ms > FRAME_BUDGET_MS
            if block_until is None or now_ms() >= block_until:
                return
            time.sleep(0.0002)

    with ClockSampler(torch.cuda.current_device()) as clk:
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
        wall = now_ms() - serve_warmup * 1e3
    st = ctx.stats()
    ctx.close()
    lat_s = sorted(lat)
    lat_a = sorted(lat_arr)
    offered = sum(1 for t, _, n in events if t >= serve_warmup * 1e3 and n % 30 != 29)
    return {"frames_per_s": done_frames / (wall / 1e3),
            "latency_ms": {"p50": float(np.percentile(lat_s, 50)) if lat_s else None,
                           "p99": float(np.percentile(lat_s, 99)) if lat_s else None,
                           "max": float(lat_s[-1]) if lat_s else None, "budget": FRAME_BUDGET_MS,
                           "over_budget": late},
            # From the frame's scheduled arrival to its completion seen by poll: includes any
            # time the frame waited before submit (submit blocks while no staging slot is free).
            "latency_from_arrival_ms": {"p50": float(np.percentile(lat_a, 50)) if lat_a else None,
                                        "p99": float(np.percentile(lat_a, 99)) if lat_a else None,
                                        "over_budget": sum(1 for x in lat_a if x > FRAME_BUDGET_MS)},
            "streams": n_streams, "seconds": seconds, "warmup_s": serve_warmup, "max_batch": max_batch,
            "lanes": lanes, "hbm_budget_gb": 40, "inputs": "pinned host buffers",
            "offered_frames": offered, "recovered_frames": done_frames, "rejected_eagain": eagain,
            "clean_frames": clean,
            "offered_tflops": sum(request_flops(wls[sid]) for t, sid, n in events
                                  if t >= serve_warmup * 1e3 and n % 30 != 29) / (wall / 1e3) / 1e12,
            "achieved_tflops": flops_done / (wall / 1e3) / 1e12, "clocks": clk.summary(), "context": st}


def measure_batch1(R, torch, precision, stream, steps, warmup, in_flight=2, graphs=True, local=0, rank=0):
    """One 640x480 RGB-D frame per launch, `in_flight` frames in flight on as
    many lanes; four streams (5/10/20/40 % loss) in turn.  Stream 2 (20 %) also
    writes the de-normalised float outputs for the quality check."""
    import synth
    cfg = R.config(**VITB, precision=precision, device=local, max_height=H, max_width=W, max_streams=8,
                   max_batch=1, lanes=in_flight, use_graphs=1 if graphs else 0, autotune=1, autotune_cache=TILE_CACHE)
    ctx = R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                    synth.flatten(synth.weights(synth.DEPTH, seed=1)), stream=stream)
    streams = [StreamIO(R, torch, ctx, sid, "640x480", 2000 + 100 * rank + sid, r, 1, True, values=sid == 2)
               for sid, r in enumerate(LOSS_RATES)]
    reqs = [s.reqs[0] for s in streams]
    run_pipelined(R, ctx, reqs, warmup, in_flight)
    torch.cuda.synchronize()
    mark = os.environ.get("REVO_PROFILE_RANGE") == "1"  # the timed frames only, for a profiler (see measure_tick)
    if mark:
        torch.cuda.profiler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat, launches = run_pipelined(R, ctx, reqs, steps, in_flight)
    e1.record(stream)
    torch.cuda.synchronize()
    if mark:
        torch.cuda.profiler.stop()
    sec = e0.elapsed_time(e1) / 1e3
    lat_s = sorted(lat)
    out = {"frames_per_s": steps / sec, "ms_per_step": sec * 1e3 / steps, "steps": steps, "batch": 1,
           "in_flight": in_flight, "latency_ms": {"p50": float(np.percentile(lat_s, 50)),
                                                  "p99": float(np.percentile(lat_s, 99))},
           "gpu_launches_per_frame": launches / steps}
    run_pipelined(R, ctx, [reqs[2]], 1, 1)
    b = streams[2].bufs[0]
    values = (b["rv"].cpu().numpy().astype(np.float64), b["dv"].cpu().numpy().astype(np.float64))
    ctx.close()
    return out, values, streams[2].planes[0]


def oracle_640_values(plane_pair):
    """The FP64 oracle's de-normalised outputs (RGB in [0, 1] units, depth in
    mm) for the 640x480 RGB-D frame the batch-1 runs write values for."""
    import synth
    from oracle import revo_oracle as O
    rgb, dep = plane_pair
    _, vr = O.recover("rgb", synth.weights(synth.RGB, seed=0), synth.RGB, rgb.refs, rgb.ref_index, rgb.decoded,
                      rgb.mask, rgb.index)
    _, vd = O.recover("depth", synth.weights(synth.DEPTH, seed=1), synth.DEPTH, dep.refs, dep.ref_index,
                      dep.decoded, dep.mask, dep.index)
    return vr, vd


def quality(values, ref, plane_pair) -> dict:
    """Error of one precision's float outputs (the de-normalised network output
    at every pixel, before the blend) against the FP64 oracle's: PSNR of RGB in
    [0, 1] units and of depth / 65535 over the whole frame (the gate) and over
    the lost pixels alone (the ones the blend takes from the network), max
    |error| in [0, 1] units and mm."""
    er = values[0] - ref[0]
    ed = values[1] - ref[1]
    lost_rgb, lost_dep = plane_pair[0].lost, plane_pair[1].lost

    def psnr(e, peak):
        mse = float(np.mean(e * e)) if e.size else 0.0
        return 10 * np.log10(peak * peak / mse) if mse > 0 else float("inf")
    return {"rgb_psnr_db": psnr(er, 1.0), "rgb_psnr_lost_db": psnr(er[lost_rgb], 1.0),
            "rgb_max_abs_err": float(np.abs(er).max()),
            "depth_psnr_db": psnr(ed / 65535.0, 1.0), "depth_psnr_lost_db": psnr(ed[lost_dep] / 65535.0, 1.0),
            "depth_max_abs_err_mm": float(np.abs(ed).max()),
            "lost_fraction": {"rgb": float(lost_rgb.mean()), "depth": float(lost_dep.mean())},
            "gate": "PSNR >= 45 dB (RGB, depth / 65535), depth max <= 8 mm; FP32: <= 1e-4 RGB, <= 1 mm depth"}


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2604_27441_b300 as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    stream = torch.cuda.Stream()
    precision = PRECISIONS[args.precision](R)
    ctx = tick_context(R, precision, stream, graphs=not args.no_graphs, serial=int(args.serial_models))
    streams = tick_streams(R, torch, ctx, True, base_seed=4000 + 100 * rank)
    for _ in range(2):  # autotuning and graph capture of the batch's size pattern
        tick_once(R, ctx, streams)
    torch.cuda.synchronize()
    rank_barrier(world)

    # Timed region: device-resident inputs and outputs, CUDA events.
    tick = measure_tick(R, torch, ctx, streams, stream, args.steps, args.warmup, clock_gpu=local)
    rank_barrier(world)
    dev_s_max = rank_max(tick["seconds"], world)
    value = whole_job_rate(args.steps, dev_s_max, world, len(MIX16))
    ctx_stats = ctx.stats()

    ctx.close()
    del streams

    # End to end: the same tick through pinned host buffers.
    e2e_steps = max(3, args.steps // 2)
    e2e_s, h2d, d2h = measure_tick_e2e(R, torch, precision, not args.no_graphs, e2e_steps, 4000 + 100 * rank,
                                       serial=int(args.serial_models))
    e2e_s = rank_max(e2e_s, world)
    e2e = {"value": world * e2e_steps * len(MIX16) / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "in_flight": 2}

    extra = {}
    if world == 1 and not args.quick:
        roof = attention_roofline(R, torch, stream) if precision != R.FP32 else None
        # FP8 tick, same workload.
        if args.precision == "bf16":
            c8 = tick_context(R, R.FP8, stream, graphs=not args.no_graphs)
            s8 = tick_streams(R, torch, c8, True)
            for _ in range(2):
                tick_once(R, c8, s8)
            t8 = measure_tick(R, torch, c8, s8, stream, max(5, args.steps // 2), 2)
            extra["tick_fp8"] = {k: t8[k] for k in ("frames_per_s", "ms_per_step", "steps", "tick_latency_ms",
                                                     "effective_tflops")}
            c8.close()
            del s8
        # Batch-1 frames at every precision, their error against the FP64 oracle.
        b1, vals, plane_pair = {}, {}, None
        for name in ("bf16", "fp8", "fp32"):
            n = 6 if name == "fp32" else 40
            b1[name], vals[name], plane_pair = measure_batch1(R, torch, PRECISIONS[name](R), stream, n, 4,
                                                              graphs=not args.no_graphs)
        ref = oracle_640_values(plane_pair) if not args.no_cpu_baseline else None
        if ref is not None:
            for name in b1:
                b1[name]["quality_vs_fp64"] = quality(vals[name], ref, plane_pair)
        b1["speedup_bf16_vs_fp32"] = b1["bf16"]["frames_per_s"] / b1["fp32"]["frames_per_s"]
        extra["batch1_640x480"] = b1
        extra["speedup_tick_vs_fp32_batch1"] = value / b1["fp32"]["frames_per_s"]
        # Real-time serving at 8 streams (BF16 and FP8).
        serving = {}
        for name in ("bf16", "fp8"):
            serving[name] = measure_serving(R, torch, PRECISIONS[name](R), args.serve_streams, args.seconds,
                                            args.serve_warmup)
        extra["serving"] = serving
        extra["latency_ms"] = dict(serving[args.precision if args.precision in serving else "bf16"]["latency_ms"],
                                   source=f"serving loop, {args.serve_streams} streams x 30 fps of the mix, "
                                          f"{args.seconds:.0f} s, {args.precision}")
        extra["roofline"] = roof
        extra["elementwise"] = elementwise_roofline(R, torch, stream)
        if precision != R.FP32:
            extra["tensor"] = tensor_roofline(R, torch, stream)
        if not args.no_cpu_baseline:
            inputs = oracle_sample_inputs()
            secs = [oracle_frame_seconds(inputs) for _ in range(args.oracle_frames)]
            per = statistics.mean(secs)
            extra["cpu_baseline"] = {"value": oracle_tick_rate(per), "unit": UNIT, "cores": os.cpu_count(),
                                     "kind": "oracle", "sample": oracle_sample_text(per, args.oracle_frames)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tick["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[args.precision],
            "data": "synthetic (seeded RGB-D frames, Gilbert-Elliott slice loss, random-init ViT-B weights)",
            "config": {**tick_config(world),
                       "launch": "kernels" if args.no_graphs else "one CUDA graph replay per modality per tick, "
                                 "autotuned GEMM tile widths",
                       "l2": "working set > L2: bf16 weights of both models (0.37 GB) and 1.4 GB of activations "
                             "per tick"},
            "flops_per_step": sum(request_flops(wl) for wl in MIX16),
            "effective_tflops": tick["effective_tflops"], "tick_latency_ms": tick["tick_latency_ms"],
            "clocks": tick["clocks"], "e2e": e2e, "gpu_launches": tick["launches"],
            "context": ctx_stats, **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_640(args) -> None:
    """The batch-1 640x480 RGB-D step alone (one precision), two frames in flight."""
    import torch

    import paper_2604_27441_b300 as R
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    with ClockSampler(0) as clk:
        out, _, _ = measure_batch1(R, torch, PRECISIONS[args.precision](R), stream, args.steps, args.warmup,
                                   in_flight=args.in_flight, graphs=not args.no_graphs)
    print(json.dumps({"metric": METRIC, "value": out["frames_per_s"], "unit": UNIT, "n_gpus": 1,
                      "dtype": DTYPE_NAMES[args.precision], "config": {"workload": "640x480 RGB-D batch 1"},
                      **out, "clocks": clk.summary()}), flush=True)


def run_serving(args) -> None:
    import torch

    import paper_2604_27441_b300 as R
    torch.cuda.set_device(0)
    out = measure_serving(R, torch, PRECISIONS[args.precision](R), args.serve_streams, args.seconds,
                          args.serve_warmup, max_batch=args.max_batch, lanes=args.lanes, graphs=not args.no_graphs)
    print(json.dumps({"metric": METRIC, "value": out["frames_per_s"], "unit": UNIT, "n_gpus": 1,
                      "dtype": DTYPE_NAMES[args.precision], "data": "synthetic",
                      "config": {"workload": f"serving: {args.serve_streams} streams at 30 fps of the mix"},
                      **out}), flush=True)


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
                                 max_batch=1, lanes=1, use_graphs=1, autotune=1, autotune_cache=TILE_CACHE),
                        synth.flatten(synth.weights(cfgs[0], seed=0)), synth.flatten(synth.weights(cfgs[1], seed=1)),
                        stream=stream)
        io = StreamIO(R, torch, ctx, 0, "640x480", 7000 + 10 * k + T, 0.2, 1, True, k=k)
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
                      "config": {"workload": "k/T sweep, 640x480 RGB-D, batch 1"}, "rows": rows}), flush=True)


def profile_launch(R, torch, name, stream):
    """One launch of a kernel of the step at the bench's shape, by name (the
    --profile-kernel choices except "embed"): returns (launch, flops, bytes);
    flops is None for the HBM-bound stages."""
    fl = flops_per_model(3, H, W)
    N, D = fl["N"], 768
    nbytes = None
    if name in ("embed_tick", "embed_tick_separate", "embed_tick_depth",
                               "embed_tick_depth_separate"):
        # The tick's RGB (K = 1536, 70200 tokens) or depth (K = 512, 44280 tokens)
        # tubelet embedding over its 16 requests: the implicit GEMM, or the
        # assemble kernel + the GEMM over the stored tokens.
        import synth
        rgb = not name.startswith("embed_tick_depth")
        C = 3 if rgb else 1
        Kt = 2 * C * 256
        jobs, taus = [], []
        for wl in MIX16:
            h, w = synth.WORKLOADS[wl]["rgb" if rgb else "depth"]
            if rgb:
                fr = [torch.randint(0, 256, (h, w, 3), dtype=torch.uint8, device="cuda") for _ in range(6)]
                ms = None
            else:
                fr = [torch.randint(300, 5000, (h, w), dtype=torch.int16, device="cuda") for _ in range(6)]
                ms = torch.tensor([2000.0, 900.0], device="cuda")
            jobs.append(dict(height=h, width=w, frames=fr, pitch_bytes=w * (3 if rgb else 2), mu_sigma=ms))
            taus.append([5, 3, 1])
        Mt = sum(tick_segments(rgb))
        Wt = (torch.randn((D, Kt), device="cuda") / 40).to(torch.bfloat16)
        b = torch.zeros(D, device="cuda")
        out = torch.empty((Mt, D), device="cuda")
        if not name.endswith("separate"):
            launch = lambda: R.op_embed_batch(C, 5, 2, jobs, taus, Wt, b, out, D, stream=stream)  # noqa: E731
        else:
            tok = torch.empty((Mt, Kt), dtype=torch.bfloat16, device="cuda")
            row, ajobs = 0, []
            for j in jobs:
                n = 3 * (j["height"] // 16) * (j["width"] // 16)
                ajobs.append(dict(j, out=tok[row:row + n]))
                row += n

            def launch():
                R.op_assemble_batch(C, 5, 2, ajobs, 1, stream=stream)
                R.op_linear(R.BF16, 0, tok, Wt, b, out, Mt, D, Kt, 256 | R.TILE_PAIR, stream=stream)
        flops = 2 * Mt * D * Kt
    elif name in ("attention", "attention_split"):
        qkv = torch.randn((N, 3 * D), device="cuda").to(torch.bfloat16)
        out = torch.empty((N, D), dtype=torch.bfloat16, device="cuda")
        split = name == "attention_split"
        launch = lambda: R.op_attention(R.BF16, qkv, out, N, D, 12, [0, N], stream=stream,  # noqa: E731
                                        split_tail=split)
        flops = fl["attn_enc_per_block"]
    elif name == "attention_tick":  # the tick's batched RGB encoder attention
        lens = tick_segments(True)
        seg = np.concatenate([[0], np.cumsum(lens)]).astype(int).tolist()
        M = seg[-1]
        qkv = torch.randn((M, 3 * D), device="cuda").to(torch.bfloat16)
        out = torch.empty((M, D), dtype=torch.bfloat16, device="cuda")
        launch = lambda: R.op_attention(R.BF16, qkv, out, M, D, 12, seg, stream=stream)  # noqa: E731
        flops = sum(4 * n * n * D for n in lens)
    elif name == "pe":  # the position embedding of one 1280x720 request at the encoder width
        S, hp, wp = 3, 45, 80
        x = torch.zeros((S * hp * wp, D), device="cuda")
        launch = lambda: R.op_add_position(x, S, hp, wp, D, [5, 3, 1], stream=stream)  # noqa: E731
        flops, nbytes = None, 2 * x.numel() * 4
    elif name in ("assemble", "blend"):  # the HBM-bound stages at 1280x720 RGB, k = 5, T = 2
        Hh, Ww, k, T, p = 720, 1280, 5, 2, 16
        frames = [torch.randint(0, 256, (Hh, Ww, 3), dtype=torch.uint8, device="cuda") for _ in range(k + 1)]
        P = (Hh // p) * (Ww // p)
        stats = torch.zeros(2, device="cuda")
        if name == "assemble":
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
    elif name in ("fc1_fp8", "fc1_fp8_pair", "fc1_fp8_tick"):  # the same fc1 with E4M3 operands
        if name == "fc1_fp8_tick":
            N = sum(tick_segments(True))
        a = torch.randint(0, 120, (N, D), dtype=torch.uint8, device="cuda")
        w = torch.randint(0, 120, (4 * D, D), dtype=torch.uint8, device="cuda")
        sa = torch.full((N,), 0.01, device="cuda")
        sw = torch.full((4 * D,), 0.01, device="cuda")
        b = torch.zeros(4 * D, device="cuda")
        out = torch.empty((N, 4 * D), dtype=torch.bfloat16, device="cuda")
        tile = 256 | (R.TILE_PAIR if name != "fc1_fp8" else 0)
        launch = lambda: R.op_linear_fp8(2, a, sa, w, sw, b, out, N, 4 * D, D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    elif name in ("fc1_tick", "fc2_tick", "proj_tick"):  # the tick's RGB rows (M = 70200), CTA-pair 256 tiles
        # nbytes: the operands read once and the output written once (the
        # residual epilogue's float32 x read and written).
        Mt = sum(tick_segments(True))
        if name == "fc1_tick":
            a = torch.randn((Mt, D), device="cuda").to(torch.bfloat16)
            w = (torch.randn((4 * D, D), device="cuda") / 28).to(torch.bfloat16)
            b = torch.zeros(4 * D, device="cuda")
            out = torch.empty((Mt, 4 * D), dtype=torch.bfloat16, device="cuda")
            launch = lambda: R.op_linear(R.BF16, 2, a, w, b, out, Mt, 4 * D, D, 256 | R.TILE_PAIR,  # noqa: E731
                                         stream=stream)
            Kt, Nt, ob = D, 4 * D, 2
        else:
            Kt = 4 * D if name == "fc2_tick" else D
            a = torch.randn((Mt, Kt), device="cuda").to(torch.bfloat16)
            w = (torch.randn((D, Kt), device="cuda") / (56 if name == "fc2_tick" else 28)).to(torch.bfloat16)
            b = torch.zeros(D, device="cuda")
            out = torch.zeros((Mt, D), device="cuda")
            launch = lambda: R.op_linear(R.BF16, 3, a, w, b, out, Mt, D, Kt, 256 | R.TILE_PAIR,  # noqa: E731
                                         stream=stream)
            Nt, ob = D, 8
        flops = 2 * Mt * Nt * Kt
        nbytes = Mt * Kt * 2 + Nt * Kt * 2 + Mt * Nt * ob
    elif name == "layernorm_tick":  # LayerNorm over the tick's RGB rows: x float32 -> h bf16 (the GEMMs' A)
        Mt = sum(tick_segments(True))
        x = torch.randn((Mt, D), device="cuda")
        g = 1 + 0.1 * torch.rand(D, device="cuda")
        b = 0.02 * torch.rand(D, device="cuda")
        h = torch.empty((Mt, D), dtype=torch.bfloat16, device="cuda")
        launch = lambda: R.op_layernorm(x, g, b, h, Mt, D, 1, stream=stream)  # noqa: E731
        flops, nbytes = None, Mt * D * (4 + 2) + 2 * D * 4
    elif name in ("fc2", "fc2_pair"):  # fc2 of an encoder block: residual f32 += [N, 3072] x [768, 3072]^T
        a = torch.randn((N, 4 * D), device="cuda").to(torch.bfloat16)
        w = (torch.randn((D, 4 * D), device="cuda") / 56).to(torch.bfloat16)
        b = torch.zeros(D, device="cuda")
        out = torch.zeros((N, D), device="cuda")
        tile = 256 | (R.TILE_PAIR if name == "fc2_pair" else 0)
        launch = lambda: R.op_linear(R.BF16, 3, a, w, b, out, N, D, 4 * D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    else:  # fc1 of an encoder block: [N, 768] x [3072, 768]^T + GELU (fc1_pair: 256-row tiles on CTA pairs)
        a = torch.randn((N, D), device="cuda").to(torch.bfloat16)
        w = (torch.randn((4 * D, D), device="cuda") / 28).to(torch.bfloat16)
        b = torch.zeros(4 * D, device="cuda")
        out = torch.empty((N, 4 * D), dtype=torch.bfloat16, device="cuda")
        tile = 256 | (R.TILE_PAIR if name == "fc1_pair" else 0)
        launch = lambda: R.op_linear(R.BF16, 2, a, w, b, out, N, 4 * D, D, tile, stream=stream)  # noqa: E731
        flops = 2 * N * D * 4 * D
    return launch, flops, nbytes


def run_profile_kernel(args) -> None:
    """Launches one kernel of the step at the bench's shape (for ncu captures):
    W warm-up + K timed launches on one stream, CUDA-event timed."""
    import torch

    import paper_2604_27441_b300 as R
    stream = torch.cuda.Stream()
    if args.profile_kernel == "embed":  # the implicit-GEMM tubelet embedding inside one 640x480 RGB-D request
        import synth
        cfg = R.config(**VITB, precision=R.BF16, max_height=480, max_width=640, max_streams=1, max_batch=1,
                       use_graphs=1, autotune=0)
        ctx = R.Context(cfg, synth.flatten(synth.weights(synth.RGB, seed=0)),
                        synth.flatten(synth.weights(synth.DEPTH, seed=1)), stream=stream)
        sio = StreamIO(R, torch, ctx, 0, "640x480", 4100, 0.2, 1, True)
        for _ in range(args.warmup):
            ctx.poll(ctx.submit(sio.reqs[0]))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.poll(ctx.submit(sio.reqs[0]))
        print(json.dumps({"kernel": "embed (whole requests)", "us_per_request": (time.perf_counter() - t0) * 1e6 /
                          args.steps, "device_error": R.take_device_error()}))
        ctx.close()
        return
    launch, flops, nbytes = profile_launch(R, torch, args.profile_kernel, stream)
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
    ap.add_argument("--profile-kernel", choices=["embed", "embed_tick", "embed_tick_separate", "embed_tick_depth",
                                                 "embed_tick_depth_separate", "attention",
                                                 "attention_split", "attention_tick", "fc1", "fc1_pair",
                                                 "fc1_fp8", "fc1_fp8_pair", "fc1_fp8_tick", "fc2", "fc2_pair",
                                                 "fc1_tick", "fc2_tick", "proj_tick", "layernorm_tick",
                                                 "assemble", "blend", "pe"],
                    default=None, help="only launch one kernel of the step (for profiler captures)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the FP64 oracle (quality and cpu_baseline)")
    ap.add_argument("--no-graphs", action="store_true", help="plain kernel launches instead of graph replay")
    ap.add_argument("--quick", action="store_true", help="the tick and its e2e only")
    ap.add_argument("--serial-models", action="store_true",
                    help="the tick's RGB and depth forwards one after the other instead of side by side")
    ap.add_argument("--workload", choices=["mixed16", "640x480", "serving", "kt"], default="mixed16",
                    help="mixed16: the headline line; 640x480: batch-1 frames only; serving: the real-time loop "
                         "only; kt: the k/T latency sweep")
    ap.add_argument("--serve-streams", "--streams", dest="serve_streams", type=int, default=8)
    ap.add_argument("--seconds", type=float, default=20.0)
    ap.add_argument("--serve-warmup", type=float, default=3.0)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--lanes", type=int, default=2)
    ap.add_argument("--oracle-frames", type=int, default=2, help="320x240 RGB-D frames the cpu_baseline times")
    ap.add_argument("--in-flight", type=int, default=2,
                    help="640x480 workload: batch-1 frames in flight (one lane each); 1 = submit, wait, repeat")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_kernel:
        run_profile_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "640x480":
        run_640(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "kt":
        run_kt(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
