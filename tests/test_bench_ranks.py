"""The benchmark's multi-rank logic on CPU: two gloo ranks, each timing its own
independent replica; the job rate uses every rank's frames over the slowest
rank's time, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [2.0, 3.0][rank]           # rank 1 is the slower replica
    bench.rank_barrier(world)
    m = bench.rank_max(secs, world)
    rate = bench.whole_job_rate(30, m, world)
    # The reference arm prints on rank 0 only; other ranks return without work.
    buf = io.StringIO()
    if rank == 1:
        class A:
            steps, warmup, gpus = 1, 3, world
        with redirect_stdout(buf):
            bench.run_reference(A())
    out.put((rank, m, rate, buf.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate, printed in res:
        assert m == 3.0
        assert rate == pytest.approx(2 * 30 / 3.0)
        if rank == 1:
            assert printed == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(1.5, 1) == 1.5
    assert bench.whole_job_rate(10, 2.0, 1) == 5.0


def test_serving_arrival_schedule():
    """30 frames/s per stream, jitter within +-5 ms, frames numbered in order."""
    import numpy as np
    import bench
    ev = bench.arrival_schedule(4, 2.0, np.random.default_rng(1))
    assert [t for t, _, _ in ev] == sorted(t for t, _, _ in ev)
    for sid in range(4):
        mine = [(t, n) for t, s, n in ev if s == sid]
        assert [n for _, n in mine] == list(range(len(mine)))
        assert 58 <= len(mine) <= 61
        for t, n in mine:
            assert abs(t - (mine[0][0] + n * 1000 / 30)) <= 10 + 1e-9


def test_mixed16_proportions():
    import bench
    assert len(bench.MIX16) == 16
    assert bench.MIX16.count("320x240") == 6 and bench.MIX16.count("640x480") == 6
    assert bench.MIX16.count("1280x720+640x576") == 4
    assert sorted(set(bench.MIX16[:3])) == sorted(set(bench.MIX16))
