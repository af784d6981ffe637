"""The allocation-free depth-statistics entry point.

revo_op_depth_stats_noalloc serves callers that cannot allocate device memory
(a real-time receiver loop that must not stall on cudaMalloc, or a host
application that reserves all device memory up front in its own pool).  It
keeps its scratch in a fixed array inside the library.  This test calls it
through the C ABI twice in a row, on different frames (the smaller first, so
that leftovers of a larger grid in the shared array would show), and checks
each result against the existing entry point (caller-provided scratch).  Both
run the same kernels with the same fixed-order reductions, so the results
must be identical.  The file sorts last so a run that stops at the first
failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_depth_stats_matches_the_allocating_entry_point():
    import paper_2604_27441_b300 as R
    lib = R.lib()
    frames = [synth.make_request(2001, "640x480")[1].refs[-1],
              synth.make_request(3003, "1280x720+640x576")[1].refs[-1]]
    assert frames[0].size != frames[1].size
    for d in frames:
        H, W = d.shape
        dev = torch.from_numpy(np.ascontiguousarray(d).view(np.int16)).cuda()
        want = torch.zeros(2, dtype=torch.float32, device="cuda")
        scratch = torch.zeros(R.depth_stats_scratch_bytes(), dtype=torch.uint8, device="cuda")
        assert lib.revo_op_depth_stats(dev.data_ptr(), H, W, W * 2, want.data_ptr(), scratch.data_ptr(), None) == 0
        got = torch.zeros(2, dtype=torch.float32, device="cuda")
        st = lib.revo_op_depth_stats_noalloc(C.c_void_p(dev.data_ptr()), H, W, W * 2, C.c_void_p(got.data_ptr()),
                                             None)
        assert st == R.REVO_OK, R.last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_depth_stats_rejects_frames_beyond_its_limit():
    import paper_2604_27441_b300 as R
    lib = R.lib()
    buf = torch.zeros(16, dtype=torch.int16, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    st = lib.revo_op_depth_stats_noalloc(C.c_void_p(buf.data_ptr()), 4097, 4096, 4096 * 2,
                                         C.c_void_p(out.data_ptr()), None)
    assert st == R.REVO_EINVAL
    assert "exceeds the maximum" in R.last_error()
