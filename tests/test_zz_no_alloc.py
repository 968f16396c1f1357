"""The allocation-free batch entry point (rt_trace_batch_noalloc).

It serves callers that cannot allocate device memory when they trace: a
real-time loop that must not stall on cudaMalloc or runs on a memory budget
fixed at start-up, or a host whose device memory is owned by another
allocator.  Its scratch lives in a static device array of the library
instead.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import corona_synth as cs

pytestmark = pytest.mark.gpu


def _requests(rt, reqs, fill):
    import torch
    from paper_2606_02413_gb300 import _abi
    arr = (_abi.Request * len(reqs))()
    outs, keep = [], []
    for i, r in enumerate(reqs):
        v = rt.view(r.view)
        f = np.ascontiguousarray(r.freqs_hz, dtype=np.float64)
        tb = torch.full((len(f), v.ny, v.nx), fill, dtype=torch.float32, device="cuda")
        keep += [v, f]
        outs.append(tb)
        arr[i] = _abi.Request(C.pointer(v), f.ctypes.data_as(C.POINTER(C.c_double)), len(f), tb.data_ptr(), None)
    return arr, outs, keep


def test_noalloc_batch_matches_trace_batch_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_02413_gb300 import _abi, build
    build.build()
    import paper_2606_02413_gb300 as rt
    L = _abi.lib()
    ctx = rt.Context(0)
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    reqs = cs.batch_requests(6, seed=11, sides=(8, 13, 32, 48), max_nf=5)
    opts = rt.options(precision=1)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    ref_arr, ref_out, keep_ref = _requests(rt, reqs, -1.0)
    assert L.rt_trace_batch(ctx.handle, grid.handle, ref_arr, len(reqs), C.byref(opts), stream) == 0

    for call in range(2):  # the static scratch keeps the previous call's contents
        arr, outs, keep = _requests(rt, reqs, -7.0)
        rc = L.rt_trace_batch_noalloc(grid.handle, arr, len(reqs), C.byref(opts), stream)
        assert rc == 0, L.rt_last_error()
        torch.cuda.synchronize()
        for a, b in zip(outs, ref_out):  # the same rays with the same arithmetic: identical maps
            assert torch.equal(a, b), f"call {call}"

    # a batch larger than the static scratch is refused with a clear error
    big = [cs.Request(cs.View(0.0, 0.0, 2048, 2048, -2.5, 2.5, -2.5, 2.5), np.array([1e8] * 8))]
    big_arr = (_abi.Request * 1)()
    vb = rt.view(big[0].view)
    fb = np.ascontiguousarray(big[0].freqs_hz)
    big_arr[0] = _abi.Request(C.pointer(vb), fb.ctypes.data_as(C.POINTER(C.c_double)), 8, 1, None)
    rc = L.rt_trace_batch_noalloc(grid.handle, big_arr, 1, C.byref(opts), stream)
    assert rc == _abi.RT_ERR_ARG and b"scratch" in L.rt_last_error()
