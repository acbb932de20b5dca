"""grin_trace_host_static: the trace entry point that allocates nothing.

It is for callers that may not call cudaMalloc; it reads the medium
description directly and stages rays and results in one fixed device array.
These checks go through the C ABI: two calls in a row must each give the
results of the ordinary host-buffer entry point (grin_trace_host with a
context and a medium) bit for bit -- both build the medium's device record
with the same routine and run the same kernel on the same inputs -- and a
batch over the fixed capacity must be refused.  This file is collected last
so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_22655_b300 import _native as N
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _call_static(lib, desc, rays_host, dopl, max_steps, precision, stream=None):
    out = tracer.empty_result(rays_host.count, "cpu")
    rs = tracer._rays_struct(rays_host)
    ps = tracer._params(dopl, max_steps, precision)
    os_ = tracer._out_struct(out)
    rc = lib.grin_trace_host_static(ctypes.byref(desc), ctypes.byref(rs), ctypes.byref(ps),
                                    ctypes.byref(os_), stream)
    return rc, out


@pytest.mark.parametrize("precision", ["mixed", "fp64", "fp64-fast"])
def test_static_entry_matches_host_entry_on_two_calls(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = N.load()
    wl = W.freeform_workload(5000)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32)
    ctx = tracer.Context(0)
    med = tracer.Medium(ctx, wl.medium)
    ref = tracer.to_numpy(tracer.trace_host(ctx, med, rays, wl.dopl, wl.max_steps, precision))
    desc, keep = tracer.medium_desc(wl.medium)
    for _ in range(2):
        rc, out = _call_static(lib, desc, rays, wl.dopl, wl.max_steps, precision)
        assert rc == 0, N.STATUS.get(rc, rc)
        got = tracer.to_numpy(out)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    med.close()
    ctx.close()


def test_static_entry_refuses_oversized_batches_and_grids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = N.load()
    wl = W.freeform_workload(N.STATIC_MAX_RAYS + 1)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32)
    desc, keep = tracer.medium_desc(wl.medium)
    rc, _ = _call_static(lib, desc, rays, wl.dopl, wl.max_steps, "mixed")
    assert rc == -1
    g = W.grid_medium(np.full((4, 4, 4), 1.5, np.float32), 1.0, size=3.0)
    gdesc, gkeep = tracer.medium_desc(g)
    small = tracer.RayBatch.from_numpy(wl.rays.origins[:8], wl.rays.dirs[:8], device="cpu",
                                       dtype=torch.float32)
    rc, _ = _call_static(lib, gdesc, small, wl.dopl, 10, "mixed")
    assert rc == -1


def test_static_entry_refuses_a_capturing_stream():
    """The call copies into host buffers and synchronises its stream, which
    graph capture does not allow: on a stream being captured it returns
    GRIN_ERR_INVALID_ARG without queuing anything, and the capture of the
    caller's own work goes on."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = N.load()
    wl = W.freeform_workload(64)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32)
    desc, keep = tracer.medium_desc(wl.medium)
    x = torch.zeros(16, device="cuda")
    graph, side = torch.cuda.CUDAGraph(), torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        rc, _ = _call_static(lib, desc, rays, wl.dopl, wl.max_steps, "mixed",
                             stream=ctypes.c_void_p(side.cuda_stream))
    assert rc == N.GRIN_ERR_INVALID_ARG
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    rc, out = _call_static(lib, desc, rays, wl.dopl, wl.max_steps, "mixed")
    assert rc == 0 and (tracer.to_numpy(out)["exit_id"] >= 0).any()
