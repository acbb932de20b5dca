"""grin_trace_host_static: the trace entry point that allocates nothing.

It is for callers that may not call cudaMalloc; it reads the medium
description directly and stages rays and results in one fixed device array.
These checks go through the C ABI: two calls in a row must each give the
results of the ordinary host-buffer entry point (grin_trace_host with a
context and a medium), within the tolerance the other mixed-precision tests
use, and a batch over the fixed capacity must be refused.  This file is
collected last so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_22655_b300 import _native as N
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W
from tests.compare import compare

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _call_static(lib, desc, rays_host, dopl, max_steps, precision):
    out = tracer.empty_result(rays_host.count, "cpu")
    rs = tracer._rays_struct(rays_host)
    ps = tracer._params(dopl, max_steps, precision)
    os_ = tracer._out_struct(out)
    rc = lib.grin_trace_host_static(ctypes.byref(desc), ctypes.byref(rs), ctypes.byref(ps),
                                    ctypes.byref(os_), None)
    return rc, out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
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
        rep = compare(tracer.to_numpy(out), ref, wl.l_ref)
        assert rep["int_mismatch_unflagged"] == 0, rep
        assert max(rep["pos"], rep["dir"], rep["opl"]) <= TOL32, rep
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
