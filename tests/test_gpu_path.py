"""grin_trace_path, the trajectory tap, through the C ABI.

The recorded polyline of every ray (the vertices P_i of Eq. 2: the first
interior point, every full step, every step cut at the surface) must be
bitwise the oracle's, since the plain FP64 tracer follows the oracle's
operations in the same order.  The exit states must be bitwise those of
grin_trace at GRIN_PREC_FP64.  Media: the freeform block (box), the
Luneburg lens (sphere, n = sqrt(p)), a homogeneous box whose side walls
reflect the rays (boundary TIR), a graded fibre (cylinder, internal TIR), the
spherical freeform medium of Sec. V, a blob grid and its layered version."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tracer.Context(0)
    yield c
    c.close()


def _fiber_rays(n):
    x = W.uniform(4, 1, n, -4.0, 4.0)
    y = W.uniform(4, 2, n, -3.0, 3.0)
    d = W.direction(W.uniform(4, 3, n, 0.0, math.radians(40)), W.uniform(4, 4, n, 0, 2 * math.pi))
    return W.Rays(np.stack([x, y, np.full(n, -1.0)], 1), d)


def _cases():
    ff = W.freeform_workload(6)
    lun = W.luneburg_workload()
    lun_rays = lun.rays.subset(np.arange(0, lun.rays.n, 700))
    blob = W.blob_workload(n_rays=5, res=32)
    lay = W.blob_workload(n_rays=5, res=32, n_levels=32)
    box = W.homogeneous_box(1.5, lo=(-1.0, -1.0, 0.0), hi=(1.0, 1.0, 20.0))
    th = np.radians([20.0, 30.0, 38.0, 42.0])
    box_rays = W.Rays(np.tile([0.0, 0.0, -1.0], (4, 1)), W.direction(th, np.radians([0.0, 20.0, 45.0, 80.0])))
    return [("freeform", ff.medium, ff.rays, ff.dopl, 20000),
            ("box_tir", box, box_rays, 0.01, 40000),
            ("luneburg", lun.medium, lun_rays, lun.dopl, lun.max_steps),
            ("fiber", W.fiber_medium(length=20.0), _fiber_rays(5), 2e-3, 40000),
            ("spherical", W.spherical_freeform_medium(), W.spherical_workload(5).rays, 1e-3, 20000),
            ("grid", blob.medium, blob.rays, 0.02, 5000),
            ("layered", lay.medium, lay.rays, 0.02, 5000)]


def _trace(ctx, medium, rays, dopl, max_steps, cap):
    med = tracer.Medium(ctx, medium)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    out, pts, cnt = tracer.trace_path(ctx, med, rb, dopl, max_steps, cap)
    ref = tracer.trace(ctx, med, rb, dopl, max_steps, "fp64")
    torch.cuda.synchronize()
    assert ctx.last_launches() == 1
    return tracer.to_numpy(out), pts.cpu().numpy(), cnt.cpu().numpy(), tracer.to_numpy(ref)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_path_equals_oracle_bitwise(ctx, case):
    name, medium, rays, dopl, max_steps = case
    cap = max_steps + 2
    g, pts, cnt, ref = _trace(ctx, medium, rays, dopl, max_steps, cap)
    for k in g:
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    for r in range(rays.n):
        o, opath = oracle.trace_path(medium, rays.origins[r], rays.dirs[r], dopl, max_steps, cap)
        assert cnt[r] == len(opath), (name, r)
        np.testing.assert_array_equal(pts[r, :cnt[r]], opath, err_msg=f"{name} ray {r}")
        assert g["exit_id"][r] == o["exit_id"][0]
        if cnt[r] and g["exit_id"][r] >= 0:
            # the exit point is the last vertex
            np.testing.assert_array_equal(pts[r, cnt[r] - 1], g["P"][r])
    if name == "fiber":
        assert (g["tir_internal"] > 0).any()
    if name == "box_tir":
        assert (g["tir_boundary"] > 0).all()


def test_path_cap_truncates_storage_not_trace(ctx):
    wl = W.freeform_workload(4)
    cap = 100
    g, pts, cnt, ref = _trace(ctx, wl.medium, wl.rays, wl.dopl, 20000, cap)
    for k in g:
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    assert (cnt > cap).all() and (cnt == g["steps"] + 1).all()
    for r in range(wl.rays.n):
        _, opath = oracle.trace_path(wl.medium, wl.rays.origins[r], wl.rays.dirs[r], wl.dopl, 20000, cap)
        np.testing.assert_array_equal(pts[r], opath)


def test_path_argument_errors(ctx):
    wl = W.freeform_workload(4)
    med = tracer.Medium(ctx, wl.medium)
    rb = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cuda")
    out = tracer.empty_result(rb.count, "cuda")
    pts = torch.zeros((rb.count, 8, 3), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(rb.count, dtype=torch.int64, device="cuda")
    import ctypes
    call = lambda prec, cap, p, c: ctx.lib.grin_trace_path(
        ctx.handle, med.handle, ctypes.byref(tracer._rays_struct(rb)),
        ctypes.byref(tracer._params(wl.dopl, 100, prec)), ctypes.byref(tracer._out_struct(out)),
        ctypes.c_void_p(p), cap, ctypes.c_void_p(c), None)
    assert call("mixed", 8, pts.data_ptr(), cnt.data_ptr()) == tracer.N.GRIN_ERR_INVALID_ARG
    assert call("fp64", 0, pts.data_ptr(), cnt.data_ptr()) == tracer.N.GRIN_ERR_INVALID_ARG
    assert call("fp64", 8, 0, cnt.data_ptr()) == tracer.N.GRIN_ERR_INVALID_ARG
    assert call("fp64", 8, pts.data_ptr(), 0) == tracer.N.GRIN_ERR_INVALID_ARG
    assert call("fp64", 8, pts.data_ptr(), cnt.data_ptr()) == tracer.N.GRIN_OK
    torch.cuda.synchronize()
