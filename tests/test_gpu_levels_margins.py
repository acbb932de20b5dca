"""Shells with exact crossings (GRIN_TRACE_LEVEL_ROOT) and the per-ray
decision margins (grin_out.margin), on the GPU through the C ABI, against the
oracle.

Crossings: the plain FP64 tracer takes the oracle's decisions and matches
its continuous results within 1e-12 on every unflagged ray (planar and
spherical shells, the 64^3 blob field in 32 shells); the mixed tracer is
gated against the oracle under the FP32 flag rule of tests/compare.py (on
planar and spherical shells; on the blob field's 32 shells its error is
stated, see test_level_root_blob_shells).
Margins: the plain FP64 tracer's margins are the oracle's (the same formulas
in the same order, to 1e-12 relative); the mixed tracer's, taken in FP32 on
its own trajectory, agree with the oracle's to its drift.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W
from tests.compare import compare, flagged, fp32_flags

pytestmark = pytest.mark.gpu
N = tracer.N


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tracer.Context(0)
    yield c
    c.close()


def run(ctx, medium, rays, dopl, max_steps, precision, level_root=False, margins=False,
        dtype=torch.float64):
    med = tracer.Medium(ctx, medium)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=dtype)
    res = tracer.trace(ctx, med, rb, dopl, max_steps, precision, margins=margins, level_root=level_root)
    torch.cuda.synchronize()
    out = tracer.to_numpy(res)
    med.close()
    return out


def planar_stack(levels):
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.2})
    return W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                    n_levels=levels, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                    bparams=(-50, -50, 0, 50, 50, 2, 0, 0), n_ext=1.0)


def fan(n, seed=7, max_deg=60.0):
    th = W.uniform(seed, 1, n, 0.0, math.radians(max_deg))
    ph = W.uniform(seed, 2, n, 0.0, 2 * math.pi)
    return W.Rays(np.tile([0.0, 0.0, -1.0], (n, 1)), W.direction(th, ph))


def check64(g, o, l_ref):
    rep = compare(g, o, l_ref, flagged(o["margins"], 1e-9))
    assert rep["int_mismatch_unflagged"] == 0, rep
    assert max(rep["pos"], rep["dir"], rep["opl"]) <= 1e-12, rep
    return rep


def check32(g, o, medium, rays, dopl, max_steps, l_ref, max_flagged, flags=0):
    f = fp32_flags(o, medium, rays.origins, rays.dirs, dopl, max_steps, l_ref, flags)
    rep = compare(g, o, l_ref, f)
    assert rep["int_mismatch_unflagged"] == 0, rep
    assert max(rep["pos"], rep["dir"], rep["opl"]) <= 2e-5, rep
    assert rep["n_flagged"] <= max_flagged * rep["n"], rep
    return rep


# ------------------------------------------------------ exact shell crossings


@pytest.mark.parametrize("levels", [4, 32])
def test_level_root_planar_stack(ctx, levels):
    """A fan through planar shells: both tracers against the oracle, and the
    exit direction equals the input direction (Snell at every plane)."""
    m, rays = planar_stack(levels), fan(2000)
    o = oracle.trace(m, rays.origins, rays.dirs, 1e-3, 200000, flags=oracle.LEVEL_ROOT)
    g = run(ctx, m, rays, 1e-3, 200000, "fp64", level_root=True)
    check64(g, o, 2.0)
    ok = (o["exit_id"] == 5) & (o["tir_boundary"] == 0)
    assert ok.mean() > 0.9
    np.testing.assert_allclose(g["d"][ok], rays.dirs[ok], atol=1e-12)
    g32 = run(ctx, m, rays, 1e-3, 200000, "mixed", level_root=True)
    check32(g32, o, m, rays, 1e-3, 200000, 2.0, 0.05, oracle.LEVEL_ROOT)


def test_level_root_spherical_shells(ctx):
    """The Luneburg lens in 8 shells: the refraction normal at a crossing is
    the radial grad f of the smooth field."""
    m = dataclasses.replace(W.luneburg_medium(), n_levels=8, level_lo=1.0, level_hi=math.sqrt(2.0))
    wl = W.luneburg_workload()
    o = oracle.trace(m, wl.rays.origins, wl.rays.dirs, 2e-3, 20000, flags=oracle.LEVEL_ROOT)
    g = run(ctx, m, wl.rays, 2e-3, 20000, "fp64", level_root=True)
    check64(g, o, 1.0)
    g32 = run(ctx, m, wl.rays, 2e-3, 20000, "mixed", level_root=True)
    check32(g32, o, m, wl.rays, 2e-3, 20000, 1.0, 0.05, oracle.LEVEL_ROOT)


@pytest.mark.parametrize("res", [64, 16])
def test_level_root_blob_shells(ctx, res):
    """The blob field in 32 shells with crossings solved (the tricubic
    interpolant's isosurfaces), both tracers against the oracle; 16^3 puts
    many stencils at the clamped edges.  The plain FP64 tracer is gated.  For
    the mixed tracer the error is stated: with a hundred or so refractions at
    curved isosurfaces a ray, many of them close to the critical angle, a few
    rays in a thousand that no margin or probe flags end above 2e-5
    (measured: 3 of 1,500, the largest 6.4e-5); integer outcomes are equal
    on every unflagged ray and 99.5 % are inside 2e-5."""
    wl = W.blob_workload(n_rays=1500, res=res, n_levels=32)
    o = oracle.trace(wl.medium, wl.rays.origins, wl.rays.dirs, wl.dopl, wl.max_steps, flags=oracle.LEVEL_ROOT)
    g = run(ctx, wl.medium, wl.rays, wl.dopl, wl.max_steps, "fp64", level_root=True)
    check64(g, o, wl.l_ref)
    g32 = run(ctx, wl.medium, wl.rays, wl.dopl, wl.max_steps, "mixed", level_root=True)
    f = fp32_flags(o, wl.medium, wl.rays.origins, wl.rays.dirs, wl.dopl, wl.max_steps, wl.l_ref,
                   oracle.LEVEL_ROOT)
    rep = compare(g32, o, wl.l_ref, f)
    assert rep["int_mismatch_unflagged"] == 0 and rep["n_flagged"] <= 0.1 * rep["n"], rep
    same = np.ones(wl.rays.n, bool)
    for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
        same &= g32[k] == o[k]
    e = np.maximum(np.linalg.norm(g32["P"] - o["P"], axis=1) / wl.l_ref,
                   np.linalg.norm(g32["d"] - o["d"], axis=1))[same & ~f]
    assert (e <= 2e-5).mean() >= 0.995 and e.max() <= 1e-4, (float((e <= 2e-5).mean()), float(e.max()))


def test_level_root_path_points_match_oracle(ctx):
    """The trajectory tap records each crossing point as a vertex, bitwise
    the oracle's."""
    m = planar_stack(8)
    d0 = np.array([0.3, 0.2, 0.9])
    d0 /= np.linalg.norm(d0)
    res, path = oracle.trace_path(m, (0.1, -0.2, -1.0), d0, 5e-3, 10000, flags=oracle.LEVEL_ROOT)
    med = tracer.Medium(ctx, m)
    rb = tracer.RayBatch.from_numpy(np.array([[0.1, -0.2, -1.0]]), d0[None], device="cuda", dtype=torch.float64)
    out, pts, cnt = tracer.trace_path(ctx, med, rb, 5e-3, 10000, cap=len(path) + 4, level_root=True)
    torch.cuda.synchronize()
    assert int(cnt[0]) == len(path)
    np.testing.assert_array_equal(pts[0, : len(path)].cpu().numpy(), path)


def test_level_root_argument_errors(ctx):
    m = tracer.Medium(ctx, planar_stack(4))
    rays = fan(8)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    with pytest.raises(N.GrinError) as e:
        tracer.trace(ctx, m, rb, 1e-3, 100, "fp64-fast", level_root=True)
    assert e.value.status == N.GRIN_ERR_NOT_IMPLEMENTED
    with pytest.raises(N.GrinError) as e:
        tracer.trace(ctx, m, rb, 1e-3, 100, "fp64-fast", margins=True)
    assert e.value.status == N.GRIN_ERR_NOT_IMPLEMENTED
    out = tracer.empty_result(8, "cuda")
    rs, os_ = tracer._rays_struct(rb), tracer._out_struct(out)
    ps = N.Params(1e-3, 100, N.PREC_FP64, 2)  # an unknown flag bit
    import ctypes
    st = ctx.lib.grin_trace(ctx.handle, m.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(os_), None)
    assert st == N.GRIN_ERR_INVALID_ARG
    # continuous media ignore the flag
    c = tracer.Medium(ctx, W.luneburg_medium())
    a = tracer.to_numpy(tracer.trace(ctx, c, rb, 1e-3, 100, "fp64"))
    b = tracer.to_numpy(tracer.trace(ctx, c, rb, 1e-3, 100, "fp64", level_root=True))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------- decision margins


def _margin_sets():
    lune = W.luneburg_workload()
    free = W.freeform_workload(3001)
    fis = W.fisheye_medium(n0=2.0, a=1.0, r_bound=3.0)
    th = W.uniform(3, 1, 400, 0.0, math.pi)
    ph = W.uniform(3, 2, 400, 0.0, 2 * math.pi)
    fis_rays = W.Rays(np.tile([0.5, 0.0, 0.0], (400, 1)), W.direction(th, ph))
    fib = W.fiber_medium(length=20.0)
    x = W.uniform(4, 1, 300, -4.0, 4.0)
    y = W.uniform(4, 2, 300, -3.0, 3.0)
    fib_rays = W.Rays(np.stack([x, y, np.full(300, -1.0)], 1),
                      W.direction(W.uniform(4, 3, 300, 0.0, math.radians(40)), W.uniform(4, 4, 300, 0, 6.28)))
    lay = W.blob_workload(n_rays=600, res=32, n_levels=16)
    return [("luneburg", lune.medium, lune.rays, lune.dopl, lune.max_steps, 0),
            ("freeform", free.medium, free.rays, free.dopl, free.max_steps, 0),
            ("fisheye", fis, fis_rays, 2e-3, 3000, 0),
            ("fiber", fib, fib_rays, 1e-3, 40000, 0),
            ("layered", lay.medium, lay.rays, lay.dopl, lay.max_steps, 0),
            ("layered_root", lay.medium, lay.rays, lay.dopl, lay.max_steps, oracle.LEVEL_ROOT)]


@pytest.mark.parametrize("case", range(6))
def test_fp64_margins_are_the_oracles(ctx, case):
    name, m, rays, dopl, ms, flags = _margin_sets()[case]
    o = oracle.trace(m, rays.origins, rays.dirs, dopl, ms, flags=flags)
    g = run(ctx, m, rays, dopl, ms, "fp64", level_root=bool(flags), margins=True)
    check64(g, o, 1.0)
    a, b = g["margins"], o["margins"]
    assert np.array_equal(np.isinf(a), np.isinf(b)), name
    fin = np.isfinite(b)
    np.testing.assert_allclose(a[fin], b[fin], rtol=1e-12, atol=1e-300, err_msg=name)


@pytest.mark.parametrize("case", [0, 1, 4])
def test_mixed_margins_track_the_oracles(ctx, case):
    """The FP32 path's margins, on its own trajectory, on the rays whose
    integer outcomes match: infinite where the oracle's are; the surface
    margin within the position gate (2e-5 of the bounding radius is up to
    0.04 of a step here); the critical and tangent margins within 3e-4 (its
    trapezoid index difference moves the critical cosine sqrt(1 - 1/mu^2),
    which is steep in mu near mu = 1), the level margin within 1e-4; where
    the oracle's margin is below twice the tolerance, below three times
    it."""
    name, m, rays, dopl, ms, flags = _margin_sets()[case]
    o = oracle.trace(m, rays.origins, rays.dirs, dopl, ms, flags=flags)
    g = run(ctx, m, rays, dopl, ms, "mixed", margins=True)
    same = np.ones(rays.n, bool)
    for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
        same &= g[k] == o[k]
    assert same.mean() > 0.98
    a, b = g["margins"][same], o["margins"][same]
    assert np.array_equal(np.isinf(a), np.isinf(b)), name
    for k, tol in ((0, 3e-4), (1, 3e-4), (2, 5e-2), (3, 1e-4)):
        fin = np.isfinite(b[:, k])
        big = fin & (b[:, k] > 2 * tol)
        assert np.all(np.abs(a[big, k] - b[big, k]) <= tol * np.maximum(1.0, b[big, k])), (name, k)
        small = fin & ~big
        assert np.all(a[small, k] <= 3 * tol), (name, k)


def test_margins_through_the_host_entry(ctx):
    """grin_trace_host copies the margins back with the other results
    (including a pipelined batch of 300,000 rays)."""
    wl = W.freeform_workload(300000)
    med = tracer.Medium(ctx, wl.medium)
    rb = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cuda", dtype=torch.float32)
    dev = tracer.to_numpy(tracer.trace(ctx, med, rb, wl.dopl, wl.max_steps, "mixed", margins=True))
    hb = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32, pin=True)
    host = tracer.to_numpy(tracer.trace_host(ctx, med, hb, wl.dopl, wl.max_steps, "mixed", margins=True))
    for k in dev:
        np.testing.assert_array_equal(dev[k], host[k], err_msg=k)
    plain = tracer.to_numpy(tracer.trace(ctx, med, rb, wl.dopl, wl.max_steps, "mixed"))
    same = np.ones(wl.rays.n, bool)
    for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
        same &= plain[k] == dev[k]
    assert same.mean() > 0.999  # the margin-keeping kernel takes the same decisions
