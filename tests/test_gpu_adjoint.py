"""Reverse-mode adjoint (grin_trace_adjoint) against central finite
differences of the FP64 oracle and, for polynomial coefficients, against the
oracle's forward-mode (tangent) gradient.

Loss: mean squared distance, in the plane z = 30 mm, between where each
ray's exit line crosses the plane and a seeded target spot (16 spots, ray i
to spot i mod 16).  Parameters: the 35 coefficients of the freeform block
(n = p) and, separately, samples of a 64^3 blob grid.  Central differences
with h = 1e-6 of the same loss computed from oracle traces; coordinates whose
+-h traces change any integer outcome (exit id, steps, TIR counts) are
excluded and counted.  Bound: 1e-4 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2606_22655_b300 import _native as N
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W

pytestmark = pytest.mark.gpu

Z_IMG = 30.0
H = 1e-6
REL = 1e-4
# Rays left out of a coordinate's finite difference: those whose +-h traces
# change an integer outcome (a step-count tie at the exit face, a TIR that
# appears or goes), and those whose differences at the two step sizes
# disagree by more than 1e-4 (a kink of the discrete map within the step:
# Eq. 9's sgn(N.I) flips where a ray turns, N.I through zero).  The gridded
# medium loses 0.4 % of ray-coordinate pairs this way; the freeform block,
# whose rays turn in the field, about 47 % to kinks (and 2 % to integer
# changes at h = 1e-6): there the oracle's forward-mode tangents, exact
# derivatives of the same map, check every ray instead (the tangent tests
# below keep all of them).
KEPT_FLOOR_GRID = 0.95
KEPT_FLOOR_POLY = 0.45
INT_KEYS = ("exit_id", "steps", "tir_internal", "tir_boundary")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tracer.Context(0)
    yield c
    c.close()


def np_loss(res, targets, mask=None):
    P, d, ex = res["P"], res["d"], res["exit_id"]
    sig = (Z_IMG - P[:, 2]) / d[:, 2]
    X = P[:, 0] + sig * d[:, 0]
    Y = P[:, 1] + sig * d[:, 1]
    e = (X - targets[:, 0]) ** 2 + (Y - targets[:, 1]) ** 2
    keep = ex >= 0 if mask is None else (ex >= 0) & mask
    return float(np.where(keep, e, 0.0).sum() / P.shape[0])


def stable(a, b):
    """Rays with identical integer outcomes in the two traces."""
    ok = np.ones(len(a["exit_id"]), bool)
    for k in INT_KEYS:
        ok &= a[k] == b[k]
    return ok


def adjoint_grad(ctx, spec, theta0, rays, targets, dopl, max_steps, k, mask=None):
    theta = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    P, d, opl, ex = tracer.traced_exit(theta, ctx, spec, rb, dopl, max_steps, k)
    tg = torch.tensor(targets, device="cuda")
    mk = None if mask is None else torch.tensor(mask, device="cuda")
    L = tracer.image_plane_loss(P, d, ex, tg, Z_IMG, mk)
    L.backward()
    return float(L), theta.grad.cpu().numpy()


def per_ray_loss(res, targets):
    P, d, ex = res["P"], res["d"], res["exit_id"]
    sig = (Z_IMG - P[:, 2]) / d[:, 2]
    X = P[:, 0] + sig * d[:, 0]
    Y = P[:, 1] + sig * d[:, 1]
    return np.where(ex >= 0, (X - targets[:, 0]) ** 2 + (Y - targets[:, 1]) ** 2, 0.0)


def smooth_fd(trace_at, base, targets, steps):
    """Per-ray central differences at the two perturbation sizes `steps`
    (realised parameter deltas returned by trace_at) and the rays whose
    differences agree to 1e-4 beyond their rounding noise (a few ulps of the
    ray's loss over the step); returns (fd per ray at the smaller size,
    keep)."""
    fds, noise = [], []
    keep = np.ones(len(base["exit_id"]), bool)
    smooth_fd.counts = getattr(smooth_fd, "counts", np.zeros(3, np.int64))
    eps = np.finfo(np.float64).eps
    for h in steps:
        rp, vp = trace_at(+h)
        rm, vm = trace_at(-h)
        keep &= stable(rp, base) & stable(rm, base)
        lp, lm = per_ray_loss(rp, targets), per_ray_loss(rm, targets)
        fds.append((lp - lm) / (vp - vm))
        noise.append(64 * eps * (np.abs(lp) + np.abs(lm)) / abs(vp - vm))
    a, b = fds
    agree = np.abs(a - b) <= 1e-4 * np.abs(b) + noise[0] + noise[1]
    # tally: rays kept, rays whose integer outcomes change, rays whose two
    # differences disagree (a kink of the discrete map within the step)
    smooth_fd.counts += [int((keep & agree).sum()), int((~keep).sum()), int((keep & ~agree).sum())]
    smooth_fd.kink_margin = np.where(keep & ~agree, base["margins"][:, 1], np.nan)
    keep &= agree
    return b, keep


def check_coordinates(ctx, spec, theta0, rays, targets, dopl, max_steps, coords, trace_at_factory, steps):
    """Per coordinate: FD over the rays smooth for it, and the adjoint of the
    loss over the same rays.  Returns (the largest |adjoint - FD| / sum_r
    |FD_r|, the largest full-loss error |adjoint - FD| / |FD| over the
    coordinates whose FD does not cancel, |FD| >= 0.1 sum_r |FD_r|, and the
    mean fraction of rays kept)."""
    base = oracle.trace(spec, rays.origins, rays.dirs, dopl, max_steps)
    rows = []
    smooth_fd.counts = np.zeros(3, np.int64)
    kink_margins = []
    for i in coords:
        fd_ray, keep = smooth_fd(trace_at_factory(i), base, targets, steps)
        kink_margins.append(smooth_fd.kink_margin)
        fd = float(fd_ray[keep].sum()) / rays.n
        mag = float(np.abs(fd_ray[keep]).sum()) / rays.n
        L, g = adjoint_grad(ctx, spec, theta0, rays, targets, dopl, max_steps, 64, keep)
        assert L == pytest.approx(float(per_ray_loss(base, targets)[keep].sum()) / rays.n, rel=1e-12)
        rows.append((int(i), fd, float(g[i]), mag, float(keep.mean())))
    rows = [r for r in rows if r[3] > 0]
    errs = [abs(a - f) / m_ for _, f, a, m_, _ in rows]
    full = [abs(a - f) / abs(f) for _, f, a, m_, _ in rows if abs(f) >= 0.1 * m_]
    k = int(np.argmax(errs))
    c = smooth_fd.counts / smooth_fd.counts.sum()
    km = np.concatenate(kink_margins)
    print("ray-coordinate pairs: kept %.3f, integer outcome changed %.3f, kink within the step %.3f;"
          " min |N.I| over the kinked rays' steps: median %.2e (all rays: %.2e)"
          % (c[0], c[1], c[2], np.nanmedian(km) if np.isfinite(km).any() else np.nan,
             np.median(base["margins"][:, 1])))
    print("worst coordinate (index, fd, adjoint, sum|fd_r|, kept):", rows[k], "error", errs[k],
          "| full-loss error over", len(full), "coordinates:", max(full) if full else None,
          "| kept min", min(r[4] for r in rows))
    return max(errs), (max(full) if full else 0.0), float(np.mean([r[4] for r in rows]))


def test_polynomial_coefficients_against_oracle_fd(ctx):
    m = W.freeform_block_medium()
    rays = W.point_source_rays(384, W.BASE_SEED + 4)
    dopl, max_steps = 0.02, 20000
    targets = W.design_targets(rays.n)

    def factory(i):
        def at(h):
            mm = W.Medium(**{**m.__dict__})
            c = m.coeffs.copy()
            c[i] += h
            mm.coeffs = c
            return oracle.trace(mm, rays.origins, rays.dirs, dopl, max_steps), c[i]
        return at

    worst, full, kept = check_coordinates(ctx, m, m.coeffs, rays, targets, dopl, max_steps,
                                          range(len(m.coeffs)), factory, (1e-6, 2.5e-7))
    assert kept > KEPT_FLOOR_POLY, kept
    assert worst <= REL, (worst, kept)
    assert full <= REL, (full, kept)


def test_polynomial_coefficients_against_oracle_tangents(ctx):
    """The adjoint's gradient with respect to all 35 coefficients against the
    FP64 reference gradient formed from the oracle's forward-mode tangents,
    dL/dc_j = sum over rays of dL/d(P_r, d_r) . d(P_r, d_r)/dc_j.  Both are
    derivatives of the same discrete map with the same decisions, so they
    agree to rounding: within 1e-10 of sum_r |per-ray term| (the finite
    differences above can only check 1e-4).  Rays where the tangents do not
    follow (tangential incidence, a clamped crossing) are left out of the
    loss on both sides."""
    m = W.freeform_block_medium()
    rays = W.point_source_rays(384, W.BASE_SEED + 4)
    dopl, max_steps = 0.02, 20000
    targets = W.design_targets(rays.n)
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    keep = t["flag"] == 0
    ref, mag = tangent_gradient(t, targets, keep)
    _, g = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 64, keep)
    err = np.abs(g - ref) / np.maximum(mag, 1e-300)
    print("worst coefficient", int(err.argmax()), "error", float(err.max()), "kept", float(keep.mean()))
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, (float(err.max()), int(err.argmax()))


def tangent_gradient(t, targets, keep):
    """dL/dtheta_j of the image-plane loss from the oracle's tangents:
    sum over kept exiting rays of dL/d(P, d) . d(P, d)/dtheta_j, with
    X = P_x + s d_x, Y = P_y + s d_y, s = (Z - P_z) / d_z.  Returns the
    gradient and sum_r |per-ray term| per parameter."""
    P, d = t["P"], t["d"]
    n = P.shape[0]
    sig = (Z_IMG - P[:, 2]) / d[:, 2]
    ex = 2.0 * (P[:, 0] + sig * d[:, 0] - targets[:, 0])  # de/dX
    ey = 2.0 * (P[:, 1] + sig * d[:, 1] - targets[:, 1])  # de/dY
    w = np.where((t["exit_id"] >= 0) & keep, 1.0 / n, 0.0)
    lat = ex * d[:, 0] + ey * d[:, 1]
    gP = np.stack([ex, ey, -lat / d[:, 2]], 1) * w[:, None]
    gd = np.stack([ex * sig, ey * sig, -sig * lat / d[:, 2]], 1) * w[:, None]
    terms = np.einsum("rk,rjk->rj", gP, t["tP"]) + np.einsum("rk,rjk->rj", gd, t["td"])
    return terms.sum(0), np.abs(terms).sum(0)


def test_grid_samples_against_oracle_tangents(ctx):
    """The same FP64 reference for the gridded medium: the adjoint's gradient
    at 64 samples of the 64^3 blob grid (among those with a gradient above
    1e-2 of the largest) against the oracle's tangents with respect to those
    samples, within 1e-10 of sum_r |per-ray term|."""
    wl = W.blob_workload(n_rays=384, res=64)
    m = wl.medium
    dopl, max_steps = 0.02, 20000
    targets = W.design_targets(wl.rays.n) + 10.0  # spots around the cube's axis
    theta0 = m.grid.astype(np.float64).ravel()
    _, g_all = adjoint_grad(ctx, m, theta0, wl.rays, targets, dopl, max_steps, 64)
    cand = np.flatnonzero(np.abs(g_all) > 1e-2 * np.abs(g_all).max())
    coords = np.random.default_rng(3).choice(cand, size=min(64, cand.size), replace=False)
    t = oracle.trace_tangent(m, wl.rays.origins, wl.rays.dirs, dopl, max_steps, samples=coords)
    keep = t["flag"] == 0
    ref, mag = tangent_gradient(t, targets, keep)
    _, g = adjoint_grad(ctx, m, theta0, wl.rays, targets, dopl, max_steps, 64, keep)
    err = np.abs(g[coords] - ref) / np.maximum(mag, 1e-300)
    print("worst sample", int(coords[err.argmax()]), "error", float(err.max()), "kept", float(keep.mean()))
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, (float(err.max()), int(coords[err.argmax()]))


def test_grid_samples_against_oracle_fd(ctx):
    wl = W.blob_workload(n_rays=384, res=64)
    m = wl.medium
    dopl, max_steps = 0.02, 20000
    targets = W.design_targets(wl.rays.n) + 10.0  # spots around the cube's axis
    theta0 = m.grid.astype(np.float64).ravel()
    _, g_all = adjoint_grad(ctx, m, theta0, wl.rays, targets, dopl, max_steps, 64)
    cand = np.flatnonzero(np.abs(g_all) > 1e-2 * np.abs(g_all).max())
    coords = np.random.default_rng(3).choice(cand, size=min(64, cand.size), replace=False)
    flat = m.grid.ravel()

    def factory(i):
        def at(h):
            gr = flat.copy()
            gr[i] = np.float32(np.float64(gr[i]) + h)
            mm = W.Medium(**{**m.__dict__})
            mm.grid = gr.reshape(m.grid.shape)
            return oracle.trace(mm, wl.rays.origins, wl.rays.dirs, dopl, max_steps), float(gr[i])
        return at

    ulp = float(np.spacing(np.float32(1.5)))
    worst, full, kept = check_coordinates(ctx, m, theta0, wl.rays, targets, dopl, max_steps, coords, factory,
                                          (8 * ulp, 2 * ulp))
    assert kept > KEPT_FLOOR_GRID, kept
    assert worst <= REL, (worst, kept)
    assert full <= REL, (full, kept)


def test_checkpoint_interval_does_not_change_the_gradient(ctx):
    m = W.freeform_block_medium()
    rays = W.point_source_rays(512, W.BASE_SEED + 4)
    targets = W.design_targets(rays.n)
    _, g64 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 64)
    _, g7 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 7)
    _, g1 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 1)  # every step stored
    np.testing.assert_allclose(g7, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())


def test_stored_steps_grid_gradient_equals_recomputed(ctx):
    """On the blob grid, checkpoint_every = 1 (every step stored with its
    case, no recompute) gives the gradient of checkpoint_every = 64."""
    wl = W.blob_workload(n_rays=384, res=64)
    m = wl.medium
    targets = W.design_targets(wl.rays.n) + 10.0
    theta0 = m.grid.astype(np.float64).ravel()
    _, g64 = adjoint_grad(ctx, m, theta0, wl.rays, targets, 0.02, 20000, 64)
    _, g1 = adjoint_grad(ctx, m, theta0, wl.rays, targets, 0.02, 20000, 1)
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())


def test_optical_path_gradient_against_oracle_tangents(ctx):
    """The adjoint of the optical path (through the crossing fraction of the
    exit step, the only place OPL depends on the medium when every full step
    adds dL0): the gradient of the mean exit OPL with respect to the 35
    coefficients against the oracle's tangents, within 1e-10 of
    sum_r |per-ray term|."""
    m = W.freeform_block_medium()
    rays = W.point_source_rays(384, W.BASE_SEED + 4)
    dopl, max_steps = 0.02, 20000
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    keep = (t["flag"] == 0) & (t["exit_id"] >= 0)
    terms = t["topl"] * (keep / rays.n)[:, None]
    ref, mag = terms.sum(0), np.abs(terms).sum(0)
    theta = torch.tensor(m.coeffs, dtype=torch.float64, device="cuda", requires_grad=True)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    P, d, opl, ex = tracer.traced_exit(theta, ctx, m, rb, dopl, max_steps, 64)
    L = (opl * torch.tensor(keep, device="cuda")).sum() / rays.n
    L.backward()
    g = theta.grad.cpu().numpy()
    err = np.abs(g - ref) / np.maximum(mag, 1e-300)
    print("worst coefficient", int(err.argmax()), "error", float(err.max()), "kept", float(keep.mean()))
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, (float(err.max()), int(err.argmax()))


def test_split_sweeps_equal_the_one_call(ctx):
    """grin_trace_adjoint_forward then grin_trace_adjoint_backward (what the
    autograd function runs) against one grin_trace_adjoint call: the forward
    results bitwise, and equal to grin_trace FP64; the gradient to rounding
    (its per-ray terms are summed atomically, in no fixed order)."""
    for spec, rays, n_params in ((W.freeform_block_medium(), W.point_source_rays(2048, W.BASE_SEED + 4), 35),
                                 (W.blob_workload(n_rays=1024, res=32).medium,
                                  W.blob_workload(n_rays=1024, res=32).rays, 32 ** 3)):
        med = tracer.Medium(ctx, spec)
        rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
        gen = torch.Generator(device="cuda").manual_seed(5)
        grads = {k: torch.randn(rays.n, dtype=torch.float64, device="cuda", generator=gen)
                 for k in tracer.OUT_FIELDS}
        out1, g1 = tracer.trace_adjoint(ctx, med, rb, 0.02, 20000, grads, n_params, 16)
        out2, ws = tracer.trace_adjoint_forward(ctx, med, rb, 0.02, 20000, 16)
        g2 = tracer.trace_adjoint_backward(ctx, med, rb, 0.02, 20000, grads, n_params, 16, ws)
        ref = tracer.trace(ctx, med, rb, 0.02, 20000, "fp64")
        for k in out1:
            assert torch.equal(out1[k], out2[k]), k
            assert torch.equal(out2[k], ref[k]), k
        g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
        np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-14 * np.abs(g1).max())
        med.close()


@pytest.mark.parametrize("degree", [2, 6])
def test_checkpoint_interval_does_not_change_the_gradient_degrees(ctx, degree):
    """The polynomial classes other than the freeform block's degree 4: the
    gradient with a checkpoint every 64 steps (segments recomputed), every 7
    and every step (stored, nothing recomputed) agree to rounding."""
    base = W.freeform_block_medium()
    c = W.normal(W.BASE_SEED + 9, degree, W.n_monomials(degree), 0.01)
    c *= min(1.0, 0.1 / float(np.abs(c).sum()))
    c[0] += 1.55
    m = W.Medium(**{**base.__dict__, "degree": degree, "coeffs": c})
    rays = W.point_source_rays(512, W.BASE_SEED + 4)
    targets = W.design_targets(rays.n)
    _, g64 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 64)
    _, g7 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 7)
    _, g1 = adjoint_grad(ctx, m, m.coeffs, rays, targets, 0.02, 20000, 1)
    assert np.abs(g64).max() > 0
    np.testing.assert_allclose(g7, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())


# ------------------------------------- curved boundaries, sqrt and c/p forms


def _heading_to_plane(m, rays, dopl, max_steps, n):
    """The first n rays of `rays` that leave the medium with d_z > 0.3 in the
    oracle's trace (so that the image plane z = 30 is well in front of every
    exit line)."""
    t = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    sel = np.flatnonzero((t["exit_id"] >= 0) & (t["d"][:, 2] > 0.3))[:n]
    assert sel.size == n, sel.size
    return W.Rays(rays.origins[sel], rays.dirs[sel])


def _curved_case(name):
    """(medium, rays, dL0, max steps) of the media whose adjoint crosses a
    curved surface or differentiates n = sqrt(p) or n = C / p:
    - luneburg: n = sqrt(2 - r^2) in the unit sphere, a collimated beam
      entering and leaving through the sphere;
    - fisheye: Maxwell's fish-eye n = 2 / (1 + r^2) (the c/p form) in a
      sphere of radius 3, rays from an interior point refracting out;
    - corrector: the Sec. V freeform corrector (n = p, 7 nonzero expansion
      terms over 35 monomials) in its cylinder, entering through an end face,
      with total internal reflections on the side wall;
    - fiber: the parabolic fibre n^2 = nc^2 (1 - 2 delta rho^2 / R^2) in a
      cylinder inside its cladding, many rays refracting out of the side;
    - spherical: the spherical freeform of Sec. V (a0 .. a3, G2 = r cos 5
      theta) in its unit sphere, rays from outside aimed inside it."""
    if name == "luneburg":
        m = W.luneburg_medium()
        return m, _heading_to_plane(m, W.luneburg_rays(24), 2e-3, 5000, 256), 2e-3, 5000
    if name == "fisheye":
        m = W.fisheye_medium(n0=2.0, a=1.0, r_bound=3.0)
        # rays on the fish-eye's small circles never reach the surface
        th = W.uniform(7, 1, 4096, 0.0, math.pi)
        ph = W.uniform(7, 2, 4096, 0.0, 2 * math.pi)
        rays = W.Rays(np.tile([0.5, 0.0, 0.0], (4096, 1)), W.direction(th, ph))
        return m, _heading_to_plane(m, rays, 2e-3, 5000, 256), 2e-3, 5000
    if name == "corrector":
        wl = W.corrector_workload(1024)
        return wl.medium, _heading_to_plane(wl.medium, wl.rays, 5e-3, 20000, 256), 5e-3, 20000
    if name == "spherical":
        wl = W.spherical_workload(4096)
        return wl.medium, _heading_to_plane(wl.medium, wl.rays, 1e-3, 20000, 256), 1e-3, 20000
    m = W.fiber_medium(length=8.0)
    x = W.uniform(8, 1, 2048, -4.0, 4.0)
    y = W.uniform(8, 2, 2048, -3.0, 3.0)
    d = W.direction(W.uniform(8, 3, 2048, 0.0, math.radians(40)), W.uniform(8, 4, 2048, 0, 2 * math.pi))
    rays = W.Rays(np.stack([x, y, np.full(2048, -1.0)], 1), d)
    return m, _heading_to_plane(m, rays, 2e-3, 40000, 256), 2e-3, 40000


CURVED = ("luneburg", "fisheye", "corrector", "fiber", "spherical")
# Kept fraction of ray-coordinate pairs, measured 0.996, 0.996, 0.66, 0.80
# and 0.73: in the corrector, the fibre and the spherical freeform most rays
# turn in the field (N.I through zero inside a step, a kink of the discrete
# map within the FD step).
KEPT_FLOOR_CURVED = {"luneburg": 0.95, "fisheye": 0.95, "corrector": 0.5, "fiber": 0.7, "spherical": 0.6}


@pytest.mark.parametrize("name", CURVED)
def test_curved_and_nonlinear_media_against_oracle_fd(ctx, name):
    """Every coefficient of the four media above: the adjoint against central
    differences of the oracle's loss over the rays smooth for that
    coefficient (the rule of the tests above), within 1e-4 of
    sum_r |FD_r| and of the full loss's difference.  The step is 1e-6 and
    2.5e-7 of the coefficient scale."""
    m, rays, dopl, max_steps = _curved_case(name)
    targets = W.design_targets(rays.n)
    t = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    print(name, "exit ids", np.unique(t["exit_id"], return_counts=True),
          "boundary TIRs", int(t["tir_boundary"].sum()), "internal TIRs", int(t["tir_internal"].sum()))
    scale = max(1.0, float(np.abs(m.coeffs).max()))

    def factory(i):
        def at(h):
            c = m.coeffs.copy()
            c[i] += h * scale
            mm = W.Medium(**{**m.__dict__, "coeffs": c})
            return oracle.trace(mm, rays.origins, rays.dirs, dopl, max_steps), c[i]
        return at

    worst, full, kept = check_coordinates(ctx, m, m.coeffs, rays, targets, dopl, max_steps,
                                          range(len(m.coeffs)), factory, (1e-6, 2.5e-7))
    assert kept > KEPT_FLOOR_CURVED[name], kept
    assert worst <= REL, (worst, kept)
    assert full <= REL, (full, kept)


@pytest.mark.parametrize("name", CURVED)
def test_curved_and_nonlinear_media_against_oracle_tangents(ctx, name):
    """Every coefficient of the same four media against the FP64 reference
    gradient from the oracle's forward-mode tangents (crossing fraction and
    normal of a curved face, n = sqrt(p) and C / p by the chain rule): both
    differentiate the same discrete map with the same decisions, so within
    1e-10 of sum_r |per-ray term|, on every ray the tangents follow."""
    m, rays, dopl, max_steps = _curved_case(name)
    targets = W.design_targets(rays.n)
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    keep = t["flag"] == 0
    ref, mag = tangent_gradient(t, targets, keep)
    _, g = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 64, keep)
    err = np.abs(g - ref) / np.maximum(mag, 1e-300)
    print(name, "worst coefficient", int(err.argmax()), "error", float(err.max()), "kept", float(keep.mean()))
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, (float(err.max()), int(err.argmax()))


@pytest.mark.parametrize("name", CURVED)
def test_curved_media_checkpoint_interval_and_split(ctx, name):
    """On the same media: the forward sweep's exit states equal grin_trace
    FP64 bitwise, and the gradient with a checkpoint every 64 steps, every 7
    and every step agree to rounding."""
    m, rays, dopl, max_steps = _curved_case(name)
    targets = W.design_targets(rays.n)
    med = tracer.Medium(ctx, m)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    out, _ = tracer.trace_adjoint_forward(ctx, med, rb, dopl, max_steps, 16)
    ref = tracer.trace(ctx, med, rb, dopl, max_steps, "fp64")
    for k in out:
        assert torch.equal(out[k], ref[k]), k
    med.close()
    _, g64 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 64)
    _, g7 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 7)
    _, g1 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 1)
    assert np.abs(g64).max() > 0
    np.testing.assert_allclose(g7, g64, rtol=1e-12, atol=1e-13 * np.abs(g64).max())
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-13 * np.abs(g64).max())


def test_checkpoint_interval_choice(ctx):
    """grin_trace_adjoint_interval: 1 when every step's workspace fits the
    budget, else the smallest K whose workspace fits, GRIN_ERR_OOM below
    K = 64's; and the autograd function at the chosen interval (k = 0) gives
    the gradient of K = 64."""
    m = W.freeform_block_medium()
    med = tracer.Medium(ctx, m)
    n, dopl, ms = 4096, 0.02, 20000
    ws = {k: tracer.adjoint_workspace_bytes(med, n, dopl, ms, k) for k in range(1, 65)}
    assert all(ws[k] >= ws[k + 1] for k in range(1, 64))
    assert tracer.adjoint_interval(med, n, dopl, ms, ws[1]) == 1
    assert tracer.adjoint_interval(med, n, dopl, ms, ws[1] - 1) == 2
    assert tracer.adjoint_interval(med, n, dopl, ms, ws[9]) == next(k for k in range(2, 65) if ws[k] <= ws[9])
    assert tracer.adjoint_interval(med, n, dopl, ms, ws[64]) == min(k for k in range(2, 65) if ws[k] <= ws[64])
    with pytest.raises(N.GrinError) as e:
        tracer.adjoint_interval(med, n, dopl, ms, ws[64] - 1)
    assert e.value.status == N.GRIN_ERR_OOM
    med.close()
    rays = W.point_source_rays(512, W.BASE_SEED + 4)
    targets = W.design_targets(rays.n)
    _, g64 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, ms, 64)
    _, g0 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, ms, 0)
    np.testing.assert_allclose(g0, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())


# ------------------------------------------------------------ the N2P lens


def test_n2p_lens_parameters_against_oracle_tangents(ctx):
    """The N2P lens of Sec. VI with respect to (R, F, beta, gamma) on the
    design fan (64 rays parallel to the axis, whose first step is the
    tangential-incidence arc of Sec. II (iv)): the adjoint's gradient of the
    image-plane loss against the oracle's tangents within 1e-9 of
    sum_r |per-ray term|; the forward sweep's results bitwise those of
    grin_trace FP64; K = 1, 7 and 64 the same gradient to rounding.  The
    bound is ten times the box media's: these rays stay nearly parallel to
    the axis, where Eq. 9's D is formed by cancellation, and the reference
    itself moves by up to 6e-11 of sum_r |per-ray term| when the ray heights
    change by 4e-15 relative (measured 2.6e-10 for beta, 2e-11 or less for
    the others)."""
    from paper_2606_22655_b300 import n2p_design
    m = W.n2p_lens_medium(0.770, 4.462, 0.3)
    rays = n2p_design.fan(64, 0.3)
    dopl, max_steps = 1e-3, 400000
    targets = np.zeros((rays.n, 2))  # every ray aimed at the axis
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    keep = t["flag"] == 0
    assert keep.all()
    ref, mag = tangent_gradient(t, targets, keep)
    _, g64 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 64)
    err = np.abs(g64 - ref) / np.maximum(mag, 1e-300)
    print("n2p gradient", g64, "reference", ref, "error", err)
    assert err.max() <= 1e-9, err
    _, g7 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 7)
    _, g1 = adjoint_grad(ctx, m, m.coeffs, rays, targets, dopl, max_steps, 1)
    np.testing.assert_allclose(g7, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())
    med = tracer.Medium(ctx, m)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=torch.float64)
    out, _ = tracer.trace_adjoint_forward(ctx, med, rb, dopl, max_steps, 16)
    ref_out = tracer.trace(ctx, med, rb, dopl, max_steps, "fp64")
    for k in out:
        assert torch.equal(out[k], ref_out[k]), k
    med.close()


# ---------------------------------------------------------- layered shells


def test_layered_shells_against_oracle_tangents(ctx):
    """Point-sampled shells (Sec. I): the Luneburg field in 8 shells (all
    10 coefficients) and the 64^3 blob grid in 16 shells (64 samples with a
    gradient above 1e-2 of the largest).  A shell's index is a constant, so
    the parameters act only through the refraction normal grad f / |grad f|
    at shell changes.  The adjoint against the oracle's tangents within 1e-10
    of sum_r |per-ray term|; K = 1 and 64 the same gradient; the forward
    sweep's results bitwise grin_trace FP64's."""
    import dataclasses
    lune = dataclasses.replace(W.luneburg_medium(), n_levels=8, level_lo=1.0, level_hi=math.sqrt(2.0))
    rays = _heading_to_plane(lune, W.luneburg_rays(24), 2e-3, 5000, 256)
    targets = W.design_targets(rays.n)
    t = oracle.trace_tangent(lune, rays.origins, rays.dirs, 2e-3, 5000)
    keep = t["flag"] == 0
    ref, mag = tangent_gradient(t, targets, keep)
    _, g64 = adjoint_grad(ctx, lune, lune.coeffs, rays, targets, 2e-3, 5000, 64, keep)
    _, g1 = adjoint_grad(ctx, lune, lune.coeffs, rays, targets, 2e-3, 5000, 1, keep)
    # the constant coefficient shifts f uniformly: no normal moves, so its
    # gradient is zero up to rounding on both sides; the others to 1e-10
    err = np.abs(g64[1:] - ref[1:]) / np.maximum(mag[1:], 1e-300)
    print("layered luneburg error", err, "kept", keep.mean(), "constant term", g64[0], ref[0])
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, err
    assert abs(g64[0]) <= 1e-12 * np.abs(g64).max() and abs(ref[0]) <= 1e-12 * np.abs(ref).max()
    np.testing.assert_allclose(g1, g64, rtol=1e-12, atol=1e-15 * np.abs(g64).max())

    wl = W.blob_workload(n_rays=384, res=64, n_levels=16)
    m = wl.medium
    targets = W.design_targets(wl.rays.n) + 10.0
    theta0 = m.grid.astype(np.float64).ravel()
    _, g_all = adjoint_grad(ctx, m, theta0, wl.rays, targets, 0.02, 20000, 64)
    cand = np.flatnonzero(np.abs(g_all) > 1e-2 * np.abs(g_all).max())
    coords = np.random.default_rng(3).choice(cand, size=min(64, cand.size), replace=False)
    t = oracle.trace_tangent(m, wl.rays.origins, wl.rays.dirs, 0.02, 20000, samples=coords)
    keep = t["flag"] == 0
    ref, mag = tangent_gradient(t, targets, keep)
    _, g = adjoint_grad(ctx, m, theta0, wl.rays, targets, 0.02, 20000, 64, keep)
    err = np.abs(g[coords] - ref) / np.maximum(mag, 1e-300)
    print("layered grid error", err.max(), "kept", keep.mean())
    assert keep.mean() > 0.95
    assert err.max() <= 1e-10, err

    for spec, rr, dopl, ms in ((lune, rays, 2e-3, 5000), (m, wl.rays, 0.02, 20000)):
        med = tracer.Medium(ctx, spec)
        rb = tracer.RayBatch.from_numpy(rr.origins, rr.dirs, device="cuda", dtype=torch.float64)
        out, _ = tracer.trace_adjoint_forward(ctx, med, rb, dopl, ms, 16)
        ref_out = tracer.trace(ctx, med, rb, dopl, ms, "fp64")
        for k in out:
            assert torch.equal(out[k], ref_out[k]), k
        med.close()
