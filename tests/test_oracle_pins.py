"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, exact rational arithmetic, a value printed in the paper, an invariant
or a convergence order.  No GPU is used.
"""
import dataclasses
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2606_22655_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _one(medium, o, d, dopl, max_steps):
    r = oracle.trace(medium, np.asarray(o, float)[None], np.asarray(d, float)[None], dopl, max_steps, threads=1)
    return {k: v[0] for k, v in r.items()}


# ------------------------------------------------------- homogeneous media


def test_homogeneous_normal_incidence_steps_and_opl():
    """Case (iii): straight steps of dL0/n; exact step count ceil(n L / dL0),
    OPL = n_ext * 1 + n L, and normal incidence leaves R = I (Eq. 8-9)."""
    n, L, dopl = 1.5, 0.8227, 0.01
    m = W.homogeneous_box(n, lo=(-1, -1, 0), hi=(1, 1, L))
    r = _one(m, (0, 0, -1), (0, 0, 1), dopl, 10000)
    assert r["exit_id"] == 5
    assert r["steps"] == math.ceil(n * L / dopl) == 124
    assert r["opl"] == pytest.approx(1.0 + n * L, rel=1e-14)
    np.testing.assert_allclose(r["P"], [0, 0, L], atol=1e-15)
    np.testing.assert_array_equal(r["d"], [0, 0, 1])


@pytest.mark.parametrize("theta_deg", [5.0, 30.0, 60.0])
def test_homogeneous_slab_oblique(theta_deg):
    """Snell at both faces of a parallel slab: lateral shift L tan(theta_in),
    exit direction equal to the input direction, OPL = outside + n L / cos."""
    n, L, dopl = 1.5, 1.0, 1e-3
    m = W.homogeneous_box(n, lo=(-10, -10, 0), hi=(10, 10, L))
    th = math.radians(theta_deg)
    d0 = np.array([math.sin(th), 0.0, math.cos(th)])
    o = np.array([0.0, 0.0, -1.0])
    r = _one(m, o, d0, dopl, 100000)
    th_in = math.asin(math.sin(th) / n)
    x_entry = math.tan(th)
    assert r["exit_id"] == 5
    np.testing.assert_allclose(r["P"], [x_entry + L * math.tan(th_in), 0, L], atol=1e-12)
    np.testing.assert_allclose(r["d"], d0, atol=1e-14)
    assert r["opl"] == pytest.approx(1.0 / math.cos(th) + n * L / math.cos(th_in), rel=1e-13)


def test_entry_refraction_vector_snell():
    """Eq. 1: n_ext N x I = n N x R at the entry face (max_steps = 0 stops
    right after the boundary refraction)."""
    n = 1.7
    m = W.homogeneous_box(n, lo=(-10, -10, 0), hi=(10, 10, 5))
    d0 = np.array([0.3, -0.5, 0.8])
    d0 /= np.linalg.norm(d0)
    r = _one(m, (0, 0, -1), d0, 1e-3, 0)
    assert r["exit_id"] == oracle.EXIT_MAXSTEPS and r["steps"] == 0
    N = np.array([0, 0, -1.0])
    np.testing.assert_allclose(1.0 * np.cross(N, d0), n * np.cross(N, r["d"]), atol=1e-15)
    assert np.dot(r["d"], [0, 0, 1]) > 0  # positive root of Eq. 9: transmitted, not reflected


@pytest.mark.parametrize("sign", [+1, -1])
def test_critical_angle_split(sign):
    """Sec. II (v): at the +x wall of a homogeneous box (n = 1.5, air
    outside) a ray 1e-6 rad beyond the critical angle is reflected, one 1e-6
    rad short of it leaves with n sin(a) = sin(a_out)."""
    n = 1.5
    m = W.homogeneous_box(n, lo=(-1, -1, -50), hi=(1, 1, 50))
    ac = math.asin(1.0 / n)
    a = ac + sign * 1e-6  # incidence angle on the x wall
    d0 = np.array([math.cos(a), 0.0, math.sin(a)])
    r = _one(m, (0, 0, 0), d0, 1e-3, 200000)
    if sign > 0:
        assert r["tir_boundary"] >= 1 and r["exit_id"] != 1
    else:
        assert r["exit_id"] == 1 and r["tir_boundary"] == 0
        assert r["d"][2] == pytest.approx(n * math.sin(a), rel=1e-12)


def test_boundary_reflection_law():
    """Sec. II (v) reflection I - 2 (I.N) N at the +x wall, then Snell out of
    the +z face: the exit direction has d_x = -n cos(a); checked in closed
    form together with the exit point."""
    n = 1.5
    m = W.homogeneous_box(n, lo=(-1, -1, 0), hi=(1, 1, 3))
    a = math.radians(70.0)  # incidence angle on the x wall, beyond critical (41.8 deg)
    d0 = np.array([math.cos(a), 0.0, math.sin(a)])
    r = _one(m, (0, 0, 0.1), d0, 1e-4, 200000)
    assert r["tir_boundary"] == 1 and r["exit_id"] == 5
    # after reflection the ray heads (-cos a, 0, sin a); at the z face the
    # tangential component is scaled by n
    dx = -n * math.cos(a)
    np.testing.assert_allclose(r["d"], [dx, 0, math.sqrt(1 - dx * dx)], atol=1e-12)
    # geometry: wall at x=1 reached after dz = tan(a); top at z = 3
    z_wall = 0.1 + math.tan(a)
    x_exit = 1.0 - (3.0 - z_wall) / math.tan(a)
    np.testing.assert_allclose(r["P"], [x_exit, 0, 3.0], atol=1e-12)


def test_miss_entry_reflect_invalid_and_zero_steps():
    m = W.luneburg_medium()
    r = _one(m, (2, 0, -1.5), (0, 0, 1), 1e-3, 10)
    assert r["exit_id"] == oracle.EXIT_MISS and r["steps"] == 0 and r["opl"] == 0
    dense = W.homogeneous_box(1.0, lo=(-1, -1, 0), hi=(1, 1, 1), n_ext=1.5)
    a = math.radians(70.0)
    r = _one(dense, (0, 0, -0.1), (math.sin(a), 0, math.cos(a)), 1e-3, 10)
    assert r["exit_id"] == oracle.EXIT_ENTRY_REFLECT
    assert r["d"][2] == pytest.approx(-math.cos(a), abs=1e-15)
    r = _one(m, (0, 0, -1.5), (float("nan"), 0, 1), 1e-3, 10)
    assert r["exit_id"] == oracle.EXIT_INVALID
    r = _one(m, (0, 0, 0.2), (0, 1, 0), 1e-3, 0)
    assert r["exit_id"] == oracle.EXIT_MAXSTEPS and r["steps"] == 0
    np.testing.assert_array_equal(r["P"], [0, 0, 0.2])


# ----------------------------------------------------- smooth GRIN media


def _luneburg_errors(dopl, idx):
    wl = W.luneburg_workload()
    rays = wl.rays.subset(idx)
    r = oracle.trace(wl.medium, rays.origins, rays.dirs, dopl, 200000)
    o = rays.origins
    pe = np.stack([o[:, 0], o[:, 1], -np.sqrt(1 - o[:, 0] ** 2 - o[:, 1] ** 2)], 1)
    ep = np.linalg.norm(r["P"] - [0, 0, 1], axis=1)
    ed = np.linalg.norm(r["d"] + pe, axis=1)
    eo = np.abs(r["opl"] - (1.5 + math.pi / 2))
    return r, ep, ed, eo


def test_luneburg_focus_closed_form():
    """Ray equation with n^2 = 2 - r^2: r(t) = P_e cos t + z sin t, so every
    ray leaves at (0, 0, 1) along -P_e with total OPL 1.5 + pi/2 from
    z = -1.5.  VRT is first order (Sec. III), so errors are O(dL0)."""
    r, ep, ed, eo = _luneburg_errors(1e-3, slice(0, 4096, 5))
    assert (r["exit_id"] == 0).all()
    assert ep.max() < 3e-3 and ed.max() < 3e-3 and eo.max() < 3e-3


def test_luneburg_first_order_convergence():
    """Halving dL0 roughly halves the mean exit error (first order, Sec. III)."""
    idx = slice(0, 4096, 97)
    e = [np.mean(_luneburg_errors(h, idx)[1]) for h in (1e-3, 5e-4, 2.5e-4)]
    for a, b in zip(e, e[1:]):
        assert 1.5 < a / b < 3.0


def test_bouguer_invariant_spherical_symmetry():
    """With N = grad n / |grad n| radial, Eq. 1 gives n_{i-1} (P_i x I_i) =
    n_i (P_i x R_i), and P_{i+1} x R_i = P_i x R_i: the discrete scheme keeps
    n(P_i) |P_i x R_i| (the Bouguer invariant of spherically symmetric media)
    exactly, up to rounding, on every segment of a refracting ray."""
    m = W.luneburg_medium()
    for h in (2e-3, 1e-3):
        res, path = oracle.trace_path(m, (0.3, 0.4, -1.5), (0, 0, 1), h, 100000)
        assert res["tir_internal"][0] == 0
        seg = np.diff(path, axis=0)
        dirs = seg / np.linalg.norm(seg, axis=1, keepdims=True)
        n, _ = oracle.medium_eval(m, path[:-1])
        inv = n * np.linalg.norm(np.cross(path[:-1], dirs), axis=1)
        assert inv[0] == pytest.approx(0.5, abs=1e-15)  # n = 1 at entry, impact parameter 0.5
        assert np.abs(inv - inv[0]).max() < 1e-12


def test_maxwell_fisheye_conjugate_point():
    """Maxwell fish-eye n = n0 / (1 + r^2): all rays from P0 pass through
    -P0 / |P0|^2."""
    m = W.fisheye_medium(n0=2.0, a=1.0, r_bound=20.0)
    p0 = np.array([0.5, 0.0, 0.0])
    target = -p0 / np.dot(p0, p0)
    for th in (0.7, 1.3, 2.1):
        d0 = np.array([math.cos(th), math.sin(th) * 0.6, math.sin(th) * 0.8])
        res, path = oracle.trace_path(m, p0, d0, 1e-4, 400000)
        dist = np.linalg.norm(path - target, axis=1).min()
        assert dist < 2e-3, (th, dist)


def test_fiber_helix_matches_paper_rmse():
    """Sec. IV: the parabolic-index fiber ray from P0 = (4, -2.6128, -3.0288)
    through (4, 0, 0) is a helix of radius 4; with dL0 = 1e-4 the paper prints
    a transverse RMSE (Eq. 23) of 5.0892e-5.  The analytic helix is
    x = 4 cos(a t), y = 4 sin(a t), z = b t with a = n_c sqrt(2 Delta) / R and
    b = sqrt(n(4)^2 - k^2), k the transverse optical momentum of the launched
    ray; the interior length follows from the printed point count."""
    g = json.load(open(os.path.join(GOLD, "helix_e1.json")))
    R, nc, D = g["R"], g["nc"], g["Delta"]
    m = W.fiber_medium(nc=nc, delta=D, radius=R, length=52.1)
    p0, pi = np.array(g["P0"]), np.array(g["PI"])
    d0 = (pi - p0) / np.linalg.norm(pi - p0)
    assert math.degrees(math.acos(d0[2])) == pytest.approx(g["angle_to_z_deg"], abs=5e-3)
    alpha = nc * math.sqrt(2 * D) / R
    n4 = nc * math.sqrt(1 - 2 * D * 16 / R ** 2)
    # transverse optical momentum is conserved through the z = 0 face and the
    # axial one, b, inside (n has no z dependence)
    kt = m.n_ext * math.sqrt(1 - d0[2] ** 2)
    assert kt == pytest.approx(4 * alpha, rel=1e-5)  # helical condition at rho = 4
    beta = math.sqrt(n4 ** 2 - kt ** 2)

    def rmse(h):
        res, path = oracle.trace_path(m, p0, d0, h, 3_000_000)
        t = path[:, 2] / beta
        e2 = (path[:, 0] - 4 * np.cos(alpha * t)) ** 2 + (path[:, 1] - 4 * np.sin(alpha * t)) ** 2
        return math.sqrt(e2.mean()), path

    e1, path = rmse(g["dL0"])
    rho = np.hypot(path[:, 0], path[:, 1])
    assert np.abs(rho - 4.0).max() < 1e-4
    assert 0.8 * g["rmse"] < e1 < 1.25 * g["rmse"]
    e2, _ = rmse(2 * g["dL0"])
    assert 1.6 < e2 / e1 < 2.4


# ------------------------------------------------------------- evaluators


def _exact_poly(coeffs, degree, off, scale, P):
    """Exact rational value and gradient of the normalised polynomial."""
    x = [(Fraction(P[a]) - Fraction(off[a])) / Fraction(scale[a]) for a in range(3)]
    v = Fraction(0)
    g = [Fraction(0)] * 3
    for c, (i, j, k) in zip(coeffs, W.monomial_exponents(degree)):
        c = Fraction(c)
        v += c * x[0] ** i * x[1] ** j * x[2] ** k
        if i:
            g[0] += c * i * x[0] ** (i - 1) * x[1] ** j * x[2] ** k
        if j:
            g[1] += c * j * x[0] ** i * x[1] ** (j - 1) * x[2] ** k
        if k:
            g[2] += c * k * x[0] ** i * x[1] ** j * x[2] ** (k - 1)
    return float(v), [float(g[a] / Fraction(scale[a])) for a in range(3)]


def test_polynomial_evaluator_exact():
    m = W.freeform_block_medium()
    pts = np.stack([W.uniform(5, 1, 20, -5, 5), W.uniform(5, 2, 20, -5, 5), W.uniform(5, 3, 20, 0, 20)], 1)
    n, g = oracle.medium_eval(m, pts)
    for i in range(len(pts)):
        v, ge = _exact_poly(m.coeffs, 4, m.off, m.scale, pts[i])
        assert n[i] == pytest.approx(v, rel=1e-14, abs=1e-15)
        np.testing.assert_allclose(g[i], ge, rtol=1e-12, atol=1e-15)


def test_sqrt_and_recip_forms_central_differences():
    for m in (W.luneburg_medium(), W.fisheye_medium()):
        pts = np.array([[0.1, -0.2, 0.3], [0.5, 0.4, -0.2], [-0.3, 0.1, 0.6]])
        n, g = oracle.medium_eval(m, pts)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (oracle.medium_eval(m, pts + e)[0] - oracle.medium_eval(m, pts - e)[0]) / (2 * h)
            np.testing.assert_allclose(g[:, a], fd, rtol=1e-7, atol=1e-9)
    m = W.luneburg_medium()
    n, _ = oracle.medium_eval(m, pts)
    np.testing.assert_allclose(n, np.sqrt(2 - (pts ** 2).sum(1)), rtol=1e-15)


def _quadratic_grid(res=12, h=0.5):
    q = lambda x, y, z: 1.5 + 0.01 * x - 0.02 * y + 0.015 * z + 0.003 * x * x - 0.002 * x * y + 0.001 * y * z + 0.0025 * z * z
    x = np.arange(res) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    grid = q(X, Y, Z).astype(np.float32)
    return grid, q


def test_tricubic_reproduces_quadratics_and_nodes():
    """Catmull-Rom reproduces polynomials of degree <= 2 exactly away from the
    clamped edges; at nodes it returns the samples."""
    grid, q = _quadratic_grid()
    h = 0.5
    m = W.grid_medium(grid, h, size=h * 11)
    # reference: the field the float32 samples actually hold is the quadratic
    # rounded per sample, so compare with a grid built from exactly
    # representable values: use the float32 samples at nodes
    nodes = np.array([[2 * h, 3 * h, 4 * h], [5 * h, 5 * h, 7 * h]])
    n, _ = oracle.medium_eval(m, nodes)
    np.testing.assert_array_equal(n, [grid[4, 3, 2], grid[7, 5, 5]])
    pts = np.stack([W.uniform(9, a, 25, 1.5 * h, 9.5 * h) for a in range(3)], 1)
    n, g = oracle.medium_eval(m, pts)
    x, y, z = pts.T
    np.testing.assert_allclose(n, q(x, y, z), atol=5e-7)  # float32 sample rounding
    gx = 0.01 + 0.006 * x - 0.002 * y
    gy = -0.02 - 0.002 * x + 0.001 * z
    gz = 0.015 + 0.001 * y + 0.005 * z
    np.testing.assert_allclose(g, np.stack([gx, gy, gz], 1), atol=2e-6)


def test_tricubic_exact_on_representable_linear_field():
    """With samples that are exact in float32 the linear field is reproduced
    to rounding."""
    res, h = 10, 0.25
    i = np.arange(res)
    K, J, I = np.meshgrid(i, i, i, indexing="ij")
    grid = (1.5 + (I + 2 * J - K) / 1024.0).astype(np.float32)
    m = W.grid_medium(grid, h, size=h * (res - 1))
    pts = np.stack([W.uniform(3, a, 30, 1.1 * h, (res - 2.1) * h) for a in range(3)], 1)
    n, g = oracle.medium_eval(m, pts)
    u = pts / h
    np.testing.assert_allclose(n, 1.5 + (u[:, 0] + 2 * u[:, 1] - u[:, 2]) / 1024.0, atol=1e-14)
    np.testing.assert_allclose(g, np.tile([1 / 1024 / h, 2 / 1024 / h, -1 / 1024 / h], (30, 1)), atol=1e-13)


def test_constant_grid_gives_straight_rays():
    grid = np.full((8, 8, 8), 1.25, dtype=np.float32)
    m = W.grid_medium(grid, 1.0, size=7.0)
    d0 = np.array([0.2, 0.1, 1.0])
    d0 /= np.linalg.norm(d0)
    r = _one(m, (2, 3, -1), d0, 1e-2, 100000)
    assert r["exit_id"] == 5
    np.testing.assert_allclose(r["d"], d0, atol=1e-14)


# ---------------------------------------------------------- layered shells


@pytest.mark.parametrize("levels", [2, 32])
def test_layered_planar_shells_conserve_tangential_momentum(levels):
    """Isoindicial shells that are planes z = const: every crossing obeys
    Snell with N = z, so n sin(theta) is conserved and a ray leaves the
    parallel stack along its input direction."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.2})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                 scale=(1, 1, 1), n_levels=levels, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                 bparams=(-50, -50, 0, 50, 50, 2, 0, 0), n_ext=1.0)
    th = math.radians(35.0)
    d0 = np.array([math.sin(th) * 0.6, math.sin(th) * 0.8, math.cos(th)])
    r = _one(m, (0, 0, -1), d0, 1e-3, 100000)
    assert r["exit_id"] == 5 and r["tir_internal"] == 0
    np.testing.assert_allclose(r["d"], d0, atol=1e-13)


def test_tangent_incidence_first_arc():
    """Case (iv): with n = 1.5 + 0.1 x and the ray along +y, the first point
    after the start has N.I = 0 exactly; the next point is
    P_i + h (sqrt(1 - k^2) I + k N) with k = (n(P_i + h N) - n(P_i)) / (2 n_i)."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (1, 0, 0): 0.1})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, bkind=W.BOUNDARY_BOX,
                 bparams=(-1, -1, -1, 1, 1, 1, 0, 0), n_ext=1.0)
    dopl = 1e-2
    r = _one(m, (0, 0, 0), (0, 1, 0), dopl, 2)
    h = dopl / 1.5
    k = (0.1 * h) / (2 * 1.5)
    expect = np.array([0.0, h, 0.0]) + h * np.array([k, math.sqrt(1 - k * k), 0.0])
    np.testing.assert_allclose(r["P"], expect, atol=1e-16)
    assert r["margins"][oracle.M_TAN] == 0.0


def test_layered_level_value_sets_optical_length():
    """A field of constant 1.52 quantised into 4 shells on [1.3, 1.7] sits in
    level 2, whose index is the level centre 1.3 + 2.5 * 0.1 = 1.55: the slab
    then takes ceil(1.55 L / dL0) straight steps and OPL = 1 + 1.55 L."""
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=0, coeffs=np.array([1.52]),
                 n_levels=4, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                 bparams=(-1, -1, 0, 1, 1, 0.8227, 0, 0), n_ext=1.0)
    r = _one(m, (0, 0, -1), (0, 0, 1), 0.01, 10000)
    assert r["exit_id"] == 5
    assert r["steps"] == math.ceil(1.55 * 0.8227 / 0.01)
    assert r["opl"] == pytest.approx(1.0 + 1.55 * 0.8227, rel=1e-13)


def test_internal_tir_step_length_uses_previous_index():
    """Sec. II (v): a ray in the n = 1.6 shell meets the n = 1.4 shell at 80
    deg (critical angle 61 deg); it is reflected at the first point past the
    plane z = 1 and the reflected step has length dL0 / n_{i-1} = dL0 / 1.6."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.2})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                 n_levels=2, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                 bparams=(-50, -50, 0, 50, 50, 2, 0, 0), n_ext=1.0)
    a = math.radians(80.0)
    d0 = np.array([math.sin(a), 0.0, -math.cos(a)])
    dopl = 1e-3
    h = dopl / 1.6
    k_star = math.floor(0.05 / (h * math.cos(a))) + 1  # first point below z = 1 (461)
    assert 0.2 < 0.05 / (h * math.cos(a)) % 1 < 0.8  # far from an integer: no rounding ambiguity
    r = _one(m, (0, 0, 1.05), d0, dopl, k_star + 1)
    assert r["tir_internal"] == 1
    p_k = np.array([0, 0, 1.05]) + k_star * h * d0
    expect = p_k + h * np.array([math.sin(a), 0.0, math.cos(a)])
    np.testing.assert_allclose(r["P"], expect, atol=1e-12)


def _fringe_trig(m, rho, t):
    """Fringe Zernike Z_m from its definition in polar form."""
    return {1: np.ones_like(rho), 2: rho * np.cos(t), 3: rho * np.sin(t), 4: 2 * rho**2 - 1,
            5: rho**2 * np.cos(2 * t), 6: rho**2 * np.sin(2 * t),
            7: (3 * rho**3 - 2 * rho) * np.cos(t), 8: (3 * rho**3 - 2 * rho) * np.sin(t),
            9: 6 * rho**4 - 6 * rho**2 + 1, 10: rho**3 * np.cos(3 * t), 11: rho**3 * np.sin(3 * t),
            12: (4 * rho**4 - 3 * rho**2) * np.cos(2 * t),
            13: (4 * rho**4 - 3 * rho**2) * np.sin(2 * t)}[m]


def _corrector_trig(p, coeffs, n_lo, n_hi, rho_max=4.2, z_max=2.5):
    x, y, z = p[:, 0] / rho_max, p[:, 1] / rho_max, 2 * p[:, 2] / z_max - 1
    rho, t = np.hypot(x, y), np.arctan2(y, x)
    legendre = {0: np.ones_like(z), 1: z, 2: 1.5 * z**2 - 0.5}
    s = sum(c * _fringe_trig(m, rho, t) * legendre[v] for (m, v), c in coeffs.items())
    return 0.5 * (n_hi + n_lo) + 0.5 * (n_hi - n_lo) * s


def test_corrector_lens_zernike_legendre_expansion():
    """Sec. V corrector lens: the medium handed to the tracers (monomials of
    the normalised coordinates) against the Zernike x Legendre expansion
    evaluated in polar form (rho, theta = atan2), for the paper's coefficients
    and for every Fringe term Z1..Z13 times V0..V2; gradient against central
    differences of the polar form."""
    rng = np.random.default_rng(11)
    k = 40
    r = 4.2 * np.sqrt(rng.uniform(0, 1, k))
    a = rng.uniform(0, 2 * np.pi, k)
    p = np.stack([r * np.cos(a), r * np.sin(a), rng.uniform(0, 2.5, k)], 1)
    cases = [(W.CORRECTOR_COEFFS, 1.5148, 1.5162), (W.CORRECTOR_COEFFS, 1.5261, 1.5608)]
    cases += [({(m, v): 1.0}, 1.0, 3.0) for m in range(1, 14) for v in range(3)]
    for coeffs, lo, hi in cases:
        med = W.corrector_lens_medium(n_lo=lo, n_hi=hi, coeffs=coeffs)
        n, g = oracle.medium_eval(med, p)
        ref = _corrector_trig(p, coeffs, lo, hi)
        np.testing.assert_allclose(n, ref, rtol=0, atol=1e-14 * max(1.0, np.abs(ref).max()))
        h = 1e-5
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            fd = (_corrector_trig(p + e, coeffs, lo, hi) - _corrector_trig(p - e, coeffs, lo, hi)) / (2 * h)
            np.testing.assert_allclose(g[:, ax], fd, rtol=0, atol=1e-8 * max(1.0, np.abs(fd).max()))
    # the paper's expansion is a degree-4 polynomial
    assert W.corrector_lens_medium().degree == 4


def _spherical_trig(p, a, radius=1.0):
    """Sec. V spherical freeform index from its definition in spherical
    coordinates (theta from +z, phi the azimuth)."""
    x, y, z = (p / radius).T
    r = np.sqrt(x * x + y * y + z * z)
    th = np.arccos(np.clip(z / r, -1.0, 1.0))
    ph = np.arctan2(y, x)
    return (a[0] + a[1] * 0.3 * (r**2 - 1) + a[2] * r * np.cos(5 * th)
            + a[3] * r**2 * np.sin(th)**2 * np.cos(2 * ph))


@pytest.mark.parametrize("a", [(1.5, 1.0, -0.2, 0.3), (1.2, -0.7, 0.9, -0.4)])
def test_spherical_freeform_field_against_definition(a):
    """The oracle's angle-free form (Chebyshev T5, x^2 - y^2) against the
    definition with arccos/arctan2 and cosines; the gradient against central
    differences of the definition; R = 2 exercises the normalisation."""
    rng = np.random.default_rng(5)
    R = 2.0
    v = rng.normal(size=(60, 3))
    p = R * (0.05 + 0.9 * rng.uniform(size=(60, 1))) * v / np.linalg.norm(v, axis=1, keepdims=True)
    m = W.spherical_freeform_medium(a=a, radius=R)
    n, g = oracle.medium_eval(m, p)
    np.testing.assert_allclose(n, _spherical_trig(p, a, R), rtol=0, atol=2e-15)
    h = 1e-6
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (_spherical_trig(p + e, a, R) - _spherical_trig(p - e, a, R)) / (2 * h)
        np.testing.assert_allclose(g[:, ax], fd, rtol=0, atol=2e-8)


def test_spherical_freeform_reduces_to_polynomial():
    """With a2 = 0 the field is the quadratic a0 + 0.3 a1 (r^2 - 1) + a3 (x^2 - y^2):
    rays through both descriptions agree to rounding."""
    a0, a1, a3 = 1.5, 1.0, 0.3
    sph = W.spherical_freeform_medium(a=(a0, a1, 0.0, a3))
    c = W.coeffs_from_terms(2, {(0, 0, 0): a0 - 0.3 * a1, (2, 0, 0): 0.3 * a1 + a3,
                                (0, 2, 0): 0.3 * a1 - a3, (0, 0, 2): 0.3 * a1})
    poly = W.Medium(kind=W.KIND_POLY, degree=2, coeffs=c, bkind=sph.bkind, bparams=sph.bparams,
                    n_ext=1.0)
    wl = W.spherical_workload(64, a=(a0, a1, 0.0, a3))
    o1 = oracle.trace(sph, wl.rays.origins, wl.rays.dirs, wl.dopl, wl.max_steps)
    o2 = oracle.trace(poly, wl.rays.origins, wl.rays.dirs, wl.dopl, wl.max_steps)
    ok = (o1["margins"][:, 0] > 1e-9) & (o1["margins"][:, 2] > 1e-9)
    assert ok.mean() > 0.9
    for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
        np.testing.assert_array_equal(o1[k][ok], o2[k][ok])
    np.testing.assert_allclose(o1["P"][ok], o2["P"][ok], rtol=0, atol=1e-9)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_spherical_freeform_axis_ray_closed_form_opl(sign):
    """On the z axis G3 and its gradient vanish and grad n is axial, so a ray
    along the axis stays on it exactly; there n = a0 - 0.3 a1 + 0.3 a1 z^2 +
    a2 z, whose integral over [-1, 1] is 2 a0 - 0.4 a1.  The discrete optical
    path converges to 1 (the unit exterior segment) + that, at first order."""
    a = (1.5, 1.0, -0.2, 0.3)
    m = W.spherical_freeform_medium(a=a)
    exact = 1.0 + 2 * a[0] - 0.4 * a[1]
    errs = []
    for dopl in (1e-3, 5e-4):
        o = oracle.trace(m, np.array([[0.0, 0.0, -2.0 * sign]]), np.array([[0.0, 0.0, sign]]), dopl, 100000)
        assert o["exit_id"][0] == 0
        np.testing.assert_array_equal(o["P"][0, :2], [0.0, 0.0])
        np.testing.assert_array_equal(o["d"][0], [0.0, 0.0, sign])
        errs.append(abs(o["opl"][0] - exact))
    assert errs[0] < 5e-3
    assert 1.5 < errs[0] / errs[1] < 2.5


def _n2p_def(p, R, F, beta, gamma):
    """Sec. VI N2P index evaluated through logarithms (a different route from
    the oracle's pow): n = exp(gamma log(1 + exp(beta log u)))."""
    rho2 = p[:, 0] ** 2 + p[:, 1] ** 2
    u = (R * R - rho2 / 4.0) / (F * F)
    return np.exp(gamma * np.log1p(np.exp(beta * np.log(u))))


@pytest.mark.parametrize("beta,gamma", [(0.772, 4.469), (1.0932, 5.0069), (0.6791, 2.7007)])
def test_n2p_lens_field(beta, gamma):
    """N2P-GRIN lens (Sec. VI): the oracle's field against the definition by
    another route, its gradient against central differences, no dependence on
    z, and the closed-form values on the axis and at the rim."""
    R, F, L = 1.0, 2.0, 0.3
    m = W.n2p_lens_medium(beta, gamma, L, R, F)
    rng = np.random.default_rng(3)
    r = R * np.sqrt(rng.uniform(0, 1, 50))
    a = rng.uniform(0, 2 * np.pi, 50)
    p = np.stack([r * np.cos(a), r * np.sin(a), rng.uniform(-L, 0, 50)], 1)
    n, g = oracle.medium_eval(m, p)
    np.testing.assert_allclose(n, _n2p_def(p, R, F, beta, gamma), rtol=1e-14, atol=0)
    h = 1e-6
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (_n2p_def(p + e, R, F, beta, gamma) - _n2p_def(p - e, R, F, beta, gamma)) / (2 * h)
        np.testing.assert_allclose(g[:, ax], fd, rtol=0, atol=1e-7 * max(1.0, np.abs(fd).max()))
    assert (g[:, 2] == 0.0).all()
    n_axis, _ = oracle.medium_eval(m, [[0.0, 0.0, -0.1]])
    n_rim, _ = oracle.medium_eval(m, [[R, 0.0, -0.1]])
    assert n_axis[0] == pytest.approx((1 + (R * R / F**2) ** beta) ** gamma, rel=1e-15)
    assert n_rim[0] == pytest.approx((1 + (0.75 * R * R / F**2) ** beta) ** gamma, rel=1e-15)


def n2p_rmse_lsa(beta, gamma, L, R=1.0, F=2.0, n=10, dopl=1e-4):
    """RMSE of the longitudinal spherical aberration (Sec. VI): n rays parallel
    to the axis at heights 0.995 R k / n, k = 1..n, launched before the lens;
    each exit ray crosses the axis at z_Int, LSA = F - z_Int."""
    m = W.n2p_lens_medium(beta, gamma, L, R, F)
    y = 0.995 * R * np.arange(1, n + 1) / n
    o = np.stack([np.zeros(n), y, np.full(n, -L - 0.5 * R)], 1)
    r = oracle.trace(m, o, np.tile([0.0, 0.0, 1.0], (n, 1)), dopl * R, 400000)
    P, D = r["P"], r["d"]
    zint = P[:, 2] - P[:, 1] * D[:, 2] / D[:, 1]
    return float(np.sqrt(np.mean((F - zint) ** 2))), r


def test_n2p_lens_reaches_the_paper_design_quality():
    """At L = 0.3 R, F = 2 R the printed formula reaches the quasi-stigmatic
    focus that Sec. VI reports (RMSE_LSA about 2.4e-3 R across L): at the
    parameters a successive refinement finds, (beta, gamma) = (0.772, 4.469),
    RMSE_LSA <= 5e-3 R with every ray leaving through the exit face, while a
    point a few percent away in (beta, gamma) is more than ten times worse."""
    e, r = n2p_rmse_lsa(0.772, 4.469, 0.3)
    assert (r["exit_id"] == 2).all()
    assert e <= 5e-3
    e_off, _ = n2p_rmse_lsa(0.74, 4.3, 0.3)
    assert e_off > 10 * e


# ------------------------------------------------- forward-mode tangents


def _tangent_vs_fd(dopl, max_steps, coords, h=1e-6):
    """Per coefficient: the oracle's tangent of (P, d, OPL) against the
    central difference of oracle traces with the coefficient moved by +-h,
    on the rays whose integer outcomes do not change and whose differences at
    h and h / 2 agree to 1e-6 (there the differences' own error, truncation
    plus rounding noise / h, is below that).  Returns the relative errors."""
    m = W.freeform_block_medium()
    rays = W.point_source_rays(64, W.BASE_SEED + 4)
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    base = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    for k in ("P", "d", "opl", "exit_id", "steps"):
        np.testing.assert_array_equal(t[k], base[k], err_msg=k)  # same values, same decisions
    errs = []
    for i in coords:
        keep = (t["flag"] == 0) & (base["exit_id"] != oracle.EXIT_MISS)
        fds = []
        for hh in (h, h / 2):
            res = []
            for s in (+hh, -hh):
                mm = W.Medium(**{**m.__dict__})
                c = m.coeffs.copy()
                c[i] += s
                mm.coeffs = c
                res.append((oracle.trace(mm, rays.origins, rays.dirs, dopl, max_steps), c[i]))
            (rp, vp), (rm, vm) = res
            for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
                keep &= (rp[k] == base[k]) & (rm[k] == base[k])
            fds.append(np.concatenate([rp["P"] - rm["P"], rp["d"] - rm["d"],
                                       (rp["opl"] - rm["opl"])[:, None]], 1) / (vp - vm))
        a, b = fds
        scale = np.abs(a).max(1) + 1e-300
        keep &= np.abs(a - b).max(1) / scale <= 1e-6
        tan = np.concatenate([t["tP"][:, i], t["td"][:, i], t["topl"][:, i][:, None]], 1)
        errs.append((np.abs(tan - a).max(1) / scale)[keep])
    return errs


def test_tangents_match_central_differences_inside():
    """Forward-mode derivatives of the ray state after 800 steps (no exit)
    with respect to six of the 35 coefficients: within 5e-5 of the central
    differences on every ray where those are accurate, with the median ray
    within 1e-6.  A dropped term (the Hessian of n, the derivative of mu or
    of the step length) gives O(1) errors on most rays."""
    for e in _tangent_vs_fd(0.02, 800, (0, 1, 5, 12, 20, 34)):
        assert e.size >= 20
        assert e.max() <= 5e-5 and np.median(e) <= 1e-6, (e.max(), np.median(e))


def test_tangents_match_central_differences_through_the_exit():
    """The same through the exit crossing and the exit refraction: dL0 =
    0.2 mm, so every ray leaves the block within about 160 steps."""
    for e in _tangent_vs_fd(0.2, 20000, (0, 5, 20)):
        assert e.size >= 20
        assert e.max() <= 5e-5 and np.median(e) <= 1e-6, (e.max(), np.median(e))


def _curved_tangent_case(name):
    """(medium, rays, dL0, max steps) whose rays meet a curved surface or an
    n = sqrt(p) or C / p field: the Luneburg lens (sqrt, collimated beam
    through the unit sphere), Maxwell's fish-eye (C / p, rays from an
    interior point refracting out of a sphere of radius 3), the Sec. V
    corrector (n = p, total internal reflections on its cylinder's side) and
    the parabolic fibre (sqrt, some rays leaving through the cylinder's
    side); and the spherical freeform of Sec. V (coefficients a0 .. a3, the
    Hessian of G2 = r cos 5 theta), rays through its unit sphere."""
    if name == "luneburg":
        return W.luneburg_medium(), W.luneburg_rays(8), 2e-3, 5000
    if name == "fisheye":
        th = W.uniform(7, 1, 256, 0.0, math.pi)
        ph = W.uniform(7, 2, 256, 0.0, 2 * math.pi)
        return (W.fisheye_medium(n0=2.0, a=1.0, r_bound=3.0),
                W.Rays(np.tile([0.5, 0.0, 0.0], (256, 1)), W.direction(th, ph)), 2e-3, 5000)
    if name == "corrector":
        wl = W.corrector_workload(128)
        return wl.medium, wl.rays, 5e-3, 20000
    if name == "spherical":
        wl = W.spherical_workload(128)
        return wl.medium, wl.rays, 1e-3, 20000
    x = W.uniform(8, 1, 128, -4.0, 4.0)
    y = W.uniform(8, 2, 128, -3.0, 3.0)
    d = W.direction(W.uniform(8, 3, 128, 0.0, math.radians(40)), W.uniform(8, 4, 128, 0, 2 * math.pi))
    return W.fiber_medium(length=8.0), W.Rays(np.stack([x, y, np.full(128, -1.0)], 1), d), 2e-3, 40000


@pytest.mark.parametrize("name", ["luneburg", "fisheye", "corrector", "fiber", "spherical"])
def test_curved_surface_and_form_tangents_match_central_differences(name):
    """The tangents on curved surfaces and through the n = sqrt(p) and C / p
    forms: the crossing fraction of a sphere or cylinder side by implicit
    differentiation of the surface along the step, the unit normal moving
    with the crossing point, and dn = F'(p) dp for n = F(p).  Against
    central differences as above (h = 1e-6 and 5e-7 on four nonzero
    coefficients and the last one): within 5e-5, median 1e-6, with the
    traced values equal to the oracle's trace.  Leaving out the moving
    normal misses by 3e-3 to 0.4 (Luneburg, fish-eye, corrector), leaving out
    F'(p) by O(1) (Luneburg, fish-eye, fibre), leaving out t's second
    derivatives in G2's Hessian likewise (spherical)."""
    m, rays, dopl, max_steps = _curved_tangent_case(name)
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    base = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    for k in ("P", "d", "opl", "exit_id", "steps"):
        np.testing.assert_array_equal(t[k], base[k], err_msg=k)
    # the surface events this case is there for
    if name in ("luneburg", "fisheye", "spherical"):
        assert (base["exit_id"] == 0).sum() >= 50
    elif name == "corrector":
        assert base["tir_boundary"].sum() >= 2
    else:
        assert (base["exit_id"] == 0).sum() >= 5
    nc = len(m.coeffs)
    coords = [i for i in range(nc) if m.coeffs[i] != 0][:4] + [nc - 1]
    h = 1e-6
    for i in coords:
        keep = (t["flag"] == 0) & (base["exit_id"] >= 0)
        fds = []
        for hh in (h, h / 2):
            res = []
            for s in (+hh, -hh):
                c = m.coeffs.copy()
                c[i] += s
                mm = W.Medium(**{**m.__dict__, "coeffs": c})
                res.append((oracle.trace(mm, rays.origins, rays.dirs, dopl, max_steps), c[i]))
            (rp, vp), (rm, vm) = res
            for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
                keep &= (rp[k] == base[k]) & (rm[k] == base[k])
            fds.append(np.concatenate([rp["P"] - rm["P"], rp["d"] - rm["d"],
                                       (rp["opl"] - rm["opl"])[:, None]], 1) / (vp - vm))
        a, b = fds
        scale = np.abs(a).max(1) + 1e-300
        keep &= np.abs(a - b).max(1) / scale <= 1e-6
        tan = np.concatenate([t["tP"][:, i], t["td"][:, i], t["topl"][:, i][:, None]], 1)
        e = (np.abs(tan - a).max(1) / scale)[keep]
        assert e.size >= 10, (i, e.size)
        assert e.max() <= 5e-5 and np.median(e) <= 1e-6, (i, e.max(), np.median(e))


def test_n2p_lens_tangents_through_the_arc_match_central_differences():
    """The N2P lens (Sec. VI) with respect to R, F, beta, gamma, on the
    design fan: rays parallel to the axis meet the radial gradient with
    N.I = 0 exactly, so their first step is the tangential-incidence arc of
    Sec. II (iv), whose tangent carries k = (n(P'') - n_i) / 2 n_i through the
    extra sample at P'' = P + hi N.  The fan's rays stay nearly parallel to
    the axis, where Eq. 9's D is formed by cancellation, so differences at
    h = 1e-6 are rounding noise; at h = 1e-4 and 5e-5 they agree to about
    1e-7, and the tangents lie within 5e-5 of them (median 1e-6) on every
    ray whose two differences agree to 2e-5.  Without the arc's dk the
    tangents miss by far more."""
    from paper_2606_22655_b300 import n2p_design
    m = W.n2p_lens_medium(0.770, 4.462, 0.3)
    rays = n2p_design.fan(64, 0.3)
    dopl, max_steps = 1e-3, 400000
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    base = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    for k in ("P", "d", "opl", "exit_id", "steps"):
        np.testing.assert_array_equal(t[k], base[k], err_msg=k)
    assert (t["flag"] == 0).all() and (base["exit_id"] == 2).all()
    h = 1e-4
    for i in range(4):
        keep = np.ones(rays.n, bool)
        fds = []
        for hh in (h, h / 2):
            res = []
            for s in (+hh, -hh):
                c = m.coeffs.copy()
                c[i] += s
                mm = W.Medium(**{**m.__dict__, "coeffs": c})
                res.append(oracle.trace(mm, rays.origins, rays.dirs, dopl, max_steps))
            for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
                keep &= (res[0][k] == base[k]) & (res[1][k] == base[k])
            fds.append(np.concatenate([res[0]["P"] - res[1]["P"], res[0]["d"] - res[1]["d"],
                                       (res[0]["opl"] - res[1]["opl"])[:, None]], 1) / (2 * hh))
        a, b = fds
        scale = np.abs(a).max(1) + 1e-300
        keep &= np.abs(a - b).max(1) / scale <= 2e-5
        tan = np.concatenate([t["tP"][:, i], t["td"][:, i], t["topl"][:, i][:, None]], 1)
        e = (np.abs(tan - b).max(1) / scale)[keep]
        assert e.size >= 30, (i, e.size)
        assert e.max() <= 5e-5 and np.median(e) <= 1e-6, (i, e.max(), np.median(e))


def test_layered_shell_tangents_match_central_differences():
    """Point-sampled shells (Sec. I): the Luneburg field in 8 shells.  A
    shell's index is a constant, so dn = 0 and the step lengths and mu do not
    move; the parameters act through the refraction normal grad f / |grad f|
    at each shell change.  Tangents against central differences (h = 1e-6
    and 5e-7) on coefficients 1-4, on every ray whose integer outcomes hold
    and whose differences agree: within 5e-5, median 1e-6; the constant
    coefficient, which shifts f uniformly, has a zero tangent (to rounding).  Taking dn from
    grad f instead (as for a continuous medium) misses by orders of
    magnitude."""
    m = dataclasses.replace(W.luneburg_medium(), n_levels=8, level_lo=1.0, level_hi=math.sqrt(2.0))
    rays = W.luneburg_rays(8)
    dopl, max_steps = 2e-3, 5000
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, dopl, max_steps)
    base = oracle.trace(m, rays.origins, rays.dirs, dopl, max_steps)
    for k in ("P", "d", "opl", "exit_id", "steps"):
        np.testing.assert_array_equal(t[k], base[k], err_msg=k)
    assert (t["flag"] == 0).all()
    big = max(np.abs(t["tP"][:, 1:]).max(), np.abs(t["td"][:, 1:]).max())
    assert max(np.abs(t["tP"][:, 0]).max(), np.abs(t["td"][:, 0]).max()) <= 1e-12 * big
    h = 1e-6
    for i in (1, 2, 3, 4):
        keep = base["exit_id"] >= 0
        fds = []
        for hh in (h, h / 2):
            res = []
            for s in (+hh, -hh):
                c = m.coeffs.copy()
                c[i] += s
                res.append((oracle.trace(W.Medium(**{**m.__dict__, "coeffs": c}), rays.origins, rays.dirs,
                                         dopl, max_steps), c[i]))
            (rp, vp), (rm, vm) = res
            for k in ("exit_id", "steps", "tir_internal", "tir_boundary"):
                keep &= (rp[k] == base[k]) & (rm[k] == base[k])
            fds.append(np.concatenate([rp["P"] - rm["P"], rp["d"] - rm["d"]], 1) / (vp - vm))
        a, b = fds
        scale = np.abs(a).max(1) + 1e-300
        keep &= np.abs(a - b).max(1) / scale <= 1e-6
        tan = np.concatenate([t["tP"][:, i], t["td"][:, i]], 1)
        e = (np.abs(tan - a).max(1) / scale)[keep]
        assert e.size >= 40, (i, e.size)
        assert e.max() <= 5e-5 and np.median(e) <= 1e-6, (i, e.max(), np.median(e))


def test_grid_sample_tangents_match_central_differences():
    """Tangents with respect to grid samples (the weight of a sample at P is
    the product of its per-axis Catmull-Rom weights, summed over the taps the
    edge clamp maps onto it, plus the interpolant's Hessian for the moved
    points): against central differences of oracle traces with the float32
    sample moved by 8 units in the last place, on each ray the sample
    influences: the tangent lies within four times the gap between the
    differences at 16 and 8 units (their own error, a few 1e-6 relative) plus
    1e-6, where a dropped term would miss by orders of magnitude.  The
    samples are the cells that eight rays cross at step 400 and, on the
    entry face, where the edge clamp sums several taps onto one sample, the
    cells they cross at step 2."""
    wl = W.blob_workload(n_rays=256, res=64)
    m, rays = wl.medium, wl.rays
    nz, ny, nx = m.grid.shape
    pts = np.concatenate([oracle.trace(m, rays.origins[:8], rays.dirs[:8], 0.02, k)["P"]
                          for k in (400, 2)])
    cell = np.floor((pts - np.array(m.origin)) / np.array(m.spacing)).astype(np.int64)
    cell = np.clip(cell, 0, [nx - 1, ny - 1, nz - 1])
    samples = (cell[:, 2] * ny + cell[:, 1]) * nx + cell[:, 0]
    t = oracle.trace_tangent(m, rays.origins, rays.dirs, 0.02, 800, samples=samples)
    base = oracle.trace(m, rays.origins, rays.dirs, 0.02, 800)
    for k in ("P", "d", "opl", "exit_id", "steps"):
        np.testing.assert_array_equal(t[k], base[k], err_msg=k)
    flat = m.grid.ravel()
    ulp = float(np.spacing(np.float32(1.5)))
    errs = []
    for q, i in enumerate(samples):
        keep = t["flag"] == 0
        fds = []
        for k in (16, 8):
            res = []
            for s in (+1, -1):
                g = flat.copy()
                g[i] = np.float32(np.float64(g[i]) + s * k * ulp)
                mm = W.Medium(**{**m.__dict__})
                mm.grid = g.reshape(m.grid.shape)
                res.append((oracle.trace(mm, rays.origins, rays.dirs, 0.02, 800), float(g[i])))
            (rp, vp), (rm, vm) = res
            for key in ("exit_id", "steps", "tir_internal", "tir_boundary"):
                keep &= (rp[key] == base[key]) & (rm[key] == base[key])
            fds.append(np.concatenate([rp["P"] - rm["P"], rp["d"] - rm["d"]], 1) / (vp - vm))
        a, b = fds
        scale = np.abs(b).max(1)
        keep &= scale > 0
        tan = np.concatenate([t["tP"][:, q], t["td"][:, q]], 1)
        gap = np.abs(a - b).max(1)
        errs.append((np.abs(tan - b).max(1) / (4.0 * gap + 1e-6 * scale + 1e-300))[keep])
        # a ray the sample cannot reach has a zero tangent
        far = np.abs(a).max(1) == 0
        assert np.abs(tan[far & (t["flag"] == 0)]).max(initial=0.0) == 0.0
    e = np.concatenate(errs)
    assert e.size >= 8
    assert e.max() <= 1.0, e.max()


# ------------------------------------------------- cylinder side wall (Sec. II (i))


def _homogeneous_cylinder(n, radius=1.0, z0=0.0, z1=10.0, n_ext=1.0):
    bk, bp = W.cylinder(0.0, 0.0, radius, z0, z1)
    return W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=0, coeffs=np.array([n]),
                    bkind=bk, bparams=bp, n_ext=n_ext)


def _circle_hits(o, d, radius):
    """Both crossings of the line o + s d with the circle x^2 + y^2 = R^2 in the
    xy plane, by geometry: the foot of the perpendicular from the axis and
    the half chord."""
    dxy = np.array([d[0], d[1]])
    u = dxy / np.linalg.norm(dxy)
    s_foot = -np.dot(o[:2], u)                      # along the projected line
    miss = np.linalg.norm(o[:2] + s_foot * u)       # distance of the line from the axis
    half = math.sqrt(radius * radius - miss * miss)
    scale = np.linalg.norm(dxy)                     # projected length per unit s
    return (s_foot - half) / scale, (s_foot + half) / scale


def test_cylinder_side_wall_entry_and_exit():
    """A homogeneous cylinder (n = 1.5 in air) entered and left through its
    side wall: the entry point is the nearer circle crossing, the outward
    normal there is (x, y, 0)/R, vector Snell (Eq. 1) holds at both walls,
    the ray crosses the chord in ceil(n L / dL0) steps (the last one cut at
    the wall), and OPL = n_ext |E - o| + n L."""
    n, dopl, R = 1.5, 1e-3, 2.0
    m = _homogeneous_cylinder(n, radius=R)
    o = np.array([-5.0, 0.6, 2.0])
    d0 = np.array([1.0, 0.2, 0.14])
    d0 /= np.linalg.norm(d0)
    r = _one(m, o, d0, dopl, 100000)
    s_in, _ = _circle_hits(o, d0, R)
    E = o + s_in * d0
    NE = np.array([E[0], E[1], 0.0]) / R           # outward unit normal
    # direction inside: tangential part of n d conserved, normal part inward
    ti = (1.0 / n) * (d0 - np.dot(d0, NE) * NE)
    Rin = ti - math.sqrt(1.0 - np.dot(ti, ti)) * NE
    np.testing.assert_allclose(1.0 * np.cross(NE, d0), n * np.cross(NE, Rin), atol=1e-15)
    # the far crossing of the chord from E (E lies on the circle)
    rxy = Rin[:2]
    L = -2.0 * np.dot(E[:2], rxy) / np.dot(rxy, rxy)
    X = E + L * Rin
    NX = np.array([X[0], X[1], 0.0]) / R
    assert r["exit_id"] == 0 and r["tir_boundary"] == 0
    assert r["steps"] == math.ceil(n * L / dopl)
    assert 0.05 < (n * L / dopl) % 1 < 0.95  # no rounding ambiguity in the count
    np.testing.assert_allclose(r["P"], X, atol=1e-12)
    assert r["opl"] == pytest.approx(s_in + n * L, rel=1e-13)
    # Snell at the exit wall with the outward normal at X
    np.testing.assert_allclose(n * np.cross(NX, Rin), 1.0 * np.cross(NX, r["d"]), atol=1e-12)
    assert np.dot(r["d"], NX) > 0


@pytest.mark.parametrize("sign", [+1, -1])
def test_cylinder_side_wall_critical_angle_split(sign):
    """Sec. II (v) at the curved wall: a meridional ray from the axis meets
    the side wall where the normal is x; 1e-6 rad beyond the critical angle
    it is reflected, 1e-6 rad short of it it leaves through the side with
    the tangential (z) component of n d conserved."""
    n = 1.5
    m = _homogeneous_cylinder(n, radius=0.7, z0=-50.0, z1=50.0)
    inc = math.asin(1.0 / n) + sign * 1e-6   # angle to the wall normal
    alpha = math.pi / 2 - inc                # angle to the axis
    d0 = np.array([math.sin(alpha), 0.0, math.cos(alpha)])
    r = _one(m, (0, 0, 0), d0, 1e-3, 20000)
    if sign > 0:
        assert r["tir_boundary"] >= 1 and r["exit_id"] != 0
    else:
        assert r["exit_id"] == 0 and r["tir_boundary"] == 0
        assert r["P"][0] == pytest.approx(0.7, abs=1e-12)
        assert r["d"][2] == pytest.approx(n * math.sin(inc), rel=1e-12)


# ------------------------------------------ decision margins (flagging of rays)


def test_boundary_margin_is_distance_in_steps():
    """A ray that runs parallel to the box face x = 1 at distance d keeps every
    step end d from it; the end face z = L sits half a step past the last
    full step, so the boundary margin is d / h with h = dL0 / n."""
    n, dopl, dist = 1.5, 0.01, 1e-4
    h = dopl / n
    z0, k = 0.1, 57
    m = W.homogeneous_box(n, lo=(-1, -1, 0), hi=(1, 1, z0 + (k + 0.5) * h))
    r = _one(m, (1.0 - dist, 0.0, z0), (0, 0, 1), dopl, 1000)
    assert r["exit_id"] == 5 and r["steps"] == k + 1
    assert r["margins"][oracle.M_BND] == pytest.approx(dist / h, rel=1e-9)


@pytest.mark.parametrize("kind", ["sphere", "cylinder"])
def test_curved_boundary_margin_is_distance_in_steps(kind):
    """For a sphere or a cylinder side wall the boundary margin measures the
    distance of a step end to the surface, in steps, to first order: a ray
    from the centre along x whose last interior step end lies half a step
    inside the wall (radius (k + 1/2) h) has margin 1/2 - O(h / R)."""
    n, dopl, k = 1.5, 0.01, 140
    h = dopl / n
    R = (k + 0.5) * h
    if kind == "sphere":
        bk, bp = W.sphere((0.0, 0.0, 0.0), R)
    else:
        bk, bp = W.cylinder(0.0, 0.0, R, -1.0, 1.0)
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=0, coeffs=np.array([n]),
                 bkind=bk, bparams=bp, n_ext=1.0)
    r = _one(m, (0, 0, 0), (1, 0, 0), dopl, 1000)
    assert r["exit_id"] == 0 and r["steps"] == k + 1
    assert r["margins"][oracle.M_BND] == pytest.approx(0.5, abs=h / R)


@pytest.mark.parametrize("deg", [50.0, 20.0])
def test_critical_margin_is_cosine_distance(deg):
    """The critical margin is the distance of |N.I| from its critical value
    cos(theta_c) = sqrt(1 - (n_ext / n)^2): for a ray inside a homogeneous
    box (n = 1.5, air outside) meeting the +x wall at incidence theta it is
    |cos(theta) - cos(theta_c)|, whether the ray leaves (20 deg) or is
    reflected (50 deg); entry refractions (mu < 1) have no critical angle."""
    n = 1.5
    th = math.radians(deg)
    m = W.homogeneous_box(n, lo=(-1, -1, -20), hi=(1, 1, 20))
    # 6000 steps reach both x walls, not the z faces
    r = _one(m, (0, 0, 0), (math.cos(th), 0.0, math.sin(th)), 1e-3, 6000)
    cc = math.cos(math.asin(1.0 / n))
    expect = abs(math.cos(th) - cc)
    if deg < 40:
        assert r["exit_id"] == 1
        assert r["margins"][oracle.M_CRIT] == pytest.approx(expect, rel=1e-12)
    else:
        assert r["tir_boundary"] >= 1
        assert r["margins"][oracle.M_CRIT] == pytest.approx(expect, rel=1e-12)


def test_tangent_margin_is_smallest_normal_cosine():
    """In n = 1.5 + 0.1 x the normal is x at every point; a ray launched at
    angle b off the y axis towards +x bends towards +x, so the smallest
    |N.I| over its refractions is the first one, sin(b)."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (1, 0, 0): 0.1})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, bkind=W.BOUNDARY_BOX,
                 bparams=(-1, -1, -1, 1, 1, 1, 0, 0), n_ext=1.0)
    b = math.radians(3.0)
    r = _one(m, (0, -0.5, 0), (math.sin(b), math.cos(b), 0.0), 1e-3, 5000)
    assert r["margins"][oracle.M_TAN] == pytest.approx(math.sin(b), rel=1e-14)


@pytest.mark.parametrize("levels,z0,expect", [(2, 0.3, 0.7), (2, 0.9, 0.1), (2, 1.6, 0.6),
                                               (4, 0.9, 0.2), (4, 0.2, 0.6)])
def test_level_margin_is_distance_to_next_shell(levels, z0, expect):
    """With f = 1.5 + 0.2 (z - 1) in L shells on [1.3, 1.7] the level
    coordinate L (f - lo) / (hi - lo) is L z / 2; a ray along x at height z0
    keeps it, and its margin is the distance to the nearest shell boundary
    among u = 1 .. L - 1 (u = 0 and u = L bound no shell: the levels
    clamp)."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.2})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                 n_levels=levels, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                 bparams=(-1, -1, 0, 1, 1, 2, 0, 0), n_ext=1.0)
    r = _one(m, (-0.5, 0, z0), (1, 0, 0), 1e-3, 5000)
    assert r["exit_id"] == 1
    assert r["margins"][oracle.M_LEVEL] == pytest.approx(expect, rel=1e-12)


# --------------------------------------------- edge-clamped tricubic (Keys 1981)


def _keys(s):
    """Keys' cubic convolution kernel with a = -1/2 and its derivative, in the
    piecewise form of the 1981 paper."""
    a = abs(s)
    if a <= 1.0:
        return 1.5 * a ** 3 - 2.5 * a ** 2 + 1.0, math.copysign(1.0, s) * (4.5 * a * a - 5.0 * a)
    if a < 2.0:
        return (-0.5 * a ** 3 + 2.5 * a ** 2 - 4.0 * a + 2.0,
                math.copysign(1.0, s) * (-1.5 * a * a + 5.0 * a - 4.0))
    return 0.0, 0.0


def _clamped_tricubic(grid, h, p):
    nz, ny, nx = grid.shape
    u = [p[a] / h for a in range(3)]
    base = [math.floor(x) for x in u]
    v, g = 0.0, [0.0, 0.0, 0.0]
    for k in range(base[2] - 1, base[2] + 3):
        for j in range(base[1] - 1, base[1] + 3):
            for i in range(base[0] - 1, base[0] + 3):
                s = float(grid[min(max(k, 0), nz - 1), min(max(j, 0), ny - 1), min(max(i, 0), nx - 1)])
                (wx, dx), (wy, dy), (wz, dz) = _keys(u[0] - i), _keys(u[1] - j), _keys(u[2] - k)
                v += wx * wy * wz * s
                g[0] += dx * wy * wz * s / h
                g[1] += wx * dy * wz * s / h
                g[2] += wx * wy * dz * s / h
    return v, g


def test_tricubic_edge_clamp_against_keys_kernel():
    """Near and beyond the grid's faces the stencil reaches past the samples;
    taps there repeat the edge sample (R17).  The oracle's value and gradient
    match a sum of Keys-kernel weights over the clamped taps, in the first
    and last cells and half a cell outside, on every axis."""
    res, h = 5, 0.5
    grid = (1.5 + 0.05 * W.uniform(17, 1, res ** 3, -1.0, 1.0)).reshape(res, res, res).astype(np.float32)
    m = W.grid_medium(grid, h, size=h * (res - 1))
    bands = [(-0.5 * h, 0.0), (0.0, h), ((res - 2) * h, (res - 1) * h), ((res - 1) * h, (res - 0.5) * h)]
    pts = []
    for s in range(24):
        lo, hi = bands[s % 4]
        p = W.uniform(18, s, 3, 0.0, 1.0)
        axis = s % 3
        q = [lo + p[0] * (hi - lo) if a == axis else (0.2 + 3.6 * p[a]) * h for a in range(3)]
        pts.append(q)
    pts = np.array(pts)
    n, g = oracle.medium_eval(m, pts)
    for i, p in enumerate(pts):
        v, gg = _clamped_tricubic(grid, h, p)
        assert n[i] == pytest.approx(v, abs=1e-14)
        np.testing.assert_allclose(g[i], gg, atol=1e-13)


# ------------------------------------------ index on the inner side at the exit (R10)


def test_exit_uses_previous_point_index():
    """At the exit face the inner index of Eq. 1 is n_{i-1}, the index at the
    last interior point (the previous point of the step that crossed).  In
    n = 1.5 + 0.1 z' the normals of every refraction are along z, so n_{i-1}
    times the transverse direction is carried unchanged from the entry face
    (where n_ext times it is the input's) to the exit face: the ray leaves
    along its input direction.  Taking n at the surface point instead would
    scale the exit's transverse part by n(P_b) / n_{i-1}, about 1 + 3e-5
    here."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.1})
    m = W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                 bkind=W.BOUNDARY_BOX, bparams=(-10, -10, 0, 10, 10, 2, 0, 0), n_ext=1.0)
    th = math.radians(40.0)
    d0 = np.array([math.sin(th) * 0.8, math.sin(th) * 0.6, math.cos(th)])
    for dopl in (1e-3, 7e-4):
        r = _one(m, (0, 0, -1), d0, dopl, 100000)
        assert r["exit_id"] == 5 and r["tir_internal"] == 0
        np.testing.assert_allclose(r["d"], d0, atol=1e-13)


# --------------------------------------- shells with exact crossings (flag LEVEL_ROOT)


def _planar_shells(levels):
    """f = 1.3 + 0.2 z on z in [0, 2] in L shells on [1.3, 1.7]: shell k is
    the slab 2k/L <= z < 2(k+1)/L with index 1.3 + (k + 1/2) 0.4 / L."""
    c = W.coeffs_from_terms(1, {(0, 0, 0): 1.5, (0, 0, 1): 0.2})
    return W.Medium(kind=W.KIND_POLY, form=W.FORM_LINEAR, degree=1, coeffs=c, off=(0, 0, 1),
                    n_levels=levels, level_lo=1.3, level_hi=1.7, bkind=W.BOUNDARY_BOX,
                    bparams=(-50, -50, 0, 50, 50, 2, 0, 0), n_ext=1.0)


@pytest.mark.parametrize("levels", [4, 32])
def test_level_root_planar_stack_closed_form(levels):
    """With crossings solved, a ray through a stack of planar shells is the
    textbook one: in shell k (thickness T = 2/L, index n_k) it runs straight
    at sin(theta_k) = sin(theta_0) / n_k (Snell at every interface), so it
    leaves at the lateral offset tan(theta_0) + sum T tan(theta_k) along its
    input direction, with OPL 1/cos(theta_0) + sum n_k T / cos(theta_k); a
    crossing does not end a step, so the steps are ceil(inner OPL / dL0)
    (the last one cut at the exit face)."""
    dopl = 1e-3
    m = _planar_shells(levels)
    th0 = math.radians(35.0)
    u = np.array([0.6, 0.8, 0.0])
    d0 = math.sin(th0) * u + np.array([0.0, 0.0, math.cos(th0)])
    res = oracle.trace(m, np.array([[0.0, 0.0, -1.0]]), d0[None], dopl, 1_000_000, threads=1,
                       flags=oracle.LEVEL_ROOT)
    r = {k: v[0] for k, v in res.items()}
    T = 2.0 / levels
    lat, opl = math.tan(th0), 1.0 / math.cos(th0)
    for k in range(levels):
        nk = 1.3 + (k + 0.5) * 0.4 / levels
        tk = math.asin(math.sin(th0) / nk)
        lk = T / math.cos(tk)
        lat += T * math.tan(tk)
        opl += nk * lk
    q = (opl - 1.0 / math.cos(th0)) / dopl
    assert 1e-6 < q % 1 < 1 - 1e-6  # no rounding ambiguity in the count
    steps = math.ceil(q)
    assert r["exit_id"] == 5 and r["tir_internal"] == 0 and r["tir_boundary"] == 0
    np.testing.assert_allclose(r["P"], lat * u + np.array([0, 0, 2.0]), atol=1e-12)
    np.testing.assert_allclose(r["d"], d0, atol=1e-13)
    assert r["opl"] == pytest.approx(opl, rel=1e-13)
    assert r["steps"] == steps


def test_level_root_total_reflection_on_the_shell_plane():
    """Sec. II (v) at an isoindicial surface: in n = 1.6 (z > 1) over n = 1.4
    (z < 1) a ray at 80 deg to the normal (critical angle 61 deg) is
    reflected exactly where it meets the plane z = 1, at x = 0.05 tan(80),
    and leaves it mirrored."""
    m = _planar_shells(2)
    a = math.radians(80.0)
    d0 = np.array([math.sin(a), 0.0, -math.cos(a)])
    h = 1e-3 / 1.6
    n_before = math.floor(0.05 / (h * math.cos(a)))
    res, path = oracle.trace_path(m, (0, 0, 1.05), d0, 1e-3, n_before + 5, flags=oracle.LEVEL_ROOT)
    assert res["tir_internal"][0] == 1
    hit = path[n_before + 1]  # entry point, n_before full steps, then the cut at the plane
    np.testing.assert_allclose(hit, [0.05 * math.tan(a), 0.0, 1.0], atol=1e-13)
    np.testing.assert_allclose(res["d"], [math.sin(a), 0.0, math.cos(a)], atol=1e-14)
    assert np.all(path[: len(path), 2] >= 1.0 - 1e-15)


def test_level_root_spherical_shells():
    """The Luneburg lens in 8 shells on [1, sqrt 2]: every level boundary is a
    sphere r_k = sqrt(2 - b_k^2), so each crossing point lies on one, and with
    the radial normal of Eq. 5 the Bouguer invariant n |r x d| of every
    segment equals the entry value (the impact parameter 0.5)."""
    m = dataclasses.replace(W.luneburg_medium(), n_levels=8, level_lo=1.0, level_hi=math.sqrt(2.0))
    res, path = oracle.trace_path(m, (0.3, 0.4, -1.5), (0, 0, 1), 2e-3, 100000, flags=oracle.LEVEL_ROOT)
    assert res["exit_id"][0] == 0
    radii = np.sqrt(2.0 - (1.0 + np.arange(1, 8) * (math.sqrt(2.0) - 1.0) / 8) ** 2)
    seg = np.diff(path, axis=0)
    dirs = seg / np.linalg.norm(seg, axis=1, keepdims=True)
    n_seg, _ = oracle.medium_eval(m, 0.5 * (path[:-1] + path[1:]))
    inv = n_seg * np.linalg.norm(np.cross(path[:-1], dirs), axis=1)
    assert np.abs(inv - 0.5).max() < 1e-12
    changes = np.nonzero(np.diff(n_seg))[0] + 1  # vertices where the shell changes
    assert len(changes) >= 8
    r = np.linalg.norm(path[changes], axis=1)
    assert np.abs(r[:, None] - radii[None, :]).min(axis=1).max() < 1e-13
