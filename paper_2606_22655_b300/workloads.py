"""Seeded synthetic inputs: media descriptions and ray bundles.

This module only draws random numbers and lays out input arrays; it holds none
of the tracing arithmetic, so both the CUDA library and the FP64 oracle can be
fed from it.  Randomness comes from a counter-based SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): output i
of stream s is the SplitMix64 finaliser applied to base(seed, s) + (i+1)*golden.

Media follow the workloads used to exercise the method of Chavez-Islas et al.:
the Luneburg lens n = sqrt(2 - r^2) (Sec. VI, the n(r_p) mapping), the
parabolic-index fiber of Sec. IV, Eq. 22, a freeform polynomial block, a
sampled blob field and its layered (isoindicial shell) version.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 20260622

# medium kinds, polynomial forms and boundary kinds (shared vocabulary only)
KIND_POLY, KIND_GRID, KIND_SPHERICAL, KIND_N2P = 0, 1, 2, 3
FORM_LINEAR, FORM_SQRT, FORM_RECIP = 0, 1, 2
BOUNDARY_BOX, BOUNDARY_SPHERE, BOUNDARY_CYLINDER = 0, 1, 2


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        return _mix(s)[0]


def u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n raw 64-bit outputs of stream `stream`, starting at counter `offset`."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_base(seed, stream) + i * GOLDEN)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform on [lo, hi) from the top 53 bits."""
    u = (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, n: int, sigma: float = 1.0) -> np.ndarray:
    """n standard-normal doubles by Box-Muller from two uniform streams."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 7919, n)
    return sigma * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def n_monomials(degree: int) -> int:
    return (degree + 1) * (degree + 2) * (degree + 3) // 6


def monomial_exponents(degree: int):
    """Graded-lex order: total degree s ascending; within s, i descending,
    then j descending (x^i y^j z^k, k = s - i - j)."""
    out = []
    for s in range(degree + 1):
        for i in range(s, -1, -1):
            for j in range(s - i, -1, -1):
                out.append((i, j, s - i - j))
    return out


def coeffs_from_terms(degree: int, terms: Dict[Tuple[int, int, int], float]) -> np.ndarray:
    idx = {e: k for k, e in enumerate(monomial_exponents(degree))}
    c = np.zeros(n_monomials(degree), dtype=np.float64)
    for e, v in terms.items():
        c[idx[e]] = v
    return c


@dataclasses.dataclass
class Medium:
    """A GRIN medium in a homogeneous surround.

    kind: KIND_POLY (polynomial p of the normalised coordinates
    x' = (x - off) / scale, with n = p, sqrt(p) or form_c / p) or KIND_GRID
    (float32 samples grid[k, j, i] at origin + (i, j, k) * spacing, read by
    Catmull-Rom tricubic interpolation) or KIND_SPHERICAL (the spherical
    freeform field of Sec. V, coeffs = a0..a3, normalised by `scale`) or
    KIND_N2P (the N2P cylinder lens of Sec. VI, coeffs = R, F, beta, gamma,
    axis through off[0], off[1]).
    n_levels > 0 quantises the field into
    that many isoindicial shells between level_lo and level_hi.  The boundary
    is a box (lo[3], hi[3]), sphere (c[3], R) or z-cylinder (cx, cy, R, z0,
    z1), surrounded by index n_ext."""

    kind: int = KIND_POLY
    form: int = FORM_LINEAR
    form_c: float = 1.0
    degree: int = 0
    coeffs: np.ndarray = dataclasses.field(default_factory=lambda: np.ones(1))
    off: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    scale: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    grid: Optional[np.ndarray] = None
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    spacing: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    n_levels: int = 0
    level_lo: float = 0.0
    level_hi: float = 1.0
    bkind: int = BOUNDARY_BOX
    bparams: Tuple[float, ...] = (0.0,) * 8
    n_ext: float = 1.0
    name: str = ""

    @property
    def grid_shape(self) -> Tuple[int, int, int]:
        if self.grid is None:
            return (0, 0, 0)
        nz, ny, nx = self.grid.shape
        return (nx, ny, nz)


@dataclasses.dataclass
class Rays:
    origins: np.ndarray  # (n, 3) float64
    dirs: np.ndarray     # (n, 3) float64, unit

    @property
    def n(self) -> int:
        return int(self.origins.shape[0])

    def subset(self, idx) -> "Rays":
        return Rays(np.ascontiguousarray(self.origins[idx]), np.ascontiguousarray(self.dirs[idx]))


@dataclasses.dataclass
class Workload:
    name: str
    medium: Medium
    rays: Rays
    dopl: float
    max_steps: int
    l_ref: float  # length scale for relative position errors


def _pad8(*v):
    v = list(v)
    return tuple(v + [0.0] * (8 - len(v)))


def box(lo, hi):
    return BOUNDARY_BOX, _pad8(*lo, *hi)


def sphere(c, r):
    return BOUNDARY_SPHERE, _pad8(*c, r)


def cylinder(cx, cy, r, z0, z1):
    return BOUNDARY_CYLINDER, _pad8(cx, cy, r, z0, z1)


def direction(theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """r(theta, phi) = (sin t cos p, sin t sin p, cos t) (the initial direction
    of the paper's flowchart, Fig. 5)."""
    st = np.sin(theta)
    return np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=1)


# ----------------------------------------------------------------- media


def luneburg_medium(radius: float = 1.0) -> Medium:
    """n = sqrt(2 - (r/R)^2) inside the sphere of radius R, n = 1 outside."""
    c = coeffs_from_terms(2, {(0, 0, 0): 2.0, (2, 0, 0): -1.0, (0, 2, 0): -1.0, (0, 0, 2): -1.0})
    bk, bp = sphere((0.0, 0.0, 0.0), radius)
    return Medium(kind=KIND_POLY, form=FORM_SQRT, degree=2, coeffs=c,
                  scale=(radius, radius, radius), bkind=bk, bparams=bp, n_ext=1.0,
                  name="luneburg")


def fisheye_medium(n0: float = 2.0, a: float = 1.0, r_bound: float = 3.0) -> Medium:
    """Maxwell fish-eye n = n0 / (1 + (r/a)^2) inside a bounding sphere."""
    c = coeffs_from_terms(2, {(0, 0, 0): 1.0, (2, 0, 0): 1.0, (0, 2, 0): 1.0, (0, 0, 2): 1.0})
    bk, bp = sphere((0.0, 0.0, 0.0), r_bound)
    return Medium(kind=KIND_POLY, form=FORM_RECIP, form_c=n0, degree=2, coeffs=c,
                  scale=(a, a, a), bkind=bk, bparams=bp, n_ext=1.0, name="fisheye")


def fiber_medium(nc: float = 1.38, delta: float = 0.2, radius: float = 5.0,
                 length: float = 60.0) -> Medium:
    """Parabolic-index fiber (Sec. IV, Eq. 22): n^2 = nc^2 (1 - 2 delta rho^2/R^2)
    in the core rho <= R, z in [0, length]; the surround has the cladding index
    nc sqrt(1 - 2 delta)."""
    c = coeffs_from_terms(2, {(0, 0, 0): nc * nc, (2, 0, 0): -2.0 * delta * nc * nc,
                              (0, 2, 0): -2.0 * delta * nc * nc})
    bk, bp = cylinder(0.0, 0.0, radius, 0.0, length)
    return Medium(kind=KIND_POLY, form=FORM_SQRT, degree=2, coeffs=c,
                  scale=(radius, radius, radius), bkind=bk, bparams=bp,
                  n_ext=nc * math.sqrt(1.0 - 2.0 * delta), name="fiber")


# Fringe Zernike polynomials Z_m (University of Arizona ordering) as monomials
# {(i, j): coefficient} of x' = rho cos(theta), y' = rho sin(theta):
# Z5 = rho^2 cos 2t, Z8 = (3 rho^3 - 2 rho) sin t, Z9 = 6 rho^4 - 6 rho^2 + 1,
# Z11 = rho^3 sin 3t, Z12 = (4 rho^4 - 3 rho^2) cos 2t, and the rest up to Z13.
FRINGE_ZERNIKE = {
    1: {(0, 0): 1.0},
    2: {(1, 0): 1.0},
    3: {(0, 1): 1.0},
    4: {(2, 0): 2.0, (0, 2): 2.0, (0, 0): -1.0},
    5: {(2, 0): 1.0, (0, 2): -1.0},
    6: {(1, 1): 2.0},
    7: {(3, 0): 3.0, (1, 2): 3.0, (1, 0): -2.0},
    8: {(2, 1): 3.0, (0, 3): 3.0, (0, 1): -2.0},
    9: {(4, 0): 6.0, (2, 2): 12.0, (0, 4): 6.0, (2, 0): -6.0, (0, 2): -6.0, (0, 0): 1.0},
    10: {(3, 0): 1.0, (1, 2): -3.0},
    11: {(2, 1): 3.0, (0, 3): -1.0},
    12: {(4, 0): 4.0, (0, 4): -4.0, (2, 0): -3.0, (0, 2): 3.0},
    13: {(3, 1): 8.0, (1, 3): 8.0, (1, 1): -6.0},
}
# Legendre polynomials V_n(z') as {power: coefficient}.
LEGENDRE = {0: {0: 1.0}, 1: {1: 1.0}, 2: {2: 1.5, 0: -0.5}}
# The corrector's nonzero expansion coefficients c_{m,n} (Sec. V).
CORRECTOR_COEFFS = {(5, 0): -0.2368, (8, 0): 0.0249, (9, 0): 0.0011, (11, 0): -0.0078,
                    (12, 0): -0.0013, (8, 1): 0.5548, (11, 1): -0.1731}


def corrector_lens_medium(n_lo: float = 1.5148, n_hi: float = 1.5162, rho_max: float = 4.2,
                          z_max: float = 2.5, coeffs=None, n_ext: float = 1.0) -> Medium:
    """Freeform cylindrical GRIN corrector (Sec. V, binary linear composition):
    n = n0 + dn sum c_mn Z_m(x', y') V_n(z') with n0 = (n_hi + n_lo)/2,
    dn = (n_hi - n_lo)/2, x' = x/rho_max, y' = y/rho_max, z' = 2z/z_max - 1,
    inside the cylinder rho <= rho_max, 0 <= z <= z_max.  Every Zernike and
    Legendre term is a polynomial, so the expansion is handed to the tracers
    as a polynomial medium of the normalised coordinates (degree 4 for the
    paper's coefficients)."""
    coeffs = CORRECTOR_COEFFS if coeffs is None else coeffs
    n0, dn = 0.5 * (n_hi + n_lo), 0.5 * (n_hi - n_lo)
    terms: Dict[Tuple[int, int, int], float] = {(0, 0, 0): n0}
    for (m, v), c in coeffs.items():
        for (i, j), zc in FRINGE_ZERNIKE[m].items():
            for k, vc in LEGENDRE[v].items():
                terms[(i, j, k)] = terms.get((i, j, k), 0.0) + dn * c * zc * vc
    degree = max(sum(e) for e in terms)
    bk, bp = cylinder(0.0, 0.0, rho_max, 0.0, z_max)
    return Medium(kind=KIND_POLY, form=FORM_LINEAR, degree=degree,
                  coeffs=coeffs_from_terms(degree, terms), off=(0.0, 0.0, 0.5 * z_max),
                  scale=(rho_max, rho_max, 0.5 * z_max), bkind=bk, bparams=bp, n_ext=n_ext,
                  name="corrector_lens")


def spherical_freeform_medium(a=(1.5, 1.0, -0.2, 0.3), radius: float = 1.0, centre=(0.0, 0.0, 0.0),
                              n_ext: float = 1.0) -> Medium:
    """Spherical freeform GRIN medium (Sec. V): n = a0 + a1 G1 + a2 G2 + a3 G3
    with G1 = 0.3 (r^2 - 1), G2 = r cos(5 theta), G3 = r^2 sin^2(theta) cos(2 phi)
    in coordinates normalised by the sphere's radius; the paper's a = (1.5, 1,
    -0.2, 0.3) and r_max = 1.  The surround index is not given; 1 is taken."""
    bk, bp = sphere(centre, radius)
    return Medium(kind=KIND_SPHERICAL, form=FORM_LINEAR, degree=0,
                  coeffs=np.asarray(a, dtype=np.float64), off=tuple(centre),
                  scale=(radius, radius, radius), bkind=bk, bparams=bp, n_ext=n_ext,
                  name="spherical_freeform")


def n2p_lens_medium(beta: float, gamma: float, L: float = 0.3, R: float = 1.0, F: float = 2.0) -> Medium:
    """Cylindrical N2P-GRIN lens (Sec. VI): n = [1 + ((R^2 - (rho/2)^2)/F^2)^beta]^gamma
    for z in [-L, 0], rho <= R, in air; axis = z."""
    bk, bp = cylinder(0.0, 0.0, R, -L, 0.0)
    return Medium(kind=KIND_N2P, form=FORM_LINEAR, degree=0,
                  coeffs=np.array([R, F, beta, gamma], dtype=np.float64), bkind=bk, bparams=bp,
                  n_ext=1.0, name="n2p_lens")


def homogeneous_box(n: float, lo=(-1.0, -1.0, 0.0), hi=(1.0, 1.0, 1.0), n_ext: float = 1.0) -> Medium:
    bk, bp = box(lo, hi)
    return Medium(kind=KIND_POLY, form=FORM_LINEAR, degree=0, coeffs=np.array([n]),
                  bkind=bk, bparams=bp, n_ext=n_ext, name="homogeneous")


def freeform_block_medium(seed: int = BASE_SEED + 1, sigma: float = 0.01, base: float = 1.55,
                          spread: float = 0.10) -> Medium:
    """10 x 10 x 20 mm box (x, y in [-5, 5], z in [0, 20]) in air with
    n = base + sum c_ijk x'^i y'^j z'^k over the 35 monomials of degree <= 4,
    x' = x/5, y' = y/5, z' = (z - 10)/10, c ~ N(0, sigma) scaled by
    min(1, spread / sum |c|) so that |n - base| <= spread everywhere."""
    c = normal(seed, 11, n_monomials(4), sigma)
    s = min(1.0, spread / float(np.abs(c).sum()))
    c = c * s
    c[0] += base
    bk, bp = box((-5.0, -5.0, 0.0), (5.0, 5.0, 20.0))
    return Medium(kind=KIND_POLY, form=FORM_LINEAR, degree=4, coeffs=c,
                  off=(0.0, 0.0, 10.0), scale=(5.0, 5.0, 10.0), bkind=bk, bparams=bp,
                  n_ext=1.0, name="freeform_block")


def blob_field(res: int, seed: int = BASE_SEED + 2, n_blobs: int = 64, size: float = 20.0,
               base: float = 1.5) -> Tuple[np.ndarray, float]:
    """n = base + sum_b a_b exp(-|x - c_b|^2 / (2 sigma_b^2)) sampled in FP64 at
    res^3 vertex-centred points of [0, size]^3 and stored as float32
    (grid[k, j, i]); centres U[0, size]^3, sigma U[1, 4] mm, a U[-0.05, 0.05]."""
    cen = uniform(seed, 21, 3 * n_blobs, 0.0, size).reshape(n_blobs, 3)
    sig = uniform(seed, 22, n_blobs, 1.0, 4.0)
    amp = uniform(seed, 23, n_blobs, -0.05, 0.05)
    h = size / (res - 1)
    x = np.arange(res, dtype=np.float64) * h
    e = [np.exp(-((x[None, :] - cen[:, a:a + 1]) ** 2) / (2.0 * sig[:, None] ** 2)) for a in range(3)]
    A = (amp[:, None, None] * e[2][:, :, None] * e[1][:, None, :]).reshape(n_blobs, res * res)
    field = base + (A.T @ e[0]).reshape(res, res, res)
    return field.astype(np.float32), h


def grid_medium(grid: np.ndarray, h: float, size: float = 20.0, n_levels: int = 0) -> Medium:
    bk, bp = box((0.0, 0.0, 0.0), (size, size, size))
    lo, hi = (float(grid.min()), float(grid.max())) if n_levels else (0.0, 1.0)
    return Medium(kind=KIND_GRID, grid=np.ascontiguousarray(grid, dtype=np.float32),
                  origin=(0.0, 0.0, 0.0), spacing=(h, h, h), n_levels=n_levels,
                  level_lo=lo, level_hi=hi, bkind=bk, bparams=bp, n_ext=1.0,
                  name="layered" if n_levels else "grid")


# ------------------------------------------------------------------ rays


def luneburg_rays(n_side: int = 64, radius: float = 0.95, z0: float = -1.5) -> Rays:
    """n_side^2 rays parallel to +z on a cell-centred n_side x n_side grid mapped
    into the disk of the given radius by the Shirley-Chiu concentric map."""
    k = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    u, v = np.meshgrid(k, k, indexing="xy")
    a = (2.0 * u - 1.0).ravel()
    b = (2.0 * v - 1.0).ravel()
    big_a = np.abs(a) > np.abs(b)
    safe_a = np.where(a == 0.0, 1.0, a)
    safe_b = np.where(b == 0.0, 1.0, b)
    r = np.where(big_a, a, b)
    phi = np.where(big_a, (math.pi / 4.0) * (b / safe_a), math.pi / 2.0 - (math.pi / 4.0) * (a / safe_b))
    o = np.stack([radius * r * np.cos(phi), radius * r * np.sin(phi), np.full(a.shape, z0)], axis=1)
    d = np.zeros_like(o)
    d[:, 2] = 1.0
    return Rays(o, d)


def point_source_rays(n: int, seed: int, src=(0.0, 0.0, -5.0), half_angle_deg: float = 30.0) -> Rays:
    """Rays from one point, polar angle uniform in [0, half_angle], azimuth
    uniform in [0, 2 pi), about +z."""
    th = uniform(seed, 31, n, 0.0, math.radians(half_angle_deg))
    ph = uniform(seed, 32, n, 0.0, 2.0 * math.pi)
    d = direction(th, ph)
    o = np.tile(np.asarray(src, dtype=np.float64), (n, 1))
    return Rays(o, d)


def collimated_face_rays(n: int, seed: int, size: float = 20.0, max_angle_deg: float = 10.0,
                         standoff: float = 1.0) -> Rays:
    """Entry points uniform on the z = 0 face, directions proportional to
    (tan ax, tan ay, 1) with ax, ay uniform in +-max_angle; each ray starts
    `standoff` before the face."""
    x = uniform(seed, 41, n, 0.0, size)
    y = uniform(seed, 42, n, 0.0, size)
    ax = uniform(seed, 43, n, -math.radians(max_angle_deg), math.radians(max_angle_deg))
    ay = uniform(seed, 44, n, -math.radians(max_angle_deg), math.radians(max_angle_deg))
    d = np.stack([np.tan(ax), np.tan(ay), np.ones(n)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.stack([x, y, np.zeros(n)], axis=1) - standoff * d / d[:, 2:3]
    return Rays(o, d)


# -------------------------------------------------------------- workloads


def luneburg_workload() -> Workload:
    """Luneburg lens R = 1, 4096 rays along +z from z = -1.5 over the disk of
    radius 0.95; dL0 = 1e-3, at most 5000 steps."""
    return Workload("luneburg_4096", luneburg_medium(), luneburg_rays(), 1e-3, 5000, 1.0)


def freeform_workload(n_rays: int = 1 << 20, seed: int = BASE_SEED + 1,
                      ray_seed: Optional[int] = None) -> Workload:
    """Analytic freeform polynomial block, point source 5 mm before the
    entrance face, half-angle 30 deg; dL0 = 0.01 mm, at most 20000 steps.
    `ray_seed` (default `seed`) draws the bundle."""
    m = freeform_block_medium(seed)
    rays = point_source_rays(n_rays, seed if ray_seed is None else ray_seed)
    return Workload(f"freeform_block_{n_rays}", m, rays, 0.01, 20000,
                    math.sqrt(5.0 ** 2 + 5.0 ** 2 + 10.0 ** 2))


def corrector_example_ray() -> Rays:
    """The corrector lens example of Fig. 3(a): P0 = (1, -5, -1.5),
    theta0 = 80 deg, phi0 = 110 deg."""
    d = direction(np.radians([80.0]), np.radians([110.0]))
    return Rays(np.array([[1.0, -5.0, -1.5]]), d)


def corrector_workload(n_rays: int = 1 << 16, seed: int = BASE_SEED + 5, **lens) -> Workload:
    """The corrector lens with a bundle launched from the plane z = -1.5:
    origins uniform over the disk of radius 4, directions within 20 deg of
    +z; dL0 = 1e-3 (about 3,800 steps through the 2.5-unit thickness), at
    most 20000 steps."""
    m = corrector_lens_medium(**lens)
    r = 4.0 * np.sqrt(uniform(seed, 1, n_rays))
    a = uniform(seed, 2, n_rays, 0.0, 2.0 * math.pi)
    o = np.stack([r * np.cos(a), r * np.sin(a), np.full(n_rays, -1.5)], 1)
    d = direction(uniform(seed, 3, n_rays, 0.0, math.radians(20.0)),
                  uniform(seed, 4, n_rays, 0.0, 2.0 * math.pi))
    return Workload(f"corrector_lens_{n_rays}", m, Rays(o, d), 1e-3, 20000,
                    math.sqrt(4.2 ** 2 + 1.25 ** 2))


def spherical_example_ray() -> Rays:
    """The spherical freeform example of Fig. 3(b): P0 = (-1, -1, -1),
    theta0 = 80 deg, phi0 = 20 deg."""
    return Rays(np.array([[-1.0, -1.0, -1.0]]), direction(np.radians([80.0]), np.radians([20.0])))


def spherical_workload(n_rays: int = 1 << 16, seed: int = BASE_SEED + 6, **medium) -> Workload:
    """The spherical freeform medium with rays from random points on the
    sphere of radius 1.5 aimed at random points within 0.7 of the centre;
    dL0 = 1e-3, at most 20000 steps."""
    m = spherical_freeform_medium(**medium)
    def on_sphere(stream):
        cz = uniform(seed, stream, n_rays, -1.0, 1.0)
        ph = uniform(seed, stream + 1, n_rays, 0.0, 2.0 * math.pi)
        s = np.sqrt(1.0 - cz * cz)
        return np.stack([s * np.cos(ph), s * np.sin(ph), cz], 1)
    o = 1.5 * on_sphere(1)
    t = 0.7 * np.cbrt(uniform(seed, 5, n_rays))[:, None] * on_sphere(3)
    d = t - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Workload(f"spherical_freeform_{n_rays}", m, Rays(o, d), 1e-3, 20000, 1.0)


def blob_workload(n_rays: int = 1 << 22, res: int = 256, n_levels: int = 0,
                  seed: int = BASE_SEED + 2) -> Workload:
    """256^3 float32 blob field over a 20 mm cube (or its 32-shell layered
    version), collimated rays within +-10 deg; dL0 = 0.005 mm."""
    g, h = blob_field(res, seed)
    m = grid_medium(g, h, n_levels=n_levels)
    name = ("layered" if n_levels else "grid") + f"_{res}_{n_rays}"
    return Workload(name, m, collimated_face_rays(n_rays, seed), 0.005, 20000,
                    math.sqrt(3.0) * 10.0)


def design_targets(n_rays: int, seed: int = BASE_SEED + 4, n_spots: int = 16, half: float = 2.0) -> np.ndarray:
    """Target spot of each ray for the image-plane design loss: n_spots spots
    uniform in [-half, half]^2 mm, ray i aimed at spot i mod n_spots."""
    spots = np.stack([uniform(seed, 51, n_spots, -half, half), uniform(seed, 52, n_spots, -half, half)], 1)
    return spots[np.arange(n_rays) % n_spots]
