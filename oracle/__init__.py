"""FP64 CPU oracle for Vectorial Ray Tracing -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  It wraps `vrt_oracle.c`, a plain FP64 C
transcription of the VRT step (Chavez-Islas et al., Sec. II), through ctypes.
It does not import the CUDA library or share any of its code; media and rays
are read from plain attribute objects (see `paper_2606_22655_b300.workloads`
for the generator that feeds both sides).

Parity status per function (pins live in tests/test_oracle_pins.py):
  - homogeneous stepping, OPL, step count: pinned (exact line, n L, ceil);
  - boundary refraction / TIR / normal incidence: pinned (Snell, critical
    angle split, reflection law);
  - interior refraction and TIR on smooth media: pinned by the Luneburg
    closed form (exit point, direction, OPL), the Maxwell fish-eye conjugate
    point, the conserved n |r x d| under spherical symmetry, the fiber helix
    RMSE and first-order step halving;
  - polynomial evaluator: pinned against exact rational arithmetic and
    central differences;
  - tricubic evaluator: pinned by exact reproduction of quadratic fields and
    of the samples at nodes;
  - layered shells: pinned by Snell's law at a planar level crossing;
  - tangent incidence (case iv): pinned by its closed-form first arc;
  - cylinder side wall (entry and exit roots, radial normal, critical-angle
    split): pinned by the half-chord geometry and vector Snell;
  - decision margins (boundary, critical, tangent, level): pinned by rays
    built with known distances, cosines and level coordinates;
  - edge-clamped tricubic taps: pinned against Keys' piecewise kernel;
  - the inner index at the exit face (n at the last interior point): pinned
    by the conserved transverse momentum of a z-stratified medium;
  - forward-mode tangents (trace_tangent; polynomial coefficients with
    n = p, sqrt(p) or C / p, the spherical freeform's a0..a3, the N2P lens's
    R, F, beta, gamma, or grid samples; box, sphere or cylinder; continuous
    or in point-sampled shells; through the tangential-incidence arc):
    values and decisions bitwise those of trace; derivatives pinned against
    central differences of trace, inside the medium, through the exit, on
    curved surfaces, at edge-clamped samples and in shells;
  - freeform and blob media as a whole: parity unpinned beyond the
    invariants above (no closed form exists).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_vrt.so")
_lib = None

EXIT_MISS, EXIT_ENTRY_REFLECT, EXIT_MAXSTEPS, EXIT_INVALID = -1, -2, -3, -4
M_CRIT, M_TAN, M_BND, M_LEVEL = 0, 1, 2, 3
LEVEL_ROOT = 1  # trace flag: shell crossings solved on the step (layered media)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 -ffp-contract=off (no fused multiply-add,
    so each operation rounds on its own)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vrt_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Medium(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("form", ctypes.c_int32), ("form_c", ctypes.c_double),
        ("degree", ctypes.c_int32), ("coeffs", ctypes.POINTER(ctypes.c_double)),
        ("off", ctypes.c_double * 3), ("scale", ctypes.c_double * 3),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("grid", ctypes.POINTER(ctypes.c_float)),
        ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
        ("n_levels", ctypes.c_int32), ("level_lo", ctypes.c_double), ("level_hi", ctypes.c_double),
        ("bkind", ctypes.c_int32), ("b", ctypes.c_double * 8), ("n_ext", ctypes.c_double),
    ]


class _Params(ctypes.Structure):
    _fields_ = [("dopl", ctypes.c_double), ("max_steps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("index_rule", ctypes.c_int32), ("perturb", ctypes.c_double), ("seed", ctypes.c_uint64)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.orc_medium_eval.argtypes = [ctypes.POINTER(_Medium), dp, dp, dp]
        lib.orc_trace_batch.argtypes = [ctypes.POINTER(_Medium), ctypes.POINTER(_Params),
                                        ctypes.c_int64, dp, dp, dp, dp, dp, ip, ip, ip, ip, dp,
                                        ctypes.c_int32]
        lib.orc_trace_path.argtypes = [ctypes.POINTER(_Medium), ctypes.POINTER(_Params), dp, dp,
                                       dp, dp, dp, ip, ip, ip, ip, dp, dp, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64)]
        lib.orc_trace_tangent.argtypes = [ctypes.POINTER(_Medium), ctypes.POINTER(_Params),
                                          ctypes.c_int64, dp, dp, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int64), dp, dp, dp, ip, ip, dp,
                                          dp, dp, ip, ctypes.c_int32]
        _lib = lib
    return _lib


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


class _Bound:
    """Keeps the numpy buffers referenced by a _Medium alive."""

    def __init__(self, m):
        self.coeffs = np.ascontiguousarray(np.asarray(m.coeffs, dtype=np.float64))
        self.grid = None if m.grid is None else np.ascontiguousarray(m.grid, dtype=np.float32)
        s = _Medium()
        s.kind, s.form, s.form_c, s.degree = int(m.kind), int(m.form), float(m.form_c), int(m.degree)
        s.coeffs = _ptr(self.coeffs)
        s.off = (ctypes.c_double * 3)(*m.off)
        s.scale = (ctypes.c_double * 3)(*m.scale)
        if self.grid is not None:
            nz, ny, nx = self.grid.shape
            s.nx, s.ny, s.nz = nx, ny, nz
            s.grid = _ptr(self.grid, ctypes.c_float)
        s.origin = (ctypes.c_double * 3)(*m.origin)
        s.spacing = (ctypes.c_double * 3)(*m.spacing)
        s.n_levels, s.level_lo, s.level_hi = int(m.n_levels), float(m.level_lo), float(m.level_hi)
        s.bkind = int(m.bkind)
        s.b = (ctypes.c_double * 8)(*m.bparams)
        s.n_ext = float(m.n_ext)
        self.s = s


def medium_eval(medium, points) -> (np.ndarray, np.ndarray):
    """n and grad n at each of the (k, 3) points (after layering, if any)."""
    lib = _load()
    b = _Bound(medium)
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    n = np.zeros(pts.shape[0])
    g = np.zeros_like(pts)
    for i in range(pts.shape[0]):
        nn = ctypes.c_double()
        lib.orc_medium_eval(ctypes.byref(b.s), _ptr(pts[i]), ctypes.byref(nn), _ptr(g[i]))
        n[i] = nn.value
    return n, g


def trace(medium, origins, dirs, dopl: float, max_steps: int,
          threads: Optional[int] = None, flags: int = 0, index_rule: int = 0,
          perturb: float = 0.0, seed: int = 0) -> Dict[str, np.ndarray]:
    """Trace every ray; returns exit point P, direction d, optical path opl,
    exit_id, steps, tir_internal, tir_boundary and margins (n, 4).
    index_rule, perturb and seed select the conditioning probe (see
    vrt_oracle.h); the defaults trace the method itself."""
    lib = _load()
    b = _Bound(medium)
    o = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    n = o.shape[0]
    out = dict(P=np.zeros((n, 3)), d=np.zeros((n, 3)), opl=np.zeros(n),
               exit_id=np.zeros(n, np.int32), steps=np.zeros(n, np.int32),
               tir_internal=np.zeros(n, np.int32), tir_boundary=np.zeros(n, np.int32),
               margins=np.zeros((n, 4)))
    prm = _Params(float(dopl), int(max_steps), int(flags), int(index_rule), float(perturb), int(seed))
    if threads is None:
        threads = os.cpu_count() or 1
    if n:
        ip = lambda a: _ptr(a, ctypes.c_int32)
        lib.orc_trace_batch(ctypes.byref(b.s), ctypes.byref(prm), n, _ptr(o), _ptr(d),
                            _ptr(out["P"]), _ptr(out["d"]), _ptr(out["opl"]), ip(out["exit_id"]),
                            ip(out["steps"]), ip(out["tir_internal"]), ip(out["tir_boundary"]),
                            _ptr(out["margins"]), int(threads))
    return out


def trace_path(medium, origin, direction, dopl: float, max_steps: int, cap: Optional[int] = None,
               flags: int = 0):
    """One ray with its full list of points inside the medium; returns
    (result dict, path (m, 3))."""
    lib = _load()
    b = _Bound(medium)
    o = np.ascontiguousarray(origin, dtype=np.float64).reshape(3)
    d = np.ascontiguousarray(direction, dtype=np.float64).reshape(3)
    cap = int(max_steps + 2 if cap is None else cap)
    path = np.zeros((cap, 3))
    out = dict(P=np.zeros(3), d=np.zeros(3), opl=np.zeros(1), exit_id=np.zeros(1, np.int32),
               steps=np.zeros(1, np.int32), tir_internal=np.zeros(1, np.int32),
               tir_boundary=np.zeros(1, np.int32), margins=np.zeros(4))
    plen = ctypes.c_int64()
    ip = lambda a: _ptr(a, ctypes.c_int32)
    prm = _Params(float(dopl), int(max_steps), int(flags), 0, 0.0, 0)
    lib.orc_trace_path(ctypes.byref(b.s), ctypes.byref(prm), _ptr(o), _ptr(d), _ptr(out["P"]),
                       _ptr(out["d"]), _ptr(out["opl"]), ip(out["exit_id"]), ip(out["steps"]),
                       ip(out["tir_internal"]), ip(out["tir_boundary"]), _ptr(out["margins"]),
                       _ptr(path), cap, ctypes.byref(plen))
    return out, path[: plen.value]


def trace_tangent(medium, origins, dirs, dopl: float, max_steps: int, samples=None,
                  threads: Optional[int] = None) -> Dict[str, np.ndarray]:
    """Exit state of every ray (as `trace`) and its forward-mode derivative
    with respect to each polynomial coefficient (polynomial media, n = p,
    sqrt(p) or form_c / p), to a0 .. a3 (the spherical freeform), to R, F,
    beta, gamma (the N2P lens) or to each
    grid sample in `samples` (flat
    indices, x fastest; grid media): tP, td (n, nc, 3), topl (n, nc); flag
    (n,) marks rays whose tangents are not followed (tangential incidence,
    clamped crossing fraction).  Box, sphere or cylinder boundaries;
    continuous media or point-sampled shells (whose constant indices have
    zero derivatives; the shells' refraction normals still move)."""
    lib = _load()
    b = _Bound(medium)
    o = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    n = o.shape[0]
    if samples is None:
        # the spherical freeform's a0 .. a3, the N2P lens's (R, F, beta, gamma)
        nc = 4 if medium.kind in (2, 3) else (medium.degree + 1) * (medium.degree + 2) * (medium.degree + 3) // 6
        par = np.zeros(1, np.int64)
    else:
        par = np.ascontiguousarray(samples, dtype=np.int64).ravel()
        nc = par.size
    out = dict(P=np.zeros((n, 3)), d=np.zeros((n, 3)), opl=np.zeros(n),
               exit_id=np.zeros(n, np.int32), steps=np.zeros(n, np.int32),
               tP=np.zeros((n, nc, 3)), td=np.zeros((n, nc, 3)), topl=np.zeros((n, nc)),
               flag=np.zeros(n, np.int32))
    prm = _Params(float(dopl), int(max_steps), 0, 0, 0.0, 0)
    ip = lambda a: _ptr(a, ctypes.c_int32)
    rc = lib.orc_trace_tangent(ctypes.byref(b.s), ctypes.byref(prm), n, _ptr(o), _ptr(d),
                               0 if samples is None else nc, _ptr(par, ctypes.c_int64),
                               _ptr(out["P"]), _ptr(out["d"]), _ptr(out["opl"]), ip(out["exit_id"]),
                               ip(out["steps"]), _ptr(out["tP"]), _ptr(out["td"]), _ptr(out["topl"]),
                               ip(out["flag"]), int(threads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("trace_tangent: polynomial or grid media, not layered, samples in range")
    return out
