"""ctypes declarations of the C ABI in include/grin.h and the library loader.

The library is the in-tree build paper_2606_22655_b300/lib/libgrin_vrt.so; if
it is missing, loading raises (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GRIN_LIB may name another build of the same library (e.g. one compiled
# with different launch bounds); it must export the same C ABI
# GRIN_CHECKED=1 loads the bounds-checked build (every kernel array index
# range-checked; grin_checked_status reports a violation)
LIB_PATH = os.environ.get("GRIN_LIB") or os.path.join(
    HERE, "lib", "libgrin_vrt_checked.so" if os.environ.get("GRIN_CHECKED") == "1" else "libgrin_vrt.so")

GRIN_OK = 0
(GRIN_ERR_INVALID_ARG, GRIN_ERR_OOM, GRIN_ERR_CUDA, GRIN_ERR_NOT_IMPLEMENTED, GRIN_ERR_TIMEOUT,
 GRIN_ERR_BUSY, GRIN_ERR_NOT_FOUND, GRIN_ERR_CANCELLED, GRIN_ERR_CHECKED_BOUNDS) = range(-1, -10, -1)
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA runtime error",
          -4: "not implemented", -5: "timed out", -6: "busy", -7: "not found", -8: "cancelled",
          -9: "index out of bounds (checked build)"}
TRACE_LEVEL_ROOT = 1
EXIT_MISS, EXIT_ENTRY_REFLECT, EXIT_MAXSTEPS, EXIT_INVALID = -1, -2, -3, -4
F32, F64 = 0, 1
PREC_FP64, PREC_FP32_MIXED, PREC_FP64_FAST = 0, 1, 2
STATIC_MAX_RAYS = 65536

_d3 = ctypes.c_double * 3
_vp = ctypes.c_void_p


class MediumDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("form", ctypes.c_int32), ("form_c", ctypes.c_double),
        ("degree", ctypes.c_int32), ("coeffs", ctypes.POINTER(ctypes.c_double)),
        ("norm_offset", _d3), ("norm_scale", _d3),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("grid", _vp), ("grid_on_device", ctypes.c_int32),
        ("origin", _d3), ("spacing", _d3),
        ("n_levels", ctypes.c_int32), ("level_lo", ctypes.c_double), ("level_hi", ctypes.c_double),
        ("boundary_kind", ctypes.c_int32), ("boundary", ctypes.c_double * 8),
        ("n_ext", ctypes.c_double),
    ]


class Rays(ctypes.Structure):
    _fields_ = [("ox", _vp), ("oy", _vp), ("oz", _vp), ("dx", _vp), ("dy", _vp), ("dz", _vp),
                ("count", ctypes.c_int64), ("dtype", ctypes.c_int32)]


class Out(ctypes.Structure):
    _fields_ = [("px", _vp), ("py", _vp), ("pz", _vp), ("dx", _vp), ("dy", _vp), ("dz", _vp),
                ("opl", _vp), ("exit_id", _vp), ("steps", _vp), ("tir_internal", _vp),
                ("tir_boundary", _vp), ("margin", _vp)]


class Params(ctypes.Structure):
    _fields_ = [("dopl", ctypes.c_double), ("max_steps", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class OutGrad(ctypes.Structure):
    _fields_ = [("px", _vp), ("py", _vp), ("pz", _vp), ("dx", _vp), ("dy", _vp), ("dz", _vp), ("opl", _vp)]


class TraceStats(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_int64), ("ray_steps", ctypes.c_int64), ("exit_face", ctypes.c_int64 * 6),
                ("exit_miss", ctypes.c_int64), ("exit_entry_reflect", ctypes.c_int64),
                ("exit_max_steps", ctypes.c_int64), ("exit_invalid", ctypes.c_int64),
                ("tir_internal", ctypes.c_int64), ("tir_boundary", ctypes.c_int64),
                ("flagged", ctypes.c_int64), ("elapsed_ms", ctypes.c_double)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("step_quantum", ctypes.c_int32),
                ("max_slots_per_job", ctypes.c_int32)]


class ServeCounters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("done", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("ticks", ctypes.c_uint64), ("ray_steps", ctypes.c_double),
                ("arena_bytes", ctypes.c_size_t), ("arena_in_use", ctypes.c_size_t),
                ("slots_total", ctypes.c_int32), ("slots_in_use", ctypes.c_int32),
                ("jobs_queued", ctypes.c_int32), ("jobs_running", ctypes.c_int32)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELLED = 0, 1, 2, 3, 4

_lib = None


def load() -> ctypes.CDLL:
    """Load libgrin_vrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run python -m paper_2606_22655_b300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "grin_ctx_create": (ctypes.c_int, [ctypes.c_int, P(_vp)]),
        "grin_ctx_destroy": (ctypes.c_int, [_vp]),
        "grin_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "grin_poly_terms": (ctypes.c_int, [ctypes.c_int]),
        "grin_medium_create": (ctypes.c_int, [_vp, P(MediumDesc), P(_vp)]),
        "grin_medium_destroy": (ctypes.c_int, [_vp]),
        "grin_medium_device_bytes": (ctypes.c_int, [_vp, P(ctypes.c_size_t)]),
        "grin_trace": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), _vp]),
        "grin_trace_host": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), _vp]),
        "grin_trace_path": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), _vp, ctypes.c_int64,
                                           _vp, _vp]),
        "grin_ctx_last_launches": (ctypes.c_int, [_vp, P(ctypes.c_int32)]),
        "grin_trace_stats_compute": (ctypes.c_int, [_vp, P(Out), ctypes.c_int64, P(ctypes.c_double),
                                                    P(TraceStats), _vp]),
        "grin_trace_host_static": (ctypes.c_int, [P(MediumDesc), P(Rays), P(Params), P(Out), _vp]),
        "grin_trace_adjoint_workspace_size": (ctypes.c_int, [_vp, ctypes.c_int64, P(Params), ctypes.c_int32,
                                                             P(ctypes.c_size_t)]),
        "grin_trace_adjoint_interval": (ctypes.c_int, [_vp, ctypes.c_int64, P(Params), ctypes.c_size_t,
                                                       P(ctypes.c_int32)]),
        "grin_trace_adjoint": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), P(OutGrad), _vp, ctypes.c_int32,
                                              _vp, ctypes.c_size_t, _vp]),
        "grin_trace_adjoint_forward": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), ctypes.c_int32,
                                                      _vp, ctypes.c_size_t, _vp]),
        "grin_trace_adjoint_backward": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(OutGrad), _vp,
                                                       ctypes.c_int32, _vp, ctypes.c_size_t, _vp]),
        "grin_serve_create": (ctypes.c_int, [_vp, P(ServeConfig), P(_vp)]),
        "grin_serve_destroy": (ctypes.c_int, [_vp]),
        "grin_serve_submit": (ctypes.c_int, [_vp, _vp, P(Rays), P(Params), P(Out), P(ctypes.c_uint64)]),
        "grin_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, P(ctypes.c_int32), P(ctypes.c_double)]),
        "grin_serve_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, P(ctypes.c_int32)]),
        "grin_serve_cancel": (ctypes.c_int, [_vp, ctypes.c_uint64]),
        "grin_serve_timing": (ctypes.c_int, [_vp, ctypes.c_uint64, P(ctypes.c_double), P(ctypes.c_double)]),
        "grin_serve_stats": (ctypes.c_int, [_vp, P(ServeCounters)]),
        "grin_build_checked": (ctypes.c_int, []),
        "grin_checked_status": (ctypes.c_int, [ctypes.c_int, P(ctypes.c_int32)]),
        "grin_checked_selftest": (ctypes.c_int, [ctypes.c_int]),
        "grin_probe_fp32_fma": (ctypes.c_int, [ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_double)]),
        "grin_probe_l2_read": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, P(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class GrinError(RuntimeError):
    def __init__(self, call: str, status: int):
        super().__init__(f"{call} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


def check(call: str, status: int) -> None:
    if status != GRIN_OK:
        raise GrinError(call, status)
