"""Thin Python binding of the C ABI (argument marshalling only).

Device memory and streams come from PyTorch; every step of the trace runs in
the CUDA library (libgrin_vrt.so).  Names follow include/grin.h:

    ctx = Context(0)
    med = Medium(ctx, workloads.freeform_block_medium())
    rays = RayBatch.from_numpy(origins, dirs, device="cuda", dtype=torch.float32)
    res = trace(ctx, med, rays, dopl=0.01, max_steps=20000, precision="mixed")
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Dict, Optional

import numpy as np
import torch

from . import _native as N

PRECISION = {"fp64": N.PREC_FP64, "mixed": N.PREC_FP32_MIXED, "fp64-fast": N.PREC_FP64_FAST}
OUT_FIELDS = ("px", "py", "pz", "dx", "dy", "dz", "opl")
INT_FIELDS = ("exit_id", "steps", "tir_internal", "tir_boundary")


class Context:
    """grin_ctx_create / grin_ctx_destroy."""

    def __init__(self, device: int = 0):
        self.lib = N.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        N.check("grin_ctx_create", self.lib.grin_ctx_create(self.device, ctypes.byref(h)))
        self.handle = h

    def last_launches(self) -> int:
        v = ctypes.c_int32()
        N.check("grin_ctx_last_launches", self.lib.grin_ctx_last_launches(self.handle, ctypes.byref(v)))
        return int(v.value)

    def close(self) -> None:
        if self.handle:
            N.check("grin_ctx_destroy", self.lib.grin_ctx_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def medium_desc(spec) -> (N.MediumDesc, list):
    """Fill a grin_medium_desc from a medium description object (attributes
    as in workloads.Medium); returns the struct and the buffers it points to."""
    keep = []
    d = N.MediumDesc()
    d.kind, d.form, d.form_c = int(spec.kind), int(spec.form), float(spec.form_c)
    d.degree = int(spec.degree)
    c = np.ascontiguousarray(np.asarray(spec.coeffs, dtype=np.float64))
    keep.append(c)
    d.coeffs = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.norm_offset = (ctypes.c_double * 3)(*spec.off)
    d.norm_scale = (ctypes.c_double * 3)(*spec.scale)
    g = getattr(spec, "grid", None)
    if g is not None:
        if isinstance(g, torch.Tensor):
            t = g.contiguous().to(torch.float32)
            keep.append(t)
            d.grid = t.data_ptr()
            d.grid_on_device = 1 if t.is_cuda else 0
            nz, ny, nx = t.shape
        else:
            a = np.ascontiguousarray(g, dtype=np.float32)
            keep.append(a)
            d.grid = a.ctypes.data
            d.grid_on_device = 0
            nz, ny, nx = a.shape
        d.nx, d.ny, d.nz = nx, ny, nz
    d.origin = (ctypes.c_double * 3)(*spec.origin)
    d.spacing = (ctypes.c_double * 3)(*spec.spacing)
    d.n_levels, d.level_lo, d.level_hi = int(spec.n_levels), float(spec.level_lo), float(spec.level_hi)
    d.boundary_kind = int(spec.bkind)
    d.boundary = (ctypes.c_double * 8)(*spec.bparams)
    d.n_ext = float(spec.n_ext)
    return d, keep


class Medium:
    """grin_medium_create / grin_medium_destroy (the library keeps a device copy)."""

    def __init__(self, ctx: Context, spec):
        self.ctx = ctx
        self.spec = spec
        d, keep = medium_desc(spec)
        h = ctypes.c_void_p()
        N.check("grin_medium_create", ctx.lib.grin_medium_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        N.check("grin_medium_device_bytes", self.ctx.lib.grin_medium_device_bytes(self.handle, ctypes.byref(v)))
        return int(v.value)

    def close(self) -> None:
        if self.handle:
            N.check("grin_medium_destroy", self.ctx.lib.grin_medium_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class RayBatch:
    """Structure-of-arrays rays (six 1-D tensors of one dtype and device)."""

    ox: torch.Tensor
    oy: torch.Tensor
    oz: torch.Tensor
    dx: torch.Tensor
    dy: torch.Tensor
    dz: torch.Tensor

    @property
    def count(self) -> int:
        return int(self.ox.numel())

    @staticmethod
    def from_numpy(origins: np.ndarray, dirs: np.ndarray, device="cuda", dtype=torch.float32,
                   pin: bool = False) -> "RayBatch":
        cols = [origins[:, 0], origins[:, 1], origins[:, 2], dirs[:, 0], dirs[:, 1], dirs[:, 2]]
        ts = []
        for c in cols:
            t = torch.from_numpy(np.ascontiguousarray(c)).to(dtype)
            if pin:
                t = t.pin_memory()
            ts.append(t.to(device) if device != "cpu" else t)
        return RayBatch(*ts)

    def tensors(self):
        return (self.ox, self.oy, self.oz, self.dx, self.dy, self.dz)


def _rays_struct(r: RayBatch) -> N.Rays:
    ts = r.tensors()
    dt = ts[0].dtype
    for t in ts:
        if t.dtype != dt or not t.is_contiguous() or t.numel() != r.count:
            raise ValueError("ray arrays must be contiguous, of one dtype and one length")
    if dt == torch.float32:
        code = N.F32
    elif dt == torch.float64:
        code = N.F64
    else:
        raise ValueError("rays must be float32 or float64")
    s = N.Rays()
    s.ox, s.oy, s.oz, s.dx, s.dy, s.dz = [t.data_ptr() for t in ts]
    s.count, s.dtype = r.count, code
    return s


def empty_result(n: int, device) -> Dict[str, torch.Tensor]:
    pin = device == "cpu" and torch.cuda.is_available()
    kw = dict(device=device, pin_memory=pin) if pin else dict(device=device)
    out = {k: torch.empty(n, dtype=torch.float64, **kw) for k in OUT_FIELDS}
    out.update({k: torch.empty(n, dtype=torch.int32, **kw) for k in INT_FIELDS})
    return out


def _out_struct(out: Dict[str, torch.Tensor]) -> N.Out:
    s = N.Out()
    for k in OUT_FIELDS + INT_FIELDS:
        setattr(s, k, out[k].data_ptr())
    return s


def _params(dopl: float, max_steps: int, precision: str) -> N.Params:
    if precision not in PRECISION:
        raise ValueError(f"precision must be one of {sorted(PRECISION)}")
    return N.Params(float(dopl), int(max_steps), PRECISION[precision], 0)


def trace(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
          precision: str = "mixed", stream: Optional[torch.cuda.Stream] = None,
          out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """grin_trace on device tensors; asynchronous on `stream` (default: the
    current torch stream)."""
    if out is None:
        out = empty_result(rays.count, rays.ox.device)
    if stream is None:
        stream = torch.cuda.current_stream(rays.ox.device)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, precision)
    N.check("grin_trace", ctx.lib.grin_trace(ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps),
                                             ctypes.byref(os_), ctypes.c_void_p(stream.cuda_stream)))
    return out


def trace_host(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
               precision: str = "mixed", stream: Optional[torch.cuda.Stream] = None,
               out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """grin_trace_host: rays and results in host memory (copies and the
    synchronisation happen inside the call)."""
    if out is None:
        out = empty_result(rays.count, "cpu")
    if stream is None:
        stream = torch.cuda.current_stream(ctx.device)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, precision)
    N.check("grin_trace_host", ctx.lib.grin_trace_host(ctx.handle, medium.handle, ctypes.byref(rs),
                                                       ctypes.byref(ps), ctypes.byref(os_),
                                                       ctypes.c_void_p(stream.cuda_stream)))
    return out


def to_numpy(res: Dict[str, torch.Tensor]) -> Dict[str, np.ndarray]:
    """Results as numpy with P and d stacked to (n, 3), the oracle's layout."""
    h = {k: v.cpu().numpy() for k, v in res.items()}
    return dict(P=np.stack([h["px"], h["py"], h["pz"]], 1), d=np.stack([h["dx"], h["dy"], h["dz"]], 1),
                opl=h["opl"], exit_id=h["exit_id"], steps=h["steps"], tir_internal=h["tir_internal"],
                tir_boundary=h["tir_boundary"])


class Server:
    """grin_serve_*: continuous batching of trace jobs (mixed precision,
    host buffers).  Buffers handed to submit() are kept referenced here until
    the job has ended."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, step_quantum: int = 0,
                 max_slots_per_job: int = 0):
        self.ctx = ctx
        cfg = N.ServeConfig(int(hbm_budget_bytes), int(step_quantum), int(max_slots_per_job))
        h = ctypes.c_void_p()
        N.check("grin_serve_create", ctx.lib.grin_serve_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
               out: Optional[Dict[str, torch.Tensor]] = None):
        """Queue a job; returns (job id, result dict filled when it is DONE)."""
        if out is None:
            out = empty_result(rays.count, "cpu")
        rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, "mixed")
        jid = ctypes.c_uint64()
        N.check("grin_serve_submit", self.ctx.lib.grin_serve_submit(
            self.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(os_), ctypes.byref(jid)))
        self._keep[jid.value] = (rays, out)
        return jid.value, out

    def poll(self, job_id: int):
        st, lat = ctypes.c_int32(), ctypes.c_double()
        N.check("grin_serve_poll", self.ctx.lib.grin_serve_poll(self.handle, job_id, ctypes.byref(st), ctypes.byref(lat)))
        if st.value >= N.JOB_DONE:
            self._keep.pop(job_id, None)
        return st.value, lat.value

    def wait(self, job_id: int, timeout_s: float = 60.0) -> int:
        st = ctypes.c_int32()
        rc = self.ctx.lib.grin_serve_wait(self.handle, job_id, float(timeout_s), ctypes.byref(st))
        if rc == -5:
            return -5
        N.check("grin_serve_wait", rc)
        self._keep.pop(job_id, None)
        return st.value

    def cancel(self, job_id: int) -> None:
        N.check("grin_serve_cancel", self.ctx.lib.grin_serve_cancel(self.handle, job_id))

    def stats(self) -> Dict[str, float]:
        c = N.ServeCounters()
        N.check("grin_serve_stats", self.ctx.lib.grin_serve_stats(self.handle, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in N.ServeCounters._fields_}

    def close(self) -> None:
        if self.handle:
            N.check("grin_serve_destroy", self.ctx.lib.grin_serve_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
