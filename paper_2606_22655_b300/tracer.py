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
import weakref
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
        # objects the library context owns; close() ends them first (servers
        # before the media their jobs use)
        self._servers = weakref.WeakSet()
        self._media = weakref.WeakSet()

    def last_launches(self) -> int:
        v = ctypes.c_int32()
        N.check("grin_ctx_last_launches", self.lib.grin_ctx_last_launches(self.handle, ctypes.byref(v)))
        return int(v.value)

    def close(self) -> None:
        """Close the servers and media made on this context, then the context."""
        if self.handle:
            for obj in list(self._servers) + list(self._media):
                obj.close()
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
        ctx._media.add(self)

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


def empty_result(n: int, device, margins: bool = False) -> Dict[str, torch.Tensor]:
    """Output tensors of a trace; margins=True adds the (n, 4) decision
    margins ("margin")."""
    pin = device == "cpu" and torch.cuda.is_available()
    kw = dict(device=device, pin_memory=pin) if pin else dict(device=device)
    out = {k: torch.empty(n, dtype=torch.float64, **kw) for k in OUT_FIELDS}
    out.update({k: torch.empty(n, dtype=torch.int32, **kw) for k in INT_FIELDS})
    if margins:
        out["margin"] = torch.empty((n, 4), dtype=torch.float64, **kw)
    return out


def _out_struct(out: Dict[str, torch.Tensor]) -> N.Out:
    s = N.Out()
    for k in OUT_FIELDS + INT_FIELDS:
        setattr(s, k, out[k].data_ptr())
    s.margin = out["margin"].data_ptr() if "margin" in out else None
    return s


def _params(dopl: float, max_steps: int, precision: str, level_root: bool = False) -> N.Params:
    if precision not in PRECISION:
        raise ValueError(f"precision must be one of {sorted(PRECISION)}")
    return N.Params(float(dopl), int(max_steps), PRECISION[precision],
                    N.TRACE_LEVEL_ROOT if level_root else 0)


def trace(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
          precision: str = "mixed", stream: Optional[torch.cuda.Stream] = None,
          out: Optional[Dict[str, torch.Tensor]] = None, margins: bool = False,
          level_root: bool = False) -> Dict[str, torch.Tensor]:
    """grin_trace on device tensors; asynchronous on `stream` (default: the
    current torch stream).  margins=True also returns the decision margins;
    level_root=True refracts layered media at the exact shell crossings
    (GRIN_TRACE_LEVEL_ROOT)."""
    if out is None:
        out = empty_result(rays.count, rays.ox.device, margins)
    if stream is None:
        stream = torch.cuda.current_stream(rays.ox.device)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, precision, level_root)
    N.check("grin_trace", ctx.lib.grin_trace(ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps),
                                             ctypes.byref(os_), ctypes.c_void_p(stream.cuda_stream)))
    return out


def trace_host(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
               precision: str = "mixed", stream: Optional[torch.cuda.Stream] = None,
               out: Optional[Dict[str, torch.Tensor]] = None, margins: bool = False,
               level_root: bool = False) -> Dict[str, torch.Tensor]:
    """grin_trace_host: rays and results in host memory (copies and the
    synchronisation happen inside the call)."""
    if out is None:
        out = empty_result(rays.count, "cpu", margins)
    if stream is None:
        stream = torch.cuda.current_stream(ctx.device)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, precision, level_root)
    N.check("grin_trace_host", ctx.lib.grin_trace_host(ctx.handle, medium.handle, ctypes.byref(rs),
                                                       ctypes.byref(ps), ctypes.byref(os_),
                                                       ctypes.c_void_p(stream.cuda_stream)))
    return out


def trace_path(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int, cap: int,
               stream: Optional[torch.cuda.Stream] = None, level_root: bool = False):
    """grin_trace_path (plain FP64) on device tensors: returns (result dict,
    points (count, cap, 3) float64, point counts (count,) int64).  Ray r's
    polyline is points[r, :min(counts[r], cap)]."""
    dev = rays.ox.device
    out = empty_result(rays.count, dev)
    pts = torch.zeros((rays.count, int(cap), 3), dtype=torch.float64, device=dev)
    cnt = torch.zeros(rays.count, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, "fp64", level_root)
    N.check("grin_trace_path", ctx.lib.grin_trace_path(
        ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(os_),
        ctypes.c_void_p(pts.data_ptr()), int(cap), ctypes.c_void_p(cnt.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream)))
    return out, pts, cnt


def to_numpy(res: Dict[str, torch.Tensor]) -> Dict[str, np.ndarray]:
    """Results as numpy with P and d stacked to (n, 3), the oracle's layout
    (and the (n, 4) margins as "margins" when present)."""
    h = {k: v.cpu().numpy() for k, v in res.items()}
    r = dict(P=np.stack([h["px"], h["py"], h["pz"]], 1), d=np.stack([h["dx"], h["dy"], h["dz"]], 1),
             opl=h["opl"], exit_id=h["exit_id"], steps=h["steps"], tir_internal=h["tir_internal"],
             tir_boundary=h["tir_boundary"])
    if "margin" in h:
        r["margins"] = h["margin"]
    return r


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
        ctx._servers.add(self)

    def submit(self, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
               out: Optional[Dict[str, torch.Tensor]] = None, level_root: bool = False):
        """Queue a job; returns (job id, result dict filled when it is DONE)."""
        if out is None:
            out = empty_result(rays.count, "cpu")
        rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, "mixed", level_root)
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

    def timing(self, job_id: int):
        """(seconds queued before admission, seconds from admission to completion)."""
        q, r = ctypes.c_double(), ctypes.c_double()
        N.check("grin_serve_timing", self.ctx.lib.grin_serve_timing(self.handle, job_id, ctypes.byref(q),
                                                                     ctypes.byref(r)))
        return q.value, r.value

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


# ------------------------------------------------------------------ adjoint


def adjoint_workspace_bytes(medium: Medium, count: int, dopl: float, max_steps: int, k: int = 64) -> int:
    v = ctypes.c_size_t()
    ps = _params(dopl, max_steps, "fp64")
    N.check("grin_trace_adjoint_workspace_size", medium.ctx.lib.grin_trace_adjoint_workspace_size(
        medium.handle, int(count), ctypes.byref(ps), int(k), ctypes.byref(v)))
    return int(v.value)


def adjoint_interval(medium: Medium, count: int, dopl: float, max_steps: int,
                     budget_bytes: Optional[int] = None) -> int:
    """grin_trace_adjoint_interval: the checkpoint interval whose workspace
    fits in budget_bytes, 1 (every step stored) when it can.  The default
    budget is half of the device memory free to this process (what the CUDA
    driver reports free plus what torch's allocator holds unused)."""
    if budget_bytes is None:
        dev = torch.device("cuda", medium.ctx.device)
        free = torch.cuda.mem_get_info(dev)[0]
        cached = torch.cuda.memory_reserved(dev) - torch.cuda.memory_allocated(dev)
        budget_bytes = (free + cached) // 2
    v = ctypes.c_int32()
    ps = _params(dopl, max_steps, "fp64")
    N.check("grin_trace_adjoint_interval", medium.ctx.lib.grin_trace_adjoint_interval(
        medium.handle, int(count), ctypes.byref(ps), int(budget_bytes), ctypes.byref(v)))
    return int(v.value)


def trace_adjoint(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
                  grads: Dict[str, torch.Tensor], n_params: int, k: int = 64,
                  stream: Optional[torch.cuda.Stream] = None):
    """grin_trace_adjoint: returns (forward results, dL/d(parameters) as a
    float64 device tensor).  `grads` holds dL/d(px, py, pz, dx, dy, dz, opl)
    as float64 device tensors."""
    dev = rays.ox.device
    out = empty_result(rays.count, dev)
    grad = torch.zeros(n_params, dtype=torch.float64, device=dev)
    ws = torch.empty(max(adjoint_workspace_bytes(medium, rays.count, dopl, max_steps, k), 1),
                     dtype=torch.uint8, device=dev)
    g = {key: grads[key].contiguous().to(torch.float64) for key in OUT_FIELDS}
    gs = N.OutGrad(*[g[key].data_ptr() for key in OUT_FIELDS])
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, "fp64")
    N.check("grin_trace_adjoint", ctx.lib.grin_trace_adjoint(
        ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(os_), ctypes.byref(gs),
        ctypes.c_void_p(grad.data_ptr()), int(k), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        ctypes.c_void_p(stream.cuda_stream)))
    return out, grad


def trace_stats(ctx: Context, out: Dict[str, torch.Tensor], margin_min=None,
                stream: Optional[torch.cuda.Stream] = None) -> Dict[str, object]:
    """grin_trace_stats_compute on a result dict of trace(): totals of the
    rays' outcomes (and, with margin_min, four thresholds, the rays flagged
    by their margins), plus the device time of the context's last trace."""
    n = int(out["exit_id"].numel())
    dev = out["exit_id"].device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    st = N.TraceStats()
    mm = None if margin_min is None else (ctypes.c_double * 4)(*[float(v) for v in margin_min])
    N.check("grin_trace_stats_compute", ctx.lib.grin_trace_stats_compute(
        ctx.handle, ctypes.byref(_out_struct(out)), n, mm, ctypes.byref(st), ctypes.c_void_p(stream.cuda_stream)))
    return {"rays": st.rays, "ray_steps": st.ray_steps, "exit_face": list(st.exit_face),
            "exit_miss": st.exit_miss, "exit_entry_reflect": st.exit_entry_reflect,
            "exit_max_steps": st.exit_max_steps, "exit_invalid": st.exit_invalid,
            "tir_internal": st.tir_internal, "tir_boundary": st.tir_boundary,
            "flagged": st.flagged, "elapsed_ms": st.elapsed_ms}


def trace_adjoint_forward(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
                          k: int = 64, stream: Optional[torch.cuda.Stream] = None):
    """grin_trace_adjoint_forward: the forward sweep alone.  Returns (forward
    results, workspace); hand the workspace, unchanged, to
    trace_adjoint_backward with the same medium, rays, dopl, max_steps and k."""
    dev = rays.ox.device
    out = empty_result(rays.count, dev)
    ws = torch.empty(max(adjoint_workspace_bytes(medium, rays.count, dopl, max_steps, k), 1),
                     dtype=torch.uint8, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rs, os_, ps = _rays_struct(rays), _out_struct(out), _params(dopl, max_steps, "fp64")
    N.check("grin_trace_adjoint_forward", ctx.lib.grin_trace_adjoint_forward(
        ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(os_), int(k),
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(stream.cuda_stream)))
    return out, ws


def trace_adjoint_backward(ctx: Context, medium: Medium, rays: RayBatch, dopl: float, max_steps: int,
                           grads: Dict[str, torch.Tensor], n_params: int, k: int, ws: torch.Tensor,
                           stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """grin_trace_adjoint_backward: dL/d(parameters) (float64 device tensor)
    from the workspace a trace_adjoint_forward call filled."""
    dev = rays.ox.device
    grad = torch.zeros(n_params, dtype=torch.float64, device=dev)
    g = {key: grads[key].contiguous().to(torch.float64) for key in OUT_FIELDS}
    gs = N.OutGrad(*[g[key].data_ptr() for key in OUT_FIELDS])
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rs, ps = _rays_struct(rays), _params(dopl, max_steps, "fp64")
    N.check("grin_trace_adjoint_backward", ctx.lib.grin_trace_adjoint_backward(
        ctx.handle, medium.handle, ctypes.byref(rs), ctypes.byref(ps), ctypes.byref(gs),
        ctypes.c_void_p(grad.data_ptr()), int(k), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        ctypes.c_void_p(stream.cuda_stream)))
    return grad


def _with_params(spec, theta: torch.Tensor):
    import copy
    s = copy.copy(spec)
    if spec.kind == 1:
        s.grid = theta.detach().to(torch.float32).reshape(spec.grid.shape).contiguous()
    else:
        s.coeffs = theta.detach().cpu().numpy().astype(np.float64)
    return s


class TraceFunction(torch.autograd.Function):
    """Exit point, direction and optical path of every ray as a function of
    the medium parameters theta (polynomial coefficients, the spherical
    freeform's a0..a3, the N2P lens's R, F, beta, gamma, or grid samples).
    forward runs the adjoint's forward sweep (the plain FP64 trace, which also
    stores the checkpoints) and backward its backward sweep from them, so the
    rays are traced forward once.  k = 0 takes the checkpoint interval from
    adjoint_interval (every step stored when half the free memory holds it)."""

    @staticmethod
    def forward(fctx, theta, gctx, spec, rays, dopl, max_steps, k):
        med = Medium(gctx, _with_params(spec, theta))
        if not k:
            k = adjoint_interval(med, rays.count, dopl, max_steps)
        res, ws = trace_adjoint_forward(gctx, med, rays, dopl, max_steps, k)
        fctx.save_for_backward(theta)
        fctx.extra = (gctx, med, rays, dopl, max_steps, k, ws)
        P = torch.stack([res["px"], res["py"], res["pz"]], 1)
        d = torch.stack([res["dx"], res["dy"], res["dz"]], 1)
        fctx.mark_non_differentiable(res["exit_id"])
        return P, d, res["opl"], res["exit_id"]

    @staticmethod
    def backward(fctx, gP, gd, gopl, gexit):
        (theta,) = fctx.saved_tensors
        gctx, med, rays, dopl, max_steps, k, ws = fctx.extra
        fctx.extra = None  # the workspace is released after this sweep
        n = rays.count
        z = lambda t, i: torch.zeros(n, dtype=torch.float64, device=rays.ox.device) if t is None else t[:, i]
        grads = {"px": z(gP, 0), "py": z(gP, 1), "pz": z(gP, 2), "dx": z(gd, 0), "dy": z(gd, 1), "dz": z(gd, 2),
                 "opl": torch.zeros(n, dtype=torch.float64, device=rays.ox.device) if gopl is None else gopl}
        grad = trace_adjoint_backward(gctx, med, rays, dopl, max_steps, grads, theta.numel(), k, ws)
        return grad.reshape(theta.shape).to(theta.dtype), None, None, None, None, None, None


def traced_exit(theta: torch.Tensor, ctx: Context, spec, rays: RayBatch, dopl: float, max_steps: int,
                k: int = 0):
    """(P, d, opl, exit_id) differentiable in theta (see TraceFunction); k is
    the checkpoint interval, 0 to choose it by the free device memory."""
    return TraceFunction.apply(theta, ctx, spec, rays, dopl, max_steps, k)


def image_plane_loss(P, d, exit_id, targets, z_img: float, mask=None):
    """Mean over rays of the squared distance, in the plane z = z_img, between
    where the ray's exit line crosses the plane and its target (rays that did
    not leave through the surface, or are False in `mask`, contribute
    zero)."""
    valid = exit_id >= 0
    if mask is not None:
        valid = valid & mask
    sig = (z_img - P[:, 2]) / d[:, 2]
    X = P[:, 0] + sig * d[:, 0]
    Y = P[:, 1] + sig * d[:, 1]
    e = (X - targets[:, 0]) ** 2 + (Y - targets[:, 1]) ** 2
    return torch.where(valid, e, torch.zeros_like(e)).sum() / P.shape[0]
