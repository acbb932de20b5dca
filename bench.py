"""Benchmark: batched VRT trace of the analytic freeform GRIN block.

One step = one grin_trace call of the mixed-precision persistent tracer over
the whole batch: 1,048,576 rays from a point source 5 mm before a 10x10x20 mm
block with a degree-4 polynomial index (35 monomials), dL0 = 0.01 mm, at most
20,000 steps per ray.  Metric: ray-steps/s (sum over rays of interior steps,
divided by time), with the exit error of the measured run against the plain
FP64 GPU tracer reported beside it (gate: 2e-5 relative).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference that exists
for this method) on a bounded strided sample of the same rays.  Under
torchrun (N > 1) every rank traces its own seeded batch of the same size
(weak scaling, no collective on the data path) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-steps/s at ≤2e-5 rel exit error vs plain FP64 GPU path; serve p50/p99 latency"
UNIT = "ray-steps/s"
N_RAYS = 1 << 20
L2_FLUSH_BYTES = 256 << 20
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock


def poly_fma_count(D: int) -> int:
    """FMAs of the nested-Horner value + gradient evaluation of a total-degree
    D polynomial in three variables (the kernel's poly_vg)."""
    f = 0
    for i in range(D, -1, -1):
        for j in range(D - i, -1, -1):
            top = D - i - j
            f += max(top, 0) + max(top - 1, 0)
            if j != D - i:
                f += 2 + (j != D - i - 1)
        if i != D:
            f += 3 + (i != D - 1)
    return f


# FP32 FLOPs of one refracting VRT step besides the polynomial (FMA = 2):
# compensated position update 15, normalised coordinates 6, gradient scale 3,
# n and 1/n 2, |grad|^2 + rsqrt + N 9, N.I 5, mu / 1-mu^2 / D 10, near-critical
# band test 3, gamma 3, R = mu I + gamma N 9, renormalisation 9, step length 1.
STEP_FIXED_FLOPS = 75


def flops_per_step(degree_class: int) -> int:
    return 2 * poly_fma_count(degree_class) + STEP_FIXED_FLOPS


KERNEL_SOURCES = ["paper_2606_22655_b300/csrc/trace_mixed.cu", "paper_2606_22655_b300/csrc/grin_device.cuh",
                  "paper_2606_22655_b300/csrc/grin_internal.h"]
KERNEL = "k_trace_mixed<Cfg<4,false,false,box,linear>,false>"
PROFILE = "profiles/k_trace_mixed_freeform_block_1048576.md"


def profiled_value(key: str):
    """A figure `key: value` from the committed ncu summary of the kernel, or
    None if the kernel sources changed since that capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, PROFILE)).read()
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha: ([0-9a-f]+)", text)
    v = re.search(re.escape(key) + r": ([0-9.]+)", text)
    if not sha or not v or sha.group(1) != h.hexdigest()[:16]:
        return None
    return float(v.group(1))


def profiled_traffic():
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    v = profiled_value("traffic_bytes_per_launch")
    return None if v is None else int(v)


# CUDA-core issue peak: 148 SMs x 128 FP32 lanes x 2.032 GHz, lane operations a second
FP32_ISSUE_PEAK = 148 * 128 * 2.032e9


def fp32_issue(rate: float):
    """FP32 issue rate against the CUDA-core peak: the executed FFMA + FADD +
    FMUL lane operations per ray-step, two for each packed FFMA2, that ncu
    counted for this kernel (committed summary) times the measured
    ray-steps/s."""
    ops = profiled_value("fp32_lane_ops_per_ray_step")
    if ops is None:
        return None
    achieved = ops * rate
    return {"achieved": achieved / 1e12, "peak": FP32_ISSUE_PEAK / 1e12, "unit": "T lane-ops/s",
            "frac": achieved / FP32_ISSUE_PEAK, "fp32_lane_ops_per_ray_step": ops,
            "source": "ncu sass op counts (FFMA + FADD + FMUL + 2 FFMA2) of " + PROFILE}


def rank_ray_seed(rank: int) -> int:
    """Each rank traces its own seeded bundle of the same size (weak scaling)."""
    from paper_2606_22655_b300 import workloads as W
    return W.BASE_SEED + 1 + 1000 * rank


def aggregate(region_s: float, steps_per_trace: float, steps: int, ws: int, device=None) -> (float, float):
    """Whole-job rate: the ray-steps every rank traced over the slowest
    rank's time.  Two all-reduces (MAX of the time, SUM of the ray-steps),
    both after the timed region; the data path has none.
    Returns (seconds, ray-steps/s)."""
    work = steps_per_trace * steps
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([region_s], dtype=torch.float64, device=device)
        w = torch.tensor([work], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        region_s, work = float(t.item()), float(w.item())
    return region_s, work / region_s


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class _Nvml:
    """The few read-only NVML calls the clock sampler needs, through ctypes on
    the driver's libnvidia-ml (no Python binding needed)."""

    def __init__(self, cuda_index: int):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            p = torch.cuda.get_device_properties(cuda_index)
            bus = b"%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            pass
        if bus is None or self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) != 0:
            if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(cuda_index), ctypes.byref(self.h)) != 0:
                raise OSError("no NVML handle")

    def sample(self):
        c = self.c
        sm, mx, why = c.c_uint(), c.c_uint(), c.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(sm)) != 0 or
                self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, c.byref(mx)) != 0 or
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons(self.h, c.byref(why)) != 0):
            raise OSError("NVML read failed")
        return sm.value, mx.value, why.value


class ClockSampler:
    """SM clock and clock-event (throttle) sampling during the timed region:
    NVML read every 10 ms from a thread (reads only), else nvidia-smi at its
    shortest period."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.thread = None
        self.samples = []  # (sm_mhz, max_mhz, reasons bitmask)

    def __enter__(self):
        import threading
        try:
            nv = _Nvml(self.index)
            self.samples.append(nv.sample())
            self.stop = threading.Event()

            def run():
                while not self.stop.wait(0.01):
                    try:
                        self.samples.append(nv.sample())
                    except OSError:
                        break
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return self
        except OSError:
            self.thread = None
            self.samples = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=2)
            return
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if self.samples:
            sm = [float(a) for a, _, _ in self.samples]
            reasons = sorted({n for _, _, r in self.samples for n, b in self.REASONS.items() if r & b})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(max(b for _, b, _ in self.samples)),
                    "reasons": reasons, "samples": len(self.samples), "source": "nvml, 10 ms"}
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi"}


def oracle_rate(wl, stride: int, threads: int, rays=None):
    """ray-steps/s of the FP64 oracle on a strided sample of the workload;
    also returns the sample's indices and oracle results."""
    import oracle
    rays = wl.rays if rays is None else rays
    idx = np.arange(0, rays.n, stride)
    sub = rays.subset(idx)
    t0 = time.perf_counter()
    r = oracle.trace(wl.medium, sub.origins, sub.dirs, wl.dopl, wl.max_steps, threads=threads)
    dt = time.perf_counter() - t0
    return float(r["steps"].sum()) / dt, len(idx), dt, idx, r


def serve_load(ctx, dev_index: int, rates, jobs_per_rate: int, seed: int = 7):
    """Poisson arrivals of trace jobs into one grin_serve server; per rate:
    p50/p99 latency (submit to results in host memory) and ray-steps/s.
    Jobs draw a medium from {Luneburg lens, freeform block, blob grids at
    64^3, 128^3, 256^3 and 512^3, the 128^3 grid in 32 shells}, a ray count
    log-uniform in [1e3, 1e6] and dL0 from {0.02, 0.01, 0.005} (mm, or units
    of the lens radius); every medium stays resident on the device."""
    import torch
    from paper_2606_22655_b300 import tracer
    from paper_2606_22655_b300 import workloads as W
    names = ["luneburg", "freeform_block", "grid_64", "grid_128", "grid_256", "grid_512", "layered_128"]
    pool = [W.luneburg_workload(), W.freeform_workload(1 << 20)]
    pool += [W.blob_workload(n_rays=1 << 20, res=r) for r in (64, 128, 256, 512)]
    pool += [W.blob_workload(n_rays=1 << 20, res=128, n_levels=32)]
    dopls = [0.02, 0.01, 0.005]
    media = [tracer.Medium(ctx, wl.medium) for wl in pool]
    rays = [tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32, pin=True)
            for wl in pool]
    n_out = 48
    outs = [tracer.empty_result(1 << 20, "cpu") for _ in range(n_out)]
    srv = tracer.Server(ctx, 16 << 30)
    results = []
    for ri, rate in enumerate(rates):
        rng = np.random.default_rng(seed + ri)
        kinds = rng.integers(0, len(pool), jobs_per_rate)
        job_dopl = rng.choice(dopls, jobs_per_rate)
        counts = np.exp(rng.uniform(np.log(1e3), np.log(1e6), jobs_per_rate)).astype(np.int64)
        counts = np.minimum(counts, [pool[k].rays.n for k in kinds])
        gaps = rng.exponential(1.0 / rate, jobs_per_rate)
        t0 = time.perf_counter()
        inflight, lat, steps, qr = [], [], 0.0, []
        next_t = t0
        free = list(range(n_out))
        for j in range(jobs_per_rate):
            next_t += gaps[j]
            while True:
                now = time.perf_counter()
                done = [x for x in inflight if srv.poll(x[0])[0] >= 2]
                for x in done:
                    st, l = srv.poll(x[0])
                    lat.append(l)
                    steps += float(outs[x[1]]["steps"][: x[2]].sum())
                    qr.append(srv.timing(x[0]))
                    free.append(x[1])
                    inflight.remove(x)
                if now >= next_t and free:
                    break
                time.sleep(0.0002)
            k = int(kinds[j]); n = int(counts[j]); ob = free.pop()
            sub = tracer.RayBatch(*[t[:n] for t in rays[k].tensors()])
            out = {key: v[:n] for key, v in outs[ob].items()}
            jid, _ = srv.submit(media[k], sub, float(job_dopl[j]), 20000, out=out)
            inflight.append((jid, ob, n))
        for x in inflight:
            srv.wait(x[0], 600)
            st, l = srv.poll(x[0])
            lat.append(l)
            steps += float(outs[x[1]]["steps"][: x[2]].sum())
            qr.append(srv.timing(x[0]))
        wall = time.perf_counter() - t0
        lat = np.array(lat)
        qr = np.array(qr)
        pc = lambda v, q: 1e3 * float(np.percentile(v, q))
        results.append({"rate": rate, "jobs": jobs_per_rate, "p50_ms": pc(lat, 50), "p99_ms": pc(lat, 99),
                        "queue_p50_ms": pc(qr[:, 0], 50), "queue_p99_ms": pc(qr[:, 0], 99),
                        "run_p50_ms": pc(qr[:, 1], 50), "run_p99_ms": pc(qr[:, 1], 99),
                        "ray_steps_per_s": steps / wall, "wall_s": wall})
    st = srv.stats()
    srv.close()
    return {"sweep": results, "media": names, "dL0": dopls, "ray_count": "log-uniform [1e3, 1e6]",
            "arrivals": "Poisson", "latency": "submit to results in host memory = queue (to admission) + run",
            "ticks": st["ticks"], "failed": st["failed"]}


def adjoint_timing(ctx, dev, n_rays=1 << 18):
    """One gradient of the image-plane design loss (16 target spots on
    z = 30 mm) with respect to the 128^3 blob grid: 262,144 collimated rays
    (or n_rays, to profile a smaller case), dL0 = 0.02 mm (up to 2000 steps);
    the FP64 forward sweep with checkpoints plus the backward sweep.  The
    checkpoint interval is the library's choice for half the free device
    memory (every step stored when that fits: 55 GB here); the same gradient
    with a checkpoint every 64 steps (segments recomputed) is timed beside
    it, and so is the gradient with respect to the freeform block's 35
    coefficients on as many point-source rays."""
    import torch
    from paper_2606_22655_b300 import tracer
    from paper_2606_22655_b300 import workloads as W
    wl = W.blob_workload(n_rays=n_rays, res=128)
    med = tracer.Medium(ctx, wl.medium)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float64)
    n = rays.count
    n_par = wl.medium.grid.size
    g = {k: torch.randn(n, dtype=torch.float64, device=dev) * 1e-3 for k in tracer.OUT_FIELDS}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(k):
        tracer.trace_adjoint(ctx, med, rays, 0.02, 2000, g, n_par, k)  # warm-up
        torch.cuda.synchronize(dev)
        e0.record()
        out, grad = tracer.trace_adjoint(ctx, med, rays, 0.02, 2000, g, n_par, k)
        e1.record()
        torch.cuda.synchronize(dev)
        return out, grad, e0.elapsed_time(e1) / 1e3

    out, g64, t64 = timed(64)
    steps = float(out["steps"].sum())
    k = tracer.adjoint_interval(med, n, 0.02, 2000)
    if k != 64:
        _, gk, t = timed(k)
    else:
        gk, t = g64, t64
    same = bool(torch.allclose(gk, g64, rtol=1e-12, atol=1e-15 * float(g64.abs().max())))
    # one design iteration through the autograd function (grin_trace_adjoint
    # _forward in forward, _backward in backward: the rays traced forward
    # once), at the chosen interval and at K = 64, against a plain FP64
    # trace for the loss followed by the one-call adjoint at K = 64
    targets = torch.tensor(W.design_targets(n) + 10.0, device=dev)
    theta = torch.tensor(wl.medium.grid.astype(np.float64).ravel(), device=dev, requires_grad=True)

    def design_step(kk):
        theta.grad = None
        P, d, opl, ex = tracer.traced_exit(theta, ctx, wl.medium, rays, 0.02, 2000, kk)
        tracer.image_plane_loss(P, d, ex, targets, 30.0).backward()

    def two_trace_step():
        tracer.trace(ctx, med, rays, 0.02, 2000, "fp64")
        tracer.trace_adjoint(ctx, med, rays, 0.02, 2000, g, n_par, 64)

    design = {}
    for name, fn in (("autograd_step_seconds", lambda: design_step(0)),
                     ("autograd_step_k64_seconds", lambda: design_step(64)),
                     ("trace_then_adjoint_k64_seconds", two_trace_step)):
        fn()
        torch.cuda.synchronize(dev)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize(dev)
        design[name] = e0.elapsed_time(e1) / 1e3
    # the same loss with respect to the freeform block's 35 coefficients (the
    # point-source bundle, dL0 = 0.02 mm so that every ray leaves within 2000
    # steps), at the interval chosen by free memory
    fm = W.freeform_block_medium()
    fr = W.point_source_rays(n, W.BASE_SEED + 4)
    fmed = tracer.Medium(ctx, fm)
    frays = tracer.RayBatch.from_numpy(fr.origins, fr.dirs, device=dev, dtype=torch.float64)
    fk = tracer.adjoint_interval(fmed, n, 0.02, 2000)
    tracer.trace_adjoint(ctx, fmed, frays, 0.02, 2000, g, len(fm.coeffs), fk)  # warm-up
    torch.cuda.synchronize(dev)
    e0.record()
    fout, _ = tracer.trace_adjoint(ctx, fmed, frays, 0.02, 2000, g, len(fm.coeffs), fk)
    e1.record()
    torch.cuda.synchronize(dev)
    tf = e0.elapsed_time(e1) / 1e3
    fsteps = float(fout["steps"].sum())
    fmed.close()
    coefficients = {"workload": f"freeform block adjoint, 35 coefficients, {n} rays, dL0 0.02 mm",
                    "checkpoint_every": fk, "seconds": tf, "forward_ray_steps": fsteps,
                    "ray_steps_per_s_fwd_plus_bwd": fsteps / tf}
    return {"workload": f"grid_128 adjoint, {n} rays, dL0 0.02 mm, checkpoint interval by free memory",
            "checkpoint_every": k,
            "workspace_gb": tracer.adjoint_workspace_bytes(med, n, 0.02, 2000, k) / 1e9,
            "seconds": t, "forward_ray_steps": steps, "ray_steps_per_s_fwd_plus_bwd": steps / t,
            "precision": "fp64", "gradient_params": int(n_par),
            "recomputed_k64": {"seconds": t64, "ray_steps_per_s_fwd_plus_bwd": steps / t64,
                               "workspace_gb": tracer.adjoint_workspace_bytes(med, n, 0.02, 2000, 64) / 1e9,
                               "gradient_equals": same},
            "design_iteration": design, "coefficients": coefficients}


def media_rates(ctx, dev):
    """One mixed-precision trace per medium kind (after a warm-up trace):
    ray-steps/s of each, as grin_trace runs it (claim order included)."""
    import torch
    from paper_2606_22655_b300 import tracer
    from paper_2606_22655_b300 import workloads as W
    from paper_2606_22655_b300 import n2p_design
    fan = n2p_design.fan(1 << 16, 0.3)
    cases = [("luneburg_4096", W.luneburg_workload()),
             ("corrector_lens_262144", W.corrector_workload(1 << 18)),
             ("spherical_freeform_262144", W.spherical_workload(1 << 18)),
             ("n2p_lens_65536", W.Workload("n2p", W.n2p_lens_medium(0.770, 4.462, 0.3), fan, 1e-4, 400000, 1.0)),
             ("grid_256_1048576", W.blob_workload(n_rays=1 << 20, res=256)),
             ("layered_256_1048576", W.blob_workload(n_rays=1 << 20, res=256, n_levels=32)),
             ("layered_crossings_256_1048576", W.blob_workload(n_rays=1 << 20, res=256, n_levels=32))]
    res = {}
    for name, wl in cases:
        lr = "crossings" in name  # shells with their crossings solved
        med = tracer.Medium(ctx, wl.medium)
        rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float32)
        out = tracer.empty_result(rays.count, dev)
        tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, "mixed", out=out, level_root=lr)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, "mixed", out=out, level_root=lr)
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 1e3
        res[name] = {"ms": 1e3 * t, "ray_steps_per_s": float(out["steps"].sum()) / t}
        med.close()
    return res


def design_sweep(ctx):
    """The N2P lens design of Sec. VI (L = 0.3 R, F = 2 R): successive
    refinement of (beta, gamma), 8 rounds of 81 concurrent 10-ray jobs on the
    trace server."""
    from paper_2606_22655_b300 import n2p_design
    res = n2p_design.design(ctx, L=0.3, rounds=8, grid=9, beta=(0.5, 1.2), gamma=(3.0, 6.0))
    return {"workload": "N2P lens L=0.3R F=2R, 10-ray fan, dL0 1e-4 R, 8 rounds x 81 jobs",
            "wall_s": res["wall_s"], "jobs": res["jobs"], "jobs_per_s": res["jobs"] / res["wall_s"],
            "round_wall_s": [h["wall_s"] for h in res["rounds"]],
            "beta": res["beta"], "gamma": res["gamma"], "rmse_lsa_over_R": res["rmse_lsa"]}


def measured_peaks(ctx, dev_index: int):
    """FP32 FMA rate of the CUDA cores and read bandwidth of an L2-resident
    64 MiB buffer, measured on this GPU by the library's probes (CUDA events
    around one launch each), with the SM clock sampled during the FMA run."""
    import ctypes
    from paper_2606_22655_b300 import _native as N
    lib = ctx.lib
    flops, secs = ctypes.c_double(), ctypes.c_double()
    with ClockSampler(dev_index) as clk:
        N.check("grin_probe_fp32_fma", lib.grin_probe_fp32_fma(6_000_000, ctypes.byref(flops), ctypes.byref(secs)))
    l2 = ctypes.c_double()
    N.check("grin_probe_l2_read", lib.grin_probe_l2_read(64 << 20, 40, ctypes.byref(l2)))
    c = clk.summary()
    return {"fp32_tflops": flops.value / 1e12, "fma_seconds": secs.value, "fma_sm_mhz": c["sm_mhz"],
            "fp32_tflops_derived": FP32_PEAK_TFLOPS, "l2_read_gbs": l2.value / 1e9,
            "how": "grin_probe_fp32_fma (8 FMA chains a thread, 8 x 256-thread blocks an SM) and "
                   "grin_probe_l2_read (64 MiB, 40 reads), CUDA events"}


def grid_flops_per_step() -> int:
    """FP32 FLOPs of one ray-step on a gridded medium (FMA = 2): the
    Catmull-Rom weights and derivatives of the three axes (3 x 10 FMA), the
    tap-cache sums of value and gradient (16 rows x 8, 16 x 3, 4 x 4 FMA),
    the compensated cell fraction (3 x 9) and the rest of a refracting step."""
    return 2 * (30 + 16 * 8 + 16 * 3 + 4 * 4) + 27 + STEP_FIXED_FLOPS


def timed_trace(ctx, med, rays, wl, precision, out, reps: int = 1):
    """Mean event time of reps grin_trace calls after one warm-up call."""
    import torch
    from paper_2606_22655_b300 import tracer
    tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, precision, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, precision, out=out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def config_rates(ctx, dev, peaks):
    """The Luneburg lens (4,096 rays): the mixed tracer against the plain
    and fast FP64 tracers.  The 256^3 blob grid and its 32 shells
    (4,194,304 rays): the mixed tracer's rate, its FP32 FLOP rate
    against the measured FMA peak, and the cache traffic of its tap cache:
    256 B of shared memory a ray-step, and from L2 the 256 B of a refill on
    the 4.8 % of ray-steps that enter a new cell (ncu, 262,144 rays)."""
    import torch
    from paper_2606_22655_b300 import tracer
    from paper_2606_22655_b300 import workloads as W
    res = {}
    wl = W.luneburg_workload()
    med = tracer.Medium(ctx, wl.medium)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float32)
    out = tracer.empty_result(rays.count, dev)
    rate = {}
    for prec in ("mixed", "fp64", "fp64-fast"):
        t = timed_trace(ctx, med, rays, wl, prec, out, reps=5 if prec == "mixed" else 1)
        rate[prec] = float(out["steps"].sum()) / t
    res["luneburg_4096"] = {"mixed": rate["mixed"], "fp64": rate["fp64"], "fp64_fast": rate["fp64-fast"],
                            "speedup_vs_fp64": rate["mixed"] / rate["fp64"],
                            "speedup_vs_fp64_fast": rate["mixed"] / rate["fp64-fast"]}
    med.close()
    for levels in (0, 32):
        wl = W.blob_workload(n_rays=1 << 22, res=256, n_levels=levels)
        med = tracer.Medium(ctx, wl.medium)
        rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float32)
        out = tracer.empty_result(rays.count, dev)
        t = timed_trace(ctx, med, rays, wl, "mixed", out)
        r = float(out["steps"].sum()) / t
        entry = {"ray_steps_per_s": r, "ms": 1e3 * t}
        if not levels:
            tflops = grid_flops_per_step() * r / 1e12
            entry.update({"flops_per_ray_step": grid_flops_per_step(), "achieved_tflops": tflops,
                          "fp32_frac_of_measured": tflops / peaks["fp32_tflops"],
                          "shared_bytes_per_ray_step": 256, "l2_bytes_per_ray_step": 0.048 * 256,
                          "l2_gbs": 0.048 * 256 * r / 1e9,
                          "l2_frac_of_measured": 0.048 * 256 * r / 1e9 / peaks["l2_read_gbs"]})
        res[("grid" if not levels else "layered") + "_256_4194304"] = entry
        med.close()
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2606_22655_b300 import workloads as W
    wl = W.freeform_workload(N_RAYS)
    threads = os.cpu_count() or 1
    stride = args.ref_stride
    for _ in range(args.warmup):
        oracle_rate(wl, stride * 4, threads)
    t0 = time.perf_counter()
    total_steps = 0.0
    for k in range(args.steps):
        rate, n, dt, _, _ = oracle_rate(wl, stride, threads)
        total_steps += rate * dt
    wall = time.perf_counter() - t0
    value = total_steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "rays_per_step": n, "sample_stride": stride,
                                        "dopl_mm": wl.dopl, "max_steps": wl.max_steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"every {stride}th ray of the {wl.rays.n}-ray batch ({n} rays) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2606_22655_b300 import tracer
    from paper_2606_22655_b300 import workloads as W
    from tests.compare import compare, fp32_flags

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = tracer.Context(local)
    if args.workload == "freeform":
        wl = W.freeform_workload(args.rays, ray_seed=rank_ray_seed(rank))
    elif args.workload == "luneburg":
        wl = W.luneburg_workload()
    else:
        wl = W.blob_workload(n_rays=args.rays, res=256, n_levels=32 if args.workload == "layered" else 0)
    med = tracer.Medium(ctx, wl.medium)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float32)
    out = tracer.empty_result(rays.count, dev)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    level_root = bool(args.level_root and wl.medium.n_levels)

    def step():
        tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, "mixed", stream=stream, out=out,
                     level_root=level_root)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            step()
    torch.cuda.synchronize(dev)
    steps_per_trace = float(out["steps"].sum().item())

    # timed region: K steps, L2 flushed before each (outside the kernel events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            r0.record(stream)
            for k in range(args.steps):
                flush.zero_()
                ev[k][0].record(stream)
                step()
                launches += ctx.last_launches()
                ev[k][1].record(stream)
            r1.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
    region_s = r0.elapsed_time(r1) / 1e3
    kern_s = [a.elapsed_time(b) / 1e3 for a, b in ev]
    region_s, value = aggregate(region_s, steps_per_trace, args.steps, ws, dev)
    mean_kern = sum(kern_s) / len(kern_s)

    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "workload": wl.name + ("_crossings" if level_root else ""),
                              "value": value, "unit": UNIT,
                              "kernel_ms": 1e3 * mean_kern, "gpu_launches": launches}), flush=True)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # CPU baseline (the FP64 oracle on every 16th ray); its decision margins
    # also flag the ill-conditioned rays for the precision gate
    cpu = None
    orc_idx = orc_res = None
    if ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rays32 = W.Rays(wl.rays.origins.astype(np.float32).astype(np.float64),
                        wl.rays.dirs.astype(np.float32).astype(np.float64))
        rate, n, dt, orc_idx, orc_res = oracle_rate(wl, 16, threads, rays32)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"every 16th ray of the {wl.rays.n}-ray batch ({n} rays, {dt:.1f} s)"}
        # the same oracle on one core, on every 256th ray
        rate1, n1, dt1, _, _ = oracle_rate(wl, 256, 1, rays32)
        cpu["single_core"] = {"value": rate1, "cores": 1,
                              "sample": f"every 256th ray ({n1} rays, {dt1:.1f} s)"}

    # precision gate: this run's outputs against the plain FP64 GPU tracer
    res32 = tracer.to_numpy(out)
    rays64 = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device=dev, dtype=torch.float32)
    out64 = tracer.empty_result(rays64.count, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        tracer.trace(ctx, med, rays64, wl.dopl, wl.max_steps, "fp64", stream=stream, out=out64)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    fp64_s = e0.elapsed_time(e1) / 1e3
    out64f = tracer.empty_result(rays64.count, dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        tracer.trace(ctx, med, rays64, wl.dopl, wl.max_steps, "fp64-fast", stream=stream, out=out64f)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    fast_s = e0.elapsed_time(e1) / 1e3
    res64 = tracer.to_numpy(out64)
    gate = compare(res32, res64, wl.l_ref)
    gate_s = None
    if orc_res is not None:
        sub = lambda g: {k: v[orc_idx] for k, v in g.items()}
        r32s = rays32.subset(orc_idx)
        gate_s = compare(sub(res32), orc_res, wl.l_ref,
                         fp32_flags(orc_res, wl.medium, r32s.origins, r32s.dirs, wl.dopl, wl.max_steps, wl.l_ref))

    # end to end through the host-buffer entry point (pinned host memory)
    hrays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cpu", dtype=torch.float32, pin=True)
    hout = tracer.empty_result(hrays.count, "cpu")
    tracer.trace_host(ctx, med, hrays, wl.dopl, wl.max_steps, "mixed", stream=stream, out=hout)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_steps = 0.0
    for _ in range(args.steps):
        tracer.trace_host(ctx, med, hrays, wl.dopl, wl.max_steps, "mixed", stream=stream, out=hout)
        e2e_steps += float(hout["steps"].sum().item())
    e2e_s = time.perf_counter() - t0
    h2d = 6 * 4 * hrays.count
    d2h = (7 * 8 + 4 * 4) * hrays.count

    design = None
    media = None
    if ws == 1 and not args.no_serve:
        design = design_sweep(ctx)
        media = media_rates(ctx, dev)
    adjoint = None
    if ws == 1 and not args.no_serve:
        adjoint = adjoint_timing(ctx, dev)
    serve = None
    if ws == 1 and not args.no_serve:
        serve = serve_load(ctx, local, rates=[10.0, 40.0, 160.0, 640.0], jobs_per_rate=args.serve_jobs)

    if rank != 0:
        return 0
    peaks = measured_peaks(ctx, local)
    configs = config_rates(ctx, dev, peaks) if not args.no_serve else None
    flops_launch = flops_per_step(4) * steps_per_trace
    achieved = flops_launch / mean_kern / 1e12
    fp64_rate = float(res64["steps"].sum()) / fp64_s
    fast_rate = float(res64["steps"].sum()) / fast_s
    gate_pass = gate_s is not None and gate_s["int_mismatch_unflagged"] == 0 and \
        max(gate_s["pos"], gate_s["dir"], gate_s["opl"]) <= 2e-5
    # the keys a reader needs first (a log tail may keep only the start of
    # this long line): the metric, the precision gate, the speed-up over the
    # FP64 tracers, the workload and the roofline
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * region_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "precision_gate": None if gate_s is None else {
            "pass": gate_pass, "tolerance": 2e-5, "vs": "FP64 oracle on the same float32 rays",
            "rays": gate_s["n"], "flagged": gate_s["n_flagged"], "flagged_frac": gate_s["n_flagged"] / gate_s["n"],
            "int_mismatch_unflagged": gate_s["int_mismatch_unflagged"],
            "max_rel_pos": gate_s["pos"], "max_dir": gate_s["dir"], "max_rel_opl": gate_s["opl"],
            "p99_rel_pos": gate_s["pos_p99"], "p99_dir": gate_s["dir_p99"],
            "sample": "every 16th ray of the batch",
            "flag_rule": "oracle margin inside the FP32 drift (surface < 2^-20 S steps, level < 1e-5, "
                         "critical or |N.I| < 2^-19) or oracle unstable under the trapezoid index "
                         "difference and a 2e-6 normal perturbation (tests/compare.py)"},
        "speedup_vs_fp64": value / ws / fp64_rate, "speedup_vs_fp64_fast": value / ws / fast_rate,
        "config": {"workload": wl.name, "rays": wl.rays.n, "medium": "degree-4 polynomial, 35 monomials",
                   "dopl_mm": wl.dopl, "max_steps": wl.max_steps, "precision": "fp32-mixed",
                   "ray_steps_per_step": steps_per_trace,
                   "l2": "256 MiB buffer zeroed before every step, inside the timed region"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / peaks["fp32_tflops"],
                     "traffic": profiled_traffic() if args.rays == N_RAYS and args.workload == "freeform" else None,
                     "kernel": KERNEL, "kernel_ms": 1e3 * mean_kern,
                     "flops_per_ray_step": flops_per_step(4),
                     "peak_source": "measured: FP32 FMA probe on this GPU (grin_probe_fp32_fma)",
                     "peak_derived": FP32_PEAK_TFLOPS, "frac_of_derived": achieved / FP32_PEAK_TFLOPS,
                     "fp32_issue": fp32_issue(steps_per_trace / mean_kern)
                     if args.rays == N_RAYS and args.workload == "freeform" else None},
        "configs": configs,
        "e2e": {"value": e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "measured_peaks": peaks,
        "cpu_baseline": cpu,
        "all_rays_vs_fp64": {"rays": gate["n"], "int_mismatch": gate["int_mismatch_unflagged"],
                             "p99_rel_pos": gate["pos_p99"], "p99_dir": gate["dir_p99"],
                             "max_rel_pos": gate["pos"], "max_dir": gate["dir"],
                             "fp64_ray_steps_per_s": fp64_rate, "fp64_fast_ray_steps_per_s": fast_rate},
        "serve": serve,
        "adjoint": adjoint,
        "design_sweep": design,
        "media_rates": media,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-stride", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-latency sweep")
    ap.add_argument("--serve-jobs", type=int, default=500, help="jobs per arrival rate in the sweep")
    ap.add_argument("--rays", type=int, default=N_RAYS,
                    help="ray count (profiling of a smaller case; the line then names it)")
    ap.add_argument("--workload", choices=["freeform", "grid", "layered", "luneburg"], default="freeform",
                    help="freeform (the benchmark), or another medium for profiling")
    ap.add_argument("--profile-only", action="store_true",
                    help="timed steps only: no precision gate, e2e or CPU baseline")
    ap.add_argument("--level-root", action="store_true",
                    help="with --workload layered: the shells with their crossings solved")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="RAYS",
                    help="only the adjoint timing, on RAYS rays (to profile its kernels)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint_only:
        return run_adjoint_only(args.adjoint_only)
    return run_ours(args)


def run_adjoint_only(n_rays: int) -> int:
    """The adjoint timing alone (one warm-up call, one timed call) on one GPU."""
    import torch
    from paper_2606_22655_b300 import tracer
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = tracer.Context(0)
    print(json.dumps(dict(adjoint_only=True, **adjoint_timing(ctx, dev, n_rays))), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
