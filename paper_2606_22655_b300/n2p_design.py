"""Design of the cylindrical N2P-GRIN lens (Sec. VI) on the GPU.

The lens index n = [1 + ((R^2 - (rho/2)^2) / F^2)^beta]^gamma (z in [-L, 0],
rho <= R) has two free parameters.  They are chosen to bring a fan of rays
parallel to the axis to one focus at distance F behind the exit face: the
figure of merit is the RMSE of the longitudinal spherical aberration,
LSA_i = F - z_Int,i, where ray i crosses the axis at z_Int,i.  The search is
the successive refinement the paper describes: sample a grid of (beta, gamma),
keep the best point, shrink the interval around it, repeat.

Every grid point is one small trace job (10 rays) on the continuous-batching
server (grin_serve_*), so a whole refinement round runs as one batch of
concurrent jobs on the GPU, each with its own medium.  The host only turns
each job's exit states into an RMSE and picks the next interval.
"""
from __future__ import annotations

import time
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from . import _native as N
from . import tracer
from . import workloads as W

EXIT_FACE = 2  # the z1 end of the cylinder, the lens's exit face


def fan(n: int = 10, L: float = 0.3, R: float = 1.0) -> W.Rays:
    """n rays parallel to the axis in the y-z plane at heights 0.995 R k / n,
    k = 1..n (the paper's fan: uniform in y, y = 0 excluded, largest height
    0.995 R), launched half a radius before the entrance face z = -L."""
    y = 0.995 * R * np.arange(1, n + 1) / n
    o = np.stack([np.zeros(n), y, np.full(n, -L - 0.5 * R)], 1)
    return W.Rays(o, np.tile([0.0, 0.0, 1.0], (n, 1)))


def rmse_lsa(P: np.ndarray, d: np.ndarray, exit_id: np.ndarray, F: float) -> float:
    """RMSE of F - z_Int over the fan; infinite when a ray does not leave
    through the exit face or does not head back towards the axis."""
    if not (exit_id == EXIT_FACE).all() or not (P[:, 1] * d[:, 1] < 0).all():
        return float("inf")
    z_int = P[:, 2] - P[:, 1] * d[:, 2] / d[:, 1]
    return float(np.sqrt(np.mean((F - z_int) ** 2)))


def design(ctx: tracer.Context, L: float, F: float = 2.0, R: float = 1.0, n_rays: int = 10,
           dopl: float = 1e-4, grid: int = 9, rounds: int = 8,
           beta: Tuple[float, float] = (0.2, 4.0), gamma: Tuple[float, float] = (1.0, 30.0),
           max_steps: int = 400000, server: Optional[tracer.Server] = None) -> Dict:
    """Successive refinement of (beta, gamma) for thickness L (all lengths in
    units of R, dL0 = dopl R).  Each round traces grid x grid lenses, keeps
    the best and narrows both intervals to +-2 grid spacings around it.
    Returns the best point, its RMSE and per-round timings."""
    srv = server if server is not None else tracer.Server(ctx, 1 << 28)
    rays = fan(n_rays, L, R)
    hrays = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cpu", dtype=torch.float64)
    lo_b, hi_b = beta
    lo_g, hi_g = gamma
    best = (float("inf"), None)
    history = []
    t_all = time.perf_counter()
    try:
        for r in range(rounds):
            bs, gs = np.linspace(lo_b, hi_b, grid), np.linspace(lo_g, hi_g, grid)
            t0 = time.perf_counter()
            jobs = []
            for b in bs:
                for g in gs:
                    med = tracer.Medium(ctx, W.n2p_lens_medium(float(b), float(g), L, R, F))
                    jid, out = srv.submit(med, hrays, dopl * R, max_steps)
                    jobs.append((float(b), float(g), med, jid, out))
            errs = np.full(len(jobs), np.inf)
            for k, (b, g, med, jid, out) in enumerate(jobs):
                if srv.wait(jid, 300.0) == N.JOB_DONE:
                    res = tracer.to_numpy(out)
                    errs[k] = rmse_lsa(res["P"], res["d"], res["exit_id"], F)
                med.close()
            wall = time.perf_counter() - t0
            k = int(np.argmin(errs))
            b, g = jobs[k][0], jobs[k][1]
            if errs[k] < best[0]:
                best = (float(errs[k]), (b, g))
            history.append({"round": r, "jobs": len(jobs), "wall_s": wall, "beta": b, "gamma": g,
                            "rmse": float(errs[k]), "finite": int(np.isfinite(errs).sum())})
            db, dg = 2 * (hi_b - lo_b) / (grid - 1), 2 * (hi_g - lo_g) / (grid - 1)
            lo_b, hi_b = max(b - db, 1e-3), b + db
            lo_g, hi_g = max(g - dg, 1e-3), g + dg
    finally:
        if server is None:
            srv.close()
    return {"L": L, "F": F, "R": R, "beta": best[1][0] if best[1] else None,
            "gamma": best[1][1] if best[1] else None, "rmse_lsa": best[0],
            "rounds": history, "jobs": sum(h["jobs"] for h in history),
            "wall_s": time.perf_counter() - t_all}
