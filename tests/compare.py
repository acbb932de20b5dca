"""Element-by-element comparison of two traces of the same rays."""
import numpy as np

INT_KEYS = ("exit_id", "steps", "tir_internal", "tir_boundary")


def flagged(margins: np.ndarray, tau: float, tau_geom: float = None) -> np.ndarray:
    """Rays whose oracle decision margins fall below a threshold: distance of
    N.I from its critical value and min |N.I| below tau; distance of a step
    end to the surface (in steps) and of the field to a level threshold (in
    levels) below tau_geom (default tau)."""
    tg = tau if tau_geom is None else tau_geom
    return (margins[:, 0] < tau) | (margins[:, 1] < tau) | (margins[:, 2] < tg) | (margins[:, 3] < tg)


# The FP32 path's error model.  Its arithmetic errors per step are FP32
# roundings: a relative 1e-7 or so on the normal N (measured on the 256^3 blob
# grid with the compensated cell fraction: median 5e-8, p99 2e-7), and the
# rounding of the point, carried as a hi + lo pair.  Over S steps they drift
# the point by up to about 1e-6 S steps (measured: 3e-3 of a step after 6,000
# steps through the blob grid, 4e-3 after 3,000 through the freeform block at
# the worst ray) and N.I by up to about 2e-6.  Its one approximation is the
# index difference n_i - n_{i-1} of a refraction, which it takes by the
# trapezoid rule on grad n along the step (exact to third order in the step)
# instead of from two rounded point values.  An integer outcome is decided by
# the sign of a margin (the surface, a shell boundary, N.I, or D at the
# critical angle), so a ray is excused when its oracle margin is inside that
# drift.  Near turning points of n, Eq. 9 is steep in N.I and the exit state
# is sensitive to any small change of the map; those rays are found by
# running the oracle again with the FP32 path's approximation and twice its
# normal error.
FP32_STEP_DRIFT = 2.0 ** -20   # surface margin threshold, in steps per step taken
FP32_NI = 2.0 ** -19           # critical and tangent margin threshold (N.I)
FP32_LEVEL = 1e-5              # level margin threshold, in levels
FP32_PROBE_PERTURB = 2e-6      # relative perturbation of N in the conditioning probe
FP32_PROBE_TOL = 1e-5          # probe change (half the 2e-5 gate) that flags a ray
FP32_PROBE_SEEDS = (1, 2, 3)


def fp32_flags(o: dict, medium, origins, dirs, dopl: float, max_steps: int, l_ref: float,
               flags: int = 0) -> np.ndarray:
    """Rays the FP32 path is excused on, from the oracle result o of the same
    rays: a margin inside the path's drift (surface: below 2^-20 S steps for a
    ray of S steps; level: below 1e-5; critical distance or |N.I|: below
    2^-19), or a ray whose oracle trace changes an integer outcome or moves by
    more than 1e-5 when traced with the trapezoid index difference and a
    2e-6 relative perturbation of every normal (three seeds).  flags are the
    oracle trace flags o was traced with."""
    import oracle  # test infrastructure

    m = o["margins"]
    S = np.maximum(np.asarray(o["steps"], float), 1.0)
    f = (m[:, 2] < FP32_STEP_DRIFT * S) | (m[:, 3] < FP32_LEVEL) | (m[:, 0] < FP32_NI) | (m[:, 1] < FP32_NI)
    for seed in FP32_PROBE_SEEDS:
        p = oracle.trace(medium, origins, dirs, dopl, max_steps, flags=flags, index_rule=1,
                         perturb=FP32_PROBE_PERTURB, seed=seed)
        same = np.ones(len(S), bool)
        for k in INT_KEYS:
            same &= np.asarray(p[k]) == np.asarray(o[k])
        e = np.maximum(np.linalg.norm(p["P"] - o["P"], axis=1) / l_ref, np.linalg.norm(p["d"] - o["d"], axis=1))
        f |= ~same | (e > FP32_PROBE_TOL)
    return f


def compare(a: dict, b: dict, l_ref: float, flags: np.ndarray = None):
    """Returns a report: integer-outcome mismatches (unflagged and flagged)
    and the largest position (relative to l_ref), direction and relative OPL
    differences over rays with identical integer outcomes."""
    n = len(a["exit_id"])
    if flags is None:
        flags = np.zeros(n, bool)
    same = np.ones(n, bool)
    for k in INT_KEYS:
        same &= np.asarray(a[k]) == np.asarray(b[k])
    rep = dict(n=n, int_mismatch_unflagged=int((~same & ~flags).sum()),
               int_mismatch_flagged=int((~same & flags).sum()), n_flagged=int(flags.sum()))
    m = same
    rep["n_compared"] = int((m & ~flags).sum())
    m = m & ~flags if (m & ~flags).any() else m
    if m.any():
        dp = np.linalg.norm(a["P"][m] - b["P"][m], axis=1) / l_ref
        dd = np.linalg.norm(a["d"][m] - b["d"][m], axis=1)
        do = np.abs(a["opl"][m] - b["opl"][m]) / np.maximum(np.abs(b["opl"][m]), 1e-300)
        rep.update(pos=float(dp.max()), dir=float(dd.max()), opl=float(do.max()),
                   pos_p99=float(np.percentile(dp, 99)), dir_p99=float(np.percentile(dd, 99)))
    else:
        rep.update(pos=0.0, dir=0.0, opl=0.0, pos_p99=0.0, dir_p99=0.0)
    return rep
