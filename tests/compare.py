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


# FP32 flag thresholds: FP32 carries N.I and the direction to ~1e-7 per step,
# a few 1e-7 after thousands of steps, and positions to ~1e-6 of a step
TAU32 = 1e-6
TAU32_GEOM = 1e-5


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
