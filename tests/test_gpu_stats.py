"""grin_trace_stats_compute: the device totals of a trace's results against
the same totals taken in numpy from the results themselves."""
import numpy as np
import pytest
import torch

from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tracer.Context(0)
    yield c
    c.close()


def numpy_totals(res, margin_min=None):
    ex = res["exit_id"]
    t = {"rays": len(ex), "ray_steps": int(res["steps"].sum()),
         "exit_face": [int((ex == f).sum()) for f in range(6)],
         "exit_miss": int((ex == -1).sum()), "exit_entry_reflect": int((ex == -2).sum()),
         "exit_max_steps": int((ex == -3).sum()), "exit_invalid": int((ex == -4).sum()),
         "tir_internal": int(res["tir_internal"].sum()), "tir_boundary": int(res["tir_boundary"].sum())}
    if margin_min is not None:
        mg = np.asarray(res["margins"]).reshape(-1, 4)
        t["flagged"] = int((mg < np.asarray(margin_min)[None, :]).any(axis=1).sum())
    return t


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_stats_equal_the_results_totals(ctx, precision):
    wl = W.freeform_workload(1 << 14)
    # a few rays that miss the block and one with a zero direction
    o, d = wl.rays.origins.copy(), wl.rays.dirs.copy()
    d[:64] = [0.0, 0.0, -1.0]
    d[64] = 0.0
    med = tracer.Medium(ctx, wl.medium)
    rays = tracer.RayBatch.from_numpy(o, d, device="cuda", dtype=torch.float32)
    out = tracer.trace(ctx, med, rays, wl.dopl, 1500, precision, margins=True)
    mm = [1e-4, 1e-3, 0.5, 1e-2]
    st = tracer.trace_stats(ctx, out, mm)
    ref = numpy_totals(tracer.to_numpy(out), mm)
    for k, v in ref.items():
        assert st[k] == v, (k, st[k], v)
    assert st["exit_miss"] == 64 and st["exit_invalid"] >= 1 and st["exit_max_steps"] > 0
    assert st["elapsed_ms"] > 0.0
    # without thresholds no flag count; without margins in the results no thresholds
    assert tracer.trace_stats(ctx, out)["flagged"] == -1
    bare = {k: v for k, v in out.items() if k != "margin"}
    with pytest.raises(RuntimeError):
        tracer.trace_stats(ctx, bare, mm)
    med.close()


def test_stats_time_is_the_last_trace(ctx):
    """elapsed_ms is the device time of the context's last grin_trace: close
    to what CUDA events around the call on the same stream measure."""
    wl = W.freeform_workload(1 << 16)
    med = tracer.Medium(ctx, wl.medium)
    rays = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cuda", dtype=torch.float32)
    out = tracer.empty_result(rays.count, "cuda")
    tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, "mixed", out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tracer.trace(ctx, med, rays, wl.dopl, wl.max_steps, "mixed", out=out)
    e1.record()
    torch.cuda.synchronize()
    st = tracer.trace_stats(ctx, out)
    t = e0.elapsed_time(e1)
    assert 0.5 * t <= st["elapsed_ms"] <= t * 1.01 + 0.05, (st["elapsed_ms"], t)
    assert st["ray_steps"] == int(out["steps"].sum())
    med.close()
