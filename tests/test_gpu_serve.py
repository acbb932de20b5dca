"""The continuous-batching server (grin_serve_*), through the C ABI.

Each job's results must be bitwise those of grin_trace_host with the mixed
tracer, whether the job runs alone or among others of different media and
sizes, and match the FP64 oracle under the FP32 flag rule; two jobs run at
the same time on the device; admission respects the device arena;
cancellation and bounded waits leave the server usable.
"""
import numpy as np
import pytest
import torch

from paper_2606_22655_b300 import _native as N
from paper_2606_22655_b300 import tracer
from paper_2606_22655_b300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("px", "py", "pz", "dx", "dy", "dz", "opl", "exit_id", "steps", "tir_internal", "tir_boundary")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tracer.Context(0)
    yield c
    c.close()


def host_rays(wl, n=None, dtype=torch.float32):
    o, d = wl.rays.origins, wl.rays.dirs
    if n is not None:
        o, d = o[:n], d[:n]
    return tracer.RayBatch.from_numpy(o, d, device="cpu", dtype=dtype)


def same(a, b):
    for k in KEYS:
        np.testing.assert_array_equal(a[k].numpy(), b[k].numpy(), err_msg=k)


@pytest.fixture(scope="module")
def jobs(ctx):
    wls = [W.freeform_workload(30000), W.luneburg_workload(), W.blob_workload(n_rays=3000, res=64),
           W.blob_workload(n_rays=2000, res=64, n_levels=32), W.freeform_workload(700, ray_seed=5)]
    out = []
    for wl in wls:
        med = tracer.Medium(ctx, wl.medium)
        rays = host_rays(wl)
        ref = tracer.trace_host(ctx, med, rays, wl.dopl, wl.max_steps, "mixed")
        out.append((wl, med, rays, ref))
    return out


def test_alone_equals_trace_host(ctx, jobs):
    srv = tracer.Server(ctx, 1 << 30)
    for wl, med, rays, ref in jobs:
        jid, res = srv.submit(med, rays, wl.dopl, wl.max_steps)
        assert srv.wait(jid, 120) == N.JOB_DONE
        same(res, ref)
    st = srv.stats()
    assert st["done"] == len(jobs) and st["failed"] == 0
    srv.close()


def test_mix_equals_alone(ctx, jobs):
    srv = tracer.Server(ctx, 1 << 30, step_quantum=256)
    handles = []
    for rep in range(2):
        for wl, med, rays, ref in jobs:
            handles.append((srv.submit(med, rays, wl.dopl, wl.max_steps), ref))
    for (jid, res), ref in handles:
        assert srv.wait(jid, 120) == N.JOB_DONE
        same(res, ref)
    st = srv.stats()
    assert st["done"] == 2 * len(jobs)
    total = sum(int(ref["steps"].sum()) for _, ref in handles)
    assert st["ray_steps"] == total
    srv.close()


def test_admission_by_arena(ctx, jobs):
    wl, med, rays, ref = jobs[0]
    # room for one 30000-ray job at a time (rays, results and slots)
    budget = 30000 * (24 + 72) + 30080 * 160 + 4096
    srv = tracer.Server(ctx, budget)
    ids = [srv.submit(med, rays, wl.dopl, wl.max_steps) for _ in range(3)]
    for jid, res in ids:
        assert srv.wait(jid, 120) == N.JOB_DONE
        same(res, ref)
    big = host_rays(W.freeform_workload(200000))
    with pytest.raises(N.GrinError) as e:
        srv.submit(med, big, wl.dopl, wl.max_steps)
    assert e.value.status == -6  # BUSY: could never fit
    srv.close()


def test_cancel_and_wait_timeout_leave_server_usable(ctx, jobs):
    srv = tracer.Server(ctx, 1 << 31, step_quantum=64)
    wl = W.freeform_workload(1 << 20)
    med = tracer.Medium(ctx, wl.medium)
    jid, _ = srv.submit(med, host_rays(wl), wl.dopl, wl.max_steps)
    assert srv.wait(jid, 0.001) == -5  # timed out, job still in flight
    srv.cancel(jid)
    assert srv.wait(jid, 60) == N.JOB_CANCELLED
    wl2, med2, rays2, ref2 = jobs[1]
    jid2, res2 = srv.submit(med2, rays2, wl2.dopl, wl2.max_steps)
    assert srv.wait(jid2, 60) == N.JOB_DONE
    same(res2, ref2)
    st = srv.stats()
    assert st["cancelled"] == 1 and st["arena_in_use"] == 0
    with pytest.raises(N.GrinError) as e:
        srv.poll(123456789)
    assert e.value.status == -7
    srv.close()


def test_submit_argument_errors(ctx, jobs):
    srv = tracer.Server(ctx, 1 << 28)
    wl, med, rays, ref = jobs[0]
    for dopl, ms in ((0.0, 10), (1e-3, -1)):
        with pytest.raises(N.GrinError) as e:
            srv.submit(med, rays, dopl, ms)
        assert e.value.status == -1
    other = tracer.Context(0)
    foreign = tracer.Medium(other, wl.medium)
    with pytest.raises(N.GrinError):
        srv.submit(foreign, rays, wl.dopl, wl.max_steps)
    empty = tracer.RayBatch(*[torch.empty(0) for _ in range(6)])
    jid, _ = srv.submit(med, empty, wl.dopl, wl.max_steps)
    assert srv.poll(jid)[0] == N.JOB_DONE
    nan = host_rays(wl, 64)
    nan.dx[:8] = float("nan")
    jid, res = srv.submit(med, nan, wl.dopl, wl.max_steps)
    assert srv.wait(jid, 60) == N.JOB_DONE
    assert (res["exit_id"][:8] == N.EXIT_INVALID).all() and (res["exit_id"][8:] >= 0).all()
    srv.close()
    foreign.close()
    other.close()


def test_submit_and_wait_from_several_threads(ctx, jobs):
    """The serve API is thread-safe: four host threads submit every job and
    wait on their own ids at once (ctypes releases the GIL inside each call,
    so the calls overlap in the library).  Every result is bitwise the
    direct trace's, and the server counts all twenty jobs."""
    import threading
    srv = tracer.Server(ctx, 1 << 30, step_quantum=256)
    failures = []

    def worker():
        try:
            mine = [(srv.submit(med, rays, wl.dopl, wl.max_steps), ref) for wl, med, rays, ref in jobs]
            for (jid, res), ref in mine:
                assert srv.wait(jid, 120) == N.JOB_DONE
                same(res, ref)
        except Exception as e:  # reported on the main thread
            failures.append(e)

    threads = [threading.Thread(target=worker) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not any(t.is_alive() for t in threads)
    assert not failures, failures
    st = srv.stats()
    assert st["done"] == 4 * len(jobs) and st["failed"] == 0
    srv.close()


def test_served_jobs_match_the_oracle(ctx, jobs):
    """One served job of each medium kind (freeform block, Luneburg lens,
    64^3 blob grid, its 32 shells) against the FP64 oracle directly, on a
    strided sample of its rays, under the FP32 flag rule of tests/compare.py:
    integer outcomes equal and every continuous result within 2e-5 on the
    unflagged rays."""
    import oracle
    from tests.compare import compare, fp32_flags
    srv = tracer.Server(ctx, 1 << 30)
    for wl, med, rays, ref in jobs[:4]:
        jid, res = srv.submit(med, rays, wl.dopl, wl.max_steps)
        assert srv.wait(jid, 120) == N.JOB_DONE
        idx = np.arange(0, rays.count, max(1, rays.count // 600))
        origins = np.stack([t.numpy().astype(np.float64) for t in (rays.ox, rays.oy, rays.oz)], 1)[idx]
        dirs = np.stack([t.numpy().astype(np.float64) for t in (rays.dx, rays.dy, rays.dz)], 1)[idx]
        o = oracle.trace(wl.medium, origins, dirs, wl.dopl, wl.max_steps)
        g = tracer.to_numpy({k: v[idx] for k, v in res.items()})
        f = fp32_flags(o, wl.medium, origins, dirs, wl.dopl, wl.max_steps, wl.l_ref)
        rep = compare(g, o, wl.l_ref, f)
        assert rep["int_mismatch_unflagged"] == 0, (wl.name, rep)
        assert max(rep["pos"], rep["dir"], rep["opl"]) <= 2e-5, (wl.name, rep)
        assert rep["n_flagged"] <= 0.25 * rep["n"], (wl.name, rep)
    srv.close()


def test_concurrent_jobs_overlap_on_the_device(ctx):
    """Two jobs that each hold a quarter of the GPU's resident slots, traced
    together, finish in well under the sum of their times alone: their ticks
    run at the same time on the device, on the jobs' own streams.  The times
    are the server's own (admission to completion, grin_serve_timing).  The
    jobs step at a quarter of the benchmark's dL0, about 12,600 steps a ray
    (6 ms alone), so that their copies and the scheduler's fixed costs are a
    small part of their time."""
    wl = W.freeform_workload(40000)
    dopl = wl.dopl / 4
    med = tracer.Medium(ctx, wl.medium)
    a, b = host_rays(wl, 20000), tracer.RayBatch.from_numpy(wl.rays.origins[20000:], wl.rays.dirs[20000:],
                                                              device="cpu", dtype=torch.float32)
    srv = tracer.Server(ctx, 1 << 30)
    alone = []
    for r in (a, b, a, b):  # the second pair is the one measured
        jid, _ = srv.submit(med, r, dopl, wl.max_steps)
        assert srv.wait(jid, 120) == N.JOB_DONE
        alone.append(srv.timing(jid)[1])
    ja, _ = srv.submit(med, a, dopl, wl.max_steps)
    jb, _ = srv.submit(med, b, dopl, wl.max_steps)
    assert srv.wait(ja, 120) == N.JOB_DONE and srv.wait(jb, 120) == N.JOB_DONE
    (qa, ra), (qb, rb) = srv.timing(ja), srv.timing(jb)
    together = max(qa + ra, qb + rb)  # both submitted at once
    assert qa < 0.5 * ra and qb < 0.5 * rb, (qa, ra, qb, rb)  # admitted at once
    assert together < 0.75 * (alone[2] + alone[3]), (together, alone)
    srv.close()
