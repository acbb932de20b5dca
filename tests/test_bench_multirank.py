"""The multi-rank path of bench.py on CPU: two gloo ranks.  Each rank draws
its own ray bundle of the same size (weak scaling), the only collectives are
the MAX of the timed region and the SUM of the ray-steps, so the
whole-job rate counts every rank's ray-steps over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    import bench
    from paper_2606_22655_b300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    wl = W.freeform_workload(64, ray_seed=bench.rank_ray_seed(rank))
    region = 2.0 + rank  # rank 1 is the slower one
    t, rate = bench.aggregate(region, 1000.0 * (1 + rank), 5, ws)
    dist.destroy_process_group()
    q.put((rank, t, rate, wl.rays.origins.copy(), wl.rays.dirs.copy(), wl.medium.coeffs.copy()))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_aggregate_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, t0, v0, o0, d0, c0), (r1, t1, v1, o1, d1, c1) = out
    assert t0 == t1 == 3.0  # the slowest rank's time on both
    assert v0 == v1 == (1000.0 + 2000.0) * 5 / 3.0  # all ranks' ray-steps
    np.testing.assert_array_equal(c0, c1)  # same medium
    assert not np.array_equal(d0, d1)  # different bundles
    assert o0.shape == o1.shape
