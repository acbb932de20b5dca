"""The two-rays-a-thread mixed kernel (packed FP32 pair arithmetic) against
the one-ray-a-thread mixed kernel, through the C ABI.

Each packed operation is the same rounding as the scalar operation it
replaces, and the rare cases go through the same ordered step, so every
output of every ray must be bitwise equal between the two kernels: on the
freeform blocks of degree 2, 4 and 6 (both input dtypes), on counts that
leave pair slots and warps part-filled, and on a homogeneous box, where the
gradient is zero at every step and every step takes the slow path.  Their
agreement with the FP64 oracle is covered by test_gpu_trace.py, which runs
the packed kernel on these media by default."""
import dataclasses

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


def _poly_block(degree, seed):
    m = W.freeform_block_medium()
    c = W.normal(seed, 11, W.n_monomials(degree), 0.01)
    c = c * min(1.0, 0.10 / float(np.abs(c).sum()))
    c[0] += 1.55
    return dataclasses.replace(m, degree=degree, coeffs=c)


def _both(ctx, medium, rays, dopl, max_steps, dtype=torch.float64):
    med = tracer.Medium(ctx, medium)
    rb = tracer.RayBatch.from_numpy(rays.origins, rays.dirs, device="cuda", dtype=dtype)
    a = tracer.trace(ctx, med, rb, dopl, max_steps, "mixed")
    b = tracer.trace(ctx, med, rb, dopl, max_steps, "mixed", flags=tracer.FLAG_ONE_RAY_PER_THREAD)
    torch.cuda.synchronize()
    return tracer.to_numpy(a), tracer.to_numpy(b)


def _assert_bitwise(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("degree", [2, 4, 6])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_packed_equals_one_ray_freeform(ctx, degree, dtype):
    m = W.freeform_block_medium() if degree == 4 else _poly_block(degree, W.BASE_SEED + 40 + degree)
    rays = W.point_source_rays(20011, W.BASE_SEED + 7)
    a, b = _both(ctx, m, rays, 0.01, 20000, dtype)
    assert (a["steps"] > 100).mean() > 0.9  # long paths: the fast step dominates
    _assert_bitwise(a, b)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 63, 64, 65, 129, 1000, 37003])
def test_packed_ragged_counts(ctx, n):
    rays = W.point_source_rays(n, W.BASE_SEED + 8)
    a, b = _both(ctx, W.freeform_block_medium(), rays, 0.01, 20000)
    _assert_bitwise(a, b)


def test_packed_step_limit_and_slow_path_every_step(ctx):
    rays = W.point_source_rays(5000, W.BASE_SEED + 9)
    # step limit reached inside the medium by most rays
    a, b = _both(ctx, W.freeform_block_medium(), rays, 0.01, 700)
    assert (a["exit_id"] == tracer.N.EXIT_MAXSTEPS).mean() > 0.5
    _assert_bitwise(a, b)
    # zero gradient everywhere: every step goes through the slow path
    box = W.homogeneous_box(1.5, lo=(-5.0, -5.0, 0.0), hi=(5.0, 5.0, 20.0))
    a, b = _both(ctx, box, rays, 0.01, 20000)
    assert (a["steps"] > 100).all()
    _assert_bitwise(a, b)


def test_unknown_flag_bits_rejected(ctx):
    med = tracer.Medium(ctx, W.freeform_block_medium())
    rb = tracer.RayBatch.from_numpy(np.zeros((4, 3)), np.tile([0, 0, 1.0], (4, 1)))
    for flags in (2, 0x80000000):
        with pytest.raises(tracer.N.GrinError) as e:
            tracer.trace(ctx, med, rb, 0.01, 10, "mixed", flags=flags)
        assert e.value.status == -1
