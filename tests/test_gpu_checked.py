"""The bounds-checked build (GRIN_CHECKED=1 loads libgrin_vrt_checked.so).

Each case runs in a child process, since a process loads one build of the
library: the self-test's deliberate out-of-range index is recorded (site 4)
and cleared by the read; traces of analytic, gridded (tap cache, claim
order) and layered media record nothing and give bit for bit the results of
the ordinary build.  The whole GPU suite also runs against this build with
GRIN_CHECKED=1, its status checked after every test (tests/conftest.py).
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes, sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2606_22655_b300 import _native as N, tracer, workloads as W
lib = N.load()
out = {"checked": lib.grin_build_checked()}
if out["checked"]:
    site = ctypes.c_int32()
    assert lib.grin_checked_selftest(0) == 0
    out["selftest"] = (lib.grin_checked_status(0, ctypes.byref(site)), site.value)
    assert lib.grin_checked_status(0, ctypes.byref(site)) == 0 and site.value == 0
ctx = tracer.Context(0)
res = {}
for name, wl in (("freeform", W.freeform_workload(20000)), ("grid", W.blob_workload(n_rays=70000, res=32)),
                 ("layered", W.blob_workload(n_rays=3000, res=32, n_levels=16))):
    med = tracer.Medium(ctx, wl.medium)
    rb = tracer.RayBatch.from_numpy(wl.rays.origins, wl.rays.dirs, device="cuda", dtype=torch.float32)
    for prec in ("mixed", "fp64"):
        r = tracer.to_numpy(tracer.trace(ctx, med, rb, wl.dopl, 2000 if prec == "fp64" else wl.max_steps, prec))
        for k, v in r.items():
            res[f"{name}_{prec}_{k}"] = v
torch.cuda.synchronize()
site = ctypes.c_int32()
out["status"] = (lib.grin_checked_status(0, ctypes.byref(site)), site.value)
np.savez(sys.argv[2], **res)
print(out)
'''


def _child(tmp_path, checked):
    env = dict(os.environ, GRIN_CHECKED="1" if checked else "0")
    path = tmp_path / ("checked.npz" if checked else "plain.npz")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(path)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return eval(r.stdout.strip().splitlines()[-1]), dict(np.load(path))


def test_checked_build_catches_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    info, chk = _child(tmp_path, True)
    assert info["checked"] == 1
    assert info["selftest"] == (-9, 4)          # GRIN_ERR_CHECKED_BOUNDS at site 4
    assert info["status"] == (0, 0)             # nothing out of range in the traces
    info0, plain = _child(tmp_path, False)
    assert info0["checked"] == 0 and info0["status"] == (0, 0)
    for k in plain:
        np.testing.assert_array_equal(chk[k], plain[k], err_msg=k)
