"""The C-ABI library loads without a GPU and exports every function that
include/grin.h declares; the binding's struct layouts match the header."""
import ctypes
import os
import re

import pytest

from paper_2606_22655_b300 import _native as N
from paper_2606_22655_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("grin.h", "grin_probe.h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grin_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return N.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_poly_terms(lib):
    assert lib.grin_status_string(0) == b"ok"
    assert lib.grin_status_string(-1) == b"invalid argument"
    assert lib.grin_status_string(-9) == b"index out of bounds (checked build)"
    assert [lib.grin_poly_terms(d) for d in range(7)] == [1, 4, 10, 20, 35, 56, 84]
    assert lib.grin_poly_terms(7) == 0


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.grin_ctx_create(0, None) == -1
    assert lib.grin_ctx_destroy(None) == -1
    assert lib.grin_medium_destroy(None) == -1
    assert lib.grin_trace(None, None, None, None, None, None) == -1
    assert lib.grin_trace_host(None, None, None, None, None, None) == -1
    assert lib.grin_trace_stats_compute(None, None, 0, None, None, None) == -1


def test_struct_sizes_match_c_layout(tmp_path):
    """The binding's structs have the sizes and field offsets the C compiler
    gives the header's (a small program built against include/grin.h)."""
    import subprocess
    structs = {"grin_rays": (N.Rays, ["count", "dtype"]), "grin_out": (N.Out, ["tir_boundary", "margin"]),
               "grin_params": (N.Params, ["precision", "flags"]),
               "grin_medium_desc": (N.MediumDesc, ["grid_on_device", "n_levels", "boundary", "n_ext"]),
               "grin_serve_config": (N.ServeConfig, ["max_slots_per_job"]),
               "grin_serve_counters": (N.ServeCounters, ["ray_steps", "jobs_running"]),
               "grin_trace_stats": (N.TraceStats, ["exit_face", "exit_invalid", "flagged", "elapsed_ms"])}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "grin.h"', "int main(void) {"]
    for c, (_, fields) in structs.items():
        src.append(f'  printf("{c} %zu\\n", sizeof({c}));')
        for f in fields:
            src.append(f'  printf("{c}.{f} %zu\\n", offsetof({c}, {f}));')
    src += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(tmp_path / "layout.c"), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for c, (py, fields) in structs.items():
        assert ctypes.sizeof(py) == int(got[c]), c
        for f in fields:
            assert getattr(py, f).offset == int(got[f"{c}.{f}"]), (c, f)


def test_checked_build_exports_the_same_abi():
    """The bounds-checked build (libgrin_vrt_checked.so) exports every
    declared function and says so; the ordinary build runs no self-test."""
    build.build()
    names = declared_functions()
    checked = ctypes.CDLL(build.LIB_CHECKED)
    for n in names:
        assert hasattr(checked, n), n
    assert checked.grin_build_checked() == 1
    plain = ctypes.CDLL(build.LIB)
    assert plain.grin_build_checked() == 0
    assert plain.grin_checked_selftest(0) == N.GRIN_ERR_NOT_IMPLEMENTED
