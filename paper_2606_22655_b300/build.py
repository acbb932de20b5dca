"""Build the CUDA library libgrin_vrt.so in-tree for sm_103a (B300), and
the same library with range-checked kernel indices, libgrin_vrt_checked.so.

    python -m paper_2606_22655_b300.build [--verbose-ptxas]

Each .cu file under csrc/ is compiled to an object with nvcc
(-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo) and the objects are
linked into paper_2606_22655_b300/lib/libgrin_vrt.so.  Sources are rebuilt
only when they (or a header) are newer than the library.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "libgrin_vrt.so")
# the same library with every kernel array index range-checked (-DGRIN_CHECKED)
LIB_CHECKED = os.path.join(LIB_DIR, "libgrin_vrt_checked.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# per-source extra flags: the plain FP64 tracer must not contract a*b+c; the
# mixed tracer takes hardware-approximate FP32 division and square root
EXTRA = {"trace_fp64.cu": ["--fmad=false"], "adjoint.cu": ["--fmad=false"],
         "trace_mixed.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _flags(ptxas_verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src: str, ptxas_verbose: bool, checked: bool = False) -> str:
    out_dir = os.path.join(BUILD, "checked") if checked else BUILD
    obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [_nvcc()] + _flags(ptxas_verbose) + EXTRA.get(os.path.basename(src), []) + \
        (["-DGRIN_CHECKED"] if checked else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if ptxas_verbose:
        sys.stderr.write(r.stderr)
    return obj


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _sources() + _headers())


def build(force: bool = False, ptxas_verbose: bool = False, checked: bool = True) -> str:
    """Build libgrin_vrt.so and (checked=True) libgrin_vrt_checked.so; both
    variants' sources compile in one pool of nvcc processes."""
    variants = [False] + ([True] if checked else [])
    todo = [c for c in variants if force or ptxas_verbose or needs_build(LIB_CHECKED if c else LIB)]
    if not todo:
        return LIB
    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    jobs = [(src, c) for c in todo for src in _sources()]
    newest_header = max([os.path.getmtime(h) for h in _headers()] + [0.0])

    def obj_of(src: str, checked: bool) -> str:
        return os.path.join(BUILD, "checked" if checked else "", os.path.basename(src)[:-3] + ".o")

    def fresh(src: str, checked: bool) -> bool:
        # an object newer than its source and every header is reused
        o = obj_of(src, checked)
        return (not force and not ptxas_verbose and os.path.exists(o) and
                os.path.getmtime(o) > max(os.path.getmtime(src), newest_header))

    def one(j):
        src, c = j
        return (c, obj_of(src, c) if fresh(src, c) else _compile(src, ptxas_verbose, c))

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(one, jobs))
    for c in todo:
        lib = LIB_CHECKED if c else LIB
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for cc, o in objs if cc == c]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose-ptxas", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas_verbose=a.verbose_ptxas))
