"""Build the CUDA library libfslbm.so for sm_103a (in-tree, under _build/).

Each translation unit is compiled by its own nvcc process in parallel, then
linked into one shared library.  build(checked=True) makes the bounds-checked
variant (compiled with FSLBM_CHECKED) under _build/checked/, which the
binding loads when FSLBM_CHECKED=1 is set in the environment.  Nothing here
runs on the GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfslbm.so")
CHECKED_LIB = os.path.join(BUILD, "checked", "libfslbm.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["fslbm_step.cu", "fslbm_step_p64.cu", "fslbm_step_p32.cu", "fslbm_step_p16.cu", "fslbm_conv.cu",
           "fslbm_state.cu", "fslbm_api.cu", "fslbm_adjoint.cu", "fslbm_adjoint_p64.cu", "fslbm_adjoint_p32.cu",
           "fslbm_adjoint_p16.cu", "fslbm_noalloc.cu", "fslbm_staged.cu", "fslbm_halo.cu", "fslbm_rate.cu",
           "fslbm_pairs.cu"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr", *extra]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _stamp_ok(bdir) -> bool:
    """Objects in bdir were made on this machine type (a copy of the tree
    may carry another architecture's objects)."""
    try:
        return open(os.path.join(bdir, "STAMP")).read().strip() == platform.machine()
    except OSError:
        return False


def build(verbose: bool = False, force: bool = False, extra=(), checked: bool = False) -> str:
    bdir = os.path.dirname(CHECKED_LIB) if checked else BUILD
    lib = CHECKED_LIB if checked else LIB
    if checked:
        extra = ("-DFSLBM_CHECKED", *extra)
    os.makedirs(bdir, exist_ok=True)
    if not _stamp_ok(bdir):
        force = True
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "fslbm.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        if force or _stale(o, [s, *headers]):
            jobs.append([nvcc(), *_flags(extra), "-c", s, "-o", o])
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(lib):
        tmp = lib + f".{os.getpid()}.tmp"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
        with open(os.path.join(bdir, "STAMP"), "w") as fh:
            fh.write(platform.machine())
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else (), checked="--checked" in sys.argv))
