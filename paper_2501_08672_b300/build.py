"""Builds libgs_b300.so in-tree with nvcc for sm_103a (no GPU needed).

    python -m paper_2501_08672_b300.build [--force] [--verbose-ptxas] [--checked]

--checked builds libgs_b300_checked.so instead: the same sources compiled
with GS_CHECKED, whose compositing kernels bounds-check every index they read
from device memory and latch GS_ERR_BOUNDS instead of reading out of bounds
(loaded by the binding when GS_B300_LIB=checked).
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgs_b300.so")
LIB_CHECKED = os.path.join(HERE, "libgs_b300_checked.so")
SOURCES = ["gs_capi.cu", "gs_project.cu", "gs_sort.cu", "gs_raster.cu", "gs_adam.cu", "gs_calib.cu",
           "gs_window.cu", "gs_ssim.cu"]
HEADERS = ["gs_internal.cuh", os.path.join("..", "..", "include", "gs.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, ptxas_verbose=False, quiet=True, checked=False):
    """Compiles every .cu to an object file and links the shared library
    (the checked build with checked=True)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(ROOT, "_build", "checked") if checked else os.path.join(ROOT, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
    if checked:
        flags += ["-DGS_CHECKED=1"]
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]
    objs = []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [NVCC] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if ptxas_verbose or not quiet:
            sys.stderr.write(r.stderr)
        objs.append(obj)
    tmp = lib + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath", "-Xlinker", "/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose-ptxas", action="store_true")
    ap.add_argument("--checked", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas_verbose=a.verbose_ptxas, quiet=False, checked=a.checked))
