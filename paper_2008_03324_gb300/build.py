"""Compile the in-tree CUDA libraries for sm_103a (nvcc, no cmake).

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_2008_03324_gb300/libfif.so (the product).  csrc/probe/ holds measurement code for the
benchmark (an FP32 FMA throughput probe), linked separately into libfif_probe.so and never part
of the product library or its header.  Rebuilds only when a source is newer than its library.
Usage: ``python -m paper_2008_03324_gb300.build [--force] [--verbose]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libfif.so")
PROBE_LIB = os.path.join(HERE, "libfif_probe.so")
OBJDIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def probe_sources():
    return sorted(glob.glob(os.path.join(CSRC, "probe", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(lib, srcs) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in srcs + headers() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Build libfif.so and libfif_probe.so where stale; returns the product library's path."""
    todo = [(lib, srcs) for lib, srcs in ((LIB, sources()), (PROBE_LIB, probe_sources()))
            if force or _stale(lib, srcs)]
    if not todo:
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    nv = nvcc()
    flags = NVCC_FLAGS + list(extra_flags or [])

    def compile_one(src):
        tag = "probe_" if os.path.basename(os.path.dirname(src)) == "probe" else ""
        obj = os.path.join(OBJDIR, tag + os.path.basename(src) + ".o")
        cmd = [nv, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = {lib: list(ex.map(compile_one, srcs)) for lib, srcs in todo}
    for lib, _ in todo:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs[lib]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
