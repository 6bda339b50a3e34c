"""Build ``libbfs.so`` (the CUDA library behind ``include/bfs.h``) in-tree.

Every ``csrc/*.cu`` / ``csrc/*.cpp`` file is compiled for sm_103a in
parallel, then linked into ``paper_2503_00430_gb300/libbfs.so``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
# GBFS_BUILD_TAG builds a side variant (own object dir and library name), e.g.
# together with NVCC_APPEND_FLAGS to compare compile-time settings.
_TAG = os.environ.get("GBFS_BUILD_TAG", "")
OBJDIR = os.path.join(HERE, "_build" + _TAG)
LIB = os.path.join(HERE, f"libbfs{_TAG}.so")
# The bounds-checked variant (every data-dependent global index of the
# single-source kernels checked, first violation recorded): its own objects and
# library, built on request (build(debug_bounds=True)).
DEBUG_OBJDIR = os.path.join(HERE, "_build_dbg")
DEBUG_LIB = os.path.join(HERE, "libbfs_dbg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose_ptxas=False, objdir=OBJDIR, defines=()):
    obj = os.path.join(objdir, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + _headers()) and not verbose_ptxas:
        return obj, ""
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-I", INCLUDE, "-I", CSRC,
           *[f"-D{d}" for d in defines], "-c", src, "-o", obj + ".tmp"]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False, debug_bounds: bool = False) -> str:
    """Compile and link; returns the library path (the bounds-checked variant with debug_bounds)."""
    objdir, lib = (DEBUG_OBJDIR, DEBUG_LIB) if debug_bounds else (OBJDIR, LIB)
    defines = ("GBFS_DEBUG_BOUNDS",) if debug_bounds else ()
    os.makedirs(objdir, exist_ok=True)
    srcs = _sources()
    if force:
        for s in srcs:
            o = os.path.join(objdir, os.path.basename(s) + ".o")
            if os.path.exists(o):
                os.remove(o)
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas, objdir, defines), srcs))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    if _stale(lib, objs) or force:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
