"""Oracle for BFS distances: a plain serial queue BFS in C (``bfs_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and it shares no code with it.

The C function follows the definition of BFS distance (hop count of a
shortest path from the source; Section 1 and Listings 1-3 of the paper all
reach this unique value).  The helpers below only loop over sources or graphs
and convert encodings; they add no arithmetic of their own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle with gcc (plain C, -O2, no OpenMP)."""
    src = src or _SRC
    out = out or _LIB_PATH
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp], check=True)
        os.replace(tmp, out)
    return out


def load_library(path: str):
    """Load an oracle shared object and declare its signature."""
    lib = ctypes.CDLL(path)
    lib.oracle_bfs.restype = ctypes.c_int
    lib.oracle_bfs.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_void_p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def bfs(row_ptr: np.ndarray, col: np.ndarray, src: int, lib=None) -> np.ndarray:
    """int32 distances from ``src`` (-1 = unreachable)."""
    lib = lib or _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(row_ptr) - 1
    dist = np.empty(max(n, 0), dtype=np.int32)
    rc = lib.oracle_bfs(n, row_ptr.ctypes.data, col.ctypes.data, int(src), dist.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_bfs rejected its input (rc={rc})")
    return dist


def bfs_many(row_ptr: np.ndarray, col: np.ndarray, srcs, threads: int | None = None) -> np.ndarray:
    """Rows of ``bfs`` for each source in order, run on a thread pool.

    The C call releases the GIL, so independent sources run in parallel.
    """
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    srcs = [int(s) for s in srcs]
    n = len(row_ptr) - 1
    out = np.empty((len(srcs), n), dtype=np.int32)
    lib = _load()

    def one(i):
        out[i] = bfs(row_ptr, col, srcs[i], lib)

    threads = threads or min(len(srcs), os.cpu_count() or 1) or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(len(srcs))))
    return out


def to_uint8(dist: np.ndarray) -> np.ndarray:
    """uint8 encoding of int32 distances: -1 -> 255; values above 254 are an error."""
    if dist.size and int(dist.max()) > 254:
        raise OverflowError("distance above 254 has no uint8 encoding")
    return np.where(dist < 0, 255, dist).astype(np.uint8)
