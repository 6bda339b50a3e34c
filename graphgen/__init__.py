"""Seeded synthetic graph generators (shared input module).

This module makes inputs only.  It holds none of the BFS arithmetic, so the
oracle-side tests and the GPU path can both draw their graphs from it without
sharing any computation.  Everything is deterministic in the arguments: the
random draws come from a counter-based SplitMix64 generator keyed by
(seed, stream, index), so the same call gives the same graph on any machine
and thread count.

Graph families follow the shapes of the paper's evaluation suite (Section 3,
Table 1: a Kronecker graph, a uniform random graph, road-network-like large
diameter graphs): R-MAT, uniform random (Erdos-Renyi style), 2-D grids and
random geometric graphs, plus sets of many small uniform random graphs.

Every graph is returned as a symmetric CSR ``(row_ptr, col)`` with
``row_ptr`` int64 of length n+1 and ``col`` int32, rows sorted ascending,
no self-loops and no duplicate entries.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (g++, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i64, u64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.gg_rand64.restype = u64
        lib.gg_rand64.argtypes = [u64, u64, u64]
        lib.gg_threads.restype = i32
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, u64]
        lib.gg_er.restype = vp
        lib.gg_er.argtypes = [i64, dbl, u64]
        lib.gg_grid.restype = vp
        lib.gg_grid.argtypes = [i64, i64]
        lib.gg_rgg.restype = vp
        lib.gg_rgg.argtypes = [i64, dbl, u64]
        lib.gg_n.restype = i64
        lib.gg_n.argtypes = [vp]
        lib.gg_m.restype = i64
        lib.gg_m.argtypes = [vp]
        lib.gg_copy.restype = None
        lib.gg_copy.argtypes = [vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_sources.restype = i64
        lib.gg_sources.argtypes = [vp, i64, u64, i64, vp]
        lib.gg_uniform.restype = None
        lib.gg_uniform.argtypes = [u64, u64, u64, i64, vp]
        lib.gg_graphset.restype = i32
        lib.gg_graphset.argtypes = [i64, i64, i64, dbl, u64, i32, vp, vp, vp, vp, vp, vp, vp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _take(h) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    if not h:
        raise ValueError("graph generator rejected its arguments")
    try:
        n, m = lib.gg_n(h), lib.gg_m(h)
        row_ptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(m, dtype=np.int32)
        lib.gg_copy(h, _ptr(row_ptr), _ptr(col))
    finally:
        lib.gg_free(h)
    return row_ptr, col


def rand64(seed: int, stream: int, idx: int) -> int:
    """Draw ``idx`` of ``stream`` under ``seed`` (counter-based SplitMix64)."""
    return int(_load().gg_rand64(seed, stream, idx))


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, perm_seed: int = 1):
    """R-MAT graph with 2**scale vertices from edgefactor*2**scale pairs.

    Quadrant probabilities (a, b, c, 1-a-b-c); vertex ids permuted by a
    Fisher-Yates shuffle drawn from ``perm_seed``; symmetrised, self-loops and
    duplicates removed.
    """
    return _take(_load().gg_rmat(scale, edgefactor, a, b, c, seed, perm_seed))


def erdos_renyi(n: int, avg_deg: float, seed: int):
    """Uniform random graph from round(n*avg_deg/2) uniform pairs (cleaned)."""
    return _take(_load().gg_er(n, avg_deg, seed))


def grid2d(rows: int, cols: int):
    """rows x cols 4-neighbour grid, vertex (r, c) = r*cols + c, no wrap."""
    return _take(_load().gg_grid(rows, cols))


def rgg(n: int, radius: float, seed: int):
    """Random geometric graph of n uniform points in the unit square."""
    return _take(_load().gg_rgg(n, radius, seed))


def rgg_radius(n: int, mean_degree: float) -> float:
    """Radius giving expected degree ``mean_degree`` (pi r^2 n = mean degree, ignoring borders)."""
    return float(np.sqrt(mean_degree / (np.pi * n)))


def sources(row_ptr: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k sources drawn uniformly (with replacement) among vertices of degree > 0."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = np.empty(k, dtype=np.int32)
    r = _load().gg_sources(_ptr(row_ptr), len(row_ptr) - 1, seed, k, _ptr(out))
    if r < 0:
        raise ValueError("graph has no edge: no source of nonzero degree")
    return out


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """U[0,1) draws start..start+count-1 of (seed, stream)."""
    out = np.empty(count, dtype=np.float64)
    _load().gg_uniform(seed, stream, start, count, _ptr(out))
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int, stream: int = 9) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: cumulative -ln(1-U)/rate."""
    u = uniform(seed, stream, 0, count)
    return np.cumsum(-np.log1p(-u) / rate_per_s)


class GraphSet:
    """Concatenated set of small graphs (see ``graph_set``)."""

    def __init__(self, voff, eoff, row_ptr, col, src):
        self.voff, self.eoff, self.row_ptr, self.col, self.src = voff, eoff, row_ptr, col, src

    @property
    def count(self) -> int:
        return len(self.voff) - 1

    def graph(self, i: int):
        """(row_ptr, col) of graph i with local ids."""
        n = int(self.voff[i + 1] - self.voff[i])
        rs = int(self.voff[i]) + i
        rp = self.row_ptr[rs:rs + n + 1]
        cl = self.col[int(self.eoff[i]):int(self.eoff[i + 1])]
        return rp, cl


def graph_set(count: int, nmin: int = 1000, nmax: int = 100000, avg_deg: float = 8.0, seed: int = 4):
    """``count`` uniform random graphs with log-uniform sizes in [nmin, nmax]."""
    lib = _load()
    nv = np.zeros(1, dtype=np.int64)
    ne = np.zeros(1, dtype=np.int64)
    rc = lib.gg_graphset(count, nmin, nmax, avg_deg, seed, 1, _ptr(nv), _ptr(ne), None, None, None, None, None)
    if rc != 0:
        raise ValueError("bad graph-set arguments")
    voff = np.empty(count + 1, dtype=np.int64)
    eoff = np.empty(count + 1, dtype=np.int64)
    row_ptr = np.empty(int(nv[0]) + count, dtype=np.int64)
    col = np.empty(int(ne[0]), dtype=np.int32)
    src = np.empty(count, dtype=np.int32)
    lib.gg_graphset(count, nmin, nmax, avg_deg, seed, 0, _ptr(nv), _ptr(ne), _ptr(voff), _ptr(eoff),
                    _ptr(row_ptr), _ptr(col), _ptr(src))
    return GraphSet(voff, eoff, row_ptr, col, src)


def csr_sha256(row_ptr: np.ndarray, col: np.ndarray) -> str:
    """SHA-256 over the int64 row pointer and int32 column arrays."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(row_ptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(col, dtype=np.int32).tobytes())
    return h.hexdigest()
