"""GB300 breadth-first search: thin Python binding of ``libbfs.so``.

The functions here only marshal arguments for the C ABI declared in
``include/bfs.h`` (same names); every step of the BFS runs in the library's
CUDA kernels.  There is no CPU fallback: if ``libbfs.so`` is missing or
cannot be loaded, every call raises.

Device buffers may be passed as torch CUDA tensors (their ``data_ptr()``),
host buffers as numpy arrays; streams as ``torch.cuda.Stream`` objects, raw
``cudaStream_t`` integers or ``None`` (legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfs.so")

BFS_OK = 0
BFS_EINVAL = -1
BFS_ENOMEM = -2
BFS_ECUDA = -3
BFS_ETIMEOUT = -4
BFS_EAGAIN = -5
BFS_ERANGE = -6
BFS_ENOTFOUND = -7

BFS_HOST_PTRS = 0
BFS_DEVICE_PTRS = 1
BFS_VALIDATE = 2
BFS_VALIDATE_SYMMETRY = 4
BFS_DEGREE_ORDER = 8
BFS_NO_HEAD = 16

BFS_POLICY_AUTO = 0
BFS_POLICY_FRONTIER = 1
BFS_POLICY_EDGES = 2
BFS_POLICY_TD_ONLY = 3
BFS_POLICY_BU_FROM_1 = 4
BFS_POLICY_SCRIPT = 5
BFS_POLICY_LOCAL = 6

BFS_LAUNCH_PERSISTENT = 0
BFS_LAUNCH_PER_LEVEL = 1
BFS_LAUNCH_GRAPH = 2


class BfsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = bfs_strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class bfs_params(ctypes.Structure):
    _fields_ = [
        ("policy", ctypes.c_int32), ("launch", ctypes.c_int32), ("alpha", ctypes.c_int32),
        ("beta", ctypes.c_int32), ("tau_inv", ctypes.c_int32), ("large_diameter_degree", ctypes.c_int32),
        ("small_max", ctypes.c_int32), ("chunk", ctypes.c_int32), ("bu_warp_min", ctypes.c_int32),
        ("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
        ("timeout_ms", ctypes.c_int32), ("script", ctypes.c_uint64),
        ("test_barrier_extra", ctypes.c_int32), ("bu_chunk", ctypes.c_int32),
        ("bu_thread_max", ctypes.c_int32), ("ms_lanes", ctypes.c_int32), ("ms_ring", ctypes.c_int32),
        ("ms_heavy_min", ctypes.c_int32), ("ms_degree_order", ctypes.c_int32), ("ms_alpha", ctypes.c_int32),
        ("ms_relabel", ctypes.c_int32), ("relabel", ctypes.c_int32), ("local_levels", ctypes.c_int32),
        ("local_threads", ctypes.c_int32), ("serve_queue", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1),
    ]


class bfs_stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("td_levels", ctypes.c_int32), ("bu_levels", ctypes.c_int32),
        ("conversions", ctypes.c_int32), ("reached", ctypes.c_int64), ("edges_reached", ctypes.c_int64),
        ("td_frontier", ctypes.c_int64), ("td_edges", ctypes.c_int64), ("bu_unvisited", ctypes.c_int64),
        ("bu_edges", ctypes.c_int64), ("bu_found", ctypes.c_int64), ("conv_frontier", ctypes.c_int64),
        ("supersteps", ctypes.c_int64), ("improved", ctypes.c_int64), ("init_ns", ctypes.c_int64),
        ("finish_ns", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class bfs_multi_stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("push_levels", ctypes.c_int32), ("pull_levels", ctypes.c_int32),
        ("groups", ctypes.c_int32), ("pushed_edges", ctypes.c_int64), ("pulled_edges", ctypes.c_int64),
        ("output_bytes", ctypes.c_int64), ("pull_active", ctypes.c_int64), ("push_frontier", ctypes.c_int64),
        ("found", ctypes.c_int64), ("reserved", ctypes.c_int64 * 1),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class bfs_dup_level(ctypes.Structure):
    _fields_ = [("frontier", ctypes.c_int64), ("unique", ctypes.c_int64), ("edges", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bfs_dup_stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("pad", ctypes.c_int32), ("frontier_entries", ctypes.c_int64),
        ("unique", ctypes.c_int64), ("edges", ctypes.c_int64), ("reserved", ctypes.c_int64 * 4),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "pad")}


class bfs_graphset_stats(ctypes.Structure):
    _fields_ = [
        ("graphs", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("blocks", ctypes.c_int32),
        ("pad", ctypes.c_int32), ("levels", ctypes.c_int64), ("td_levels", ctypes.c_int64),
        ("bu_levels", ctypes.c_int64), ("reserved", ctypes.c_int64 * 4),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "pad")}


class bfs_query_stats(ctypes.Structure):
    _fields_ = [
        ("submit_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
        ("levels", ctypes.c_int32), ("lane", ctypes.c_int32), ("graph_id", ctypes.c_int32),
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int64 * 2),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class bfs_tune_report(ctypes.Structure):
    _fields_ = [
        ("trials", ctypes.c_int32), ("sources", ctypes.c_int32), ("start_ms", ctypes.c_double),
        ("best_ms", ctypes.c_double), ("reserved", ctypes.c_int64 * 4),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class bfs_level_stat(ctypes.Structure):
    _fields_ = [
        ("direction", ctypes.c_int32), ("converted", ctypes.c_int32), ("frontier", ctypes.c_int64),
        ("edges", ctypes.c_int64), ("unvisited", ctypes.c_int64), ("found", ctypes.c_int64),
        ("ns", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every entry point the binding declares.
_vp, _i32, _i64, _u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_SIGNATURES = [
    ("bfs_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("bfs_version", ctypes.c_int, []),
    ("bfs_debug_bounds", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("bfs_params_default", None, [ctypes.POINTER(bfs_params)]),
    ("bfs_graph_upload", ctypes.c_int, [_vp, ctypes.c_int, _vp, _i64, _i64, ctypes.c_int, ctypes.POINTER(_vp)]),
    ("bfs_graph_free", None, [_vp]),
    ("bfs_graph_info", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("bfs_single", ctypes.c_int, [_vp, _i32, _vp, _vp]),
    ("bfs_single_ex", ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(bfs_params), ctypes.POINTER(bfs_stats),
                                     _vp, _i32, _vp]),
    ("bfs_single_async", ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(bfs_params), _vp]),
    ("bfs_single_wait", ctypes.c_int, [_vp]),
    ("bfs_single_noalloc", ctypes.c_int, [_vp, ctypes.c_int, _vp, _i64, _i64, _i32, _vp, _vp]),
    ("bfs_parents", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("bfs_single_nonatomic", ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(bfs_dup_stats),
                                            ctypes.POINTER(bfs_dup_level), _i32, _vp]),
    ("bfs_single_nonatomic_ex", ctypes.c_int, [_vp, _i32, _vp, ctypes.c_int, ctypes.POINTER(bfs_dup_stats),
                                               ctypes.POINTER(bfs_dup_level), _i32, _vp]),
    ("bfs_multi", ctypes.c_int, [_vp, _vp, _i32, _vp, ctypes.c_int, _vp]),
    ("bfs_multi_ex", ctypes.c_int, [_vp, _vp, _i32, _vp, ctypes.c_int, ctypes.POINTER(bfs_params),
                                    ctypes.POINTER(bfs_multi_stats), _vp]),
    ("bfs_graphset_upload", ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, ctypes.c_int, ctypes.POINTER(_vp)]),
    ("bfs_graphset_free", None, [_vp]),
    ("bfs_graphset_run", ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(bfs_params),
                                        ctypes.POINTER(bfs_graphset_stats), _vp]),
    ("bfs_tune", ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(bfs_params), ctypes.POINTER(bfs_params),
                                ctypes.POINTER(bfs_tune_report)]),
    ("bfs_tune_multi", ctypes.c_int, [_vp, _vp, _i32, ctypes.c_int, ctypes.POINTER(bfs_params),
                                      ctypes.POINTER(bfs_params), ctypes.POINTER(bfs_tune_report)]),
    ("bfs_tune_graphset", ctypes.c_int, [_vp, _vp, ctypes.POINTER(bfs_params), ctypes.POINTER(bfs_params),
                                         ctypes.POINTER(bfs_tune_report)]),
    ("bfs_serve_create", ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(bfs_params), ctypes.POINTER(_vp)]),
    ("bfs_serve_add_graph", ctypes.c_int, [_vp, _vp, ctypes.POINTER(_i32)]),
    ("bfs_serve_submit", ctypes.c_int, [_vp, _i32, _i32, _vp, ctypes.POINTER(_u64)]),
    ("bfs_serve_poll", ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(bfs_query_stats)]),
    ("bfs_serve_wait", ctypes.c_int, [_vp, _u64, _i64, ctypes.POINTER(bfs_query_stats)]),
    ("bfs_serve_destroy", None, [_vp]),
]


def load(path: str | None = None):
    """Load ``libbfs.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"libbfs.so not built ({path}); run paper_2503_00430_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_names() -> list[str]:
    return [n for n, _, _ in _SIGNATURES]


def _check(rc: int, what: str):
    if rc != BFS_OK:
        raise BfsError(rc, what)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    h = getattr(stream, "cuda_stream", None)
    if h is not None:
        return int(h)
    raise TypeError("stream must be None, an int cudaStream_t or a torch.cuda.Stream")


def _ptr(buf) -> int:
    """Address of a torch tensor (data_ptr) or a numpy array."""
    if hasattr(buf, "data_ptr"):
        return int(buf.data_ptr())
    if isinstance(buf, np.ndarray):
        return int(buf.ctypes.data)
    if isinstance(buf, int):
        return buf
    raise TypeError(f"unsupported buffer type {type(buf)}")


def bfs_strerror(code: int) -> str:
    return load().bfs_strerror(code).decode()


def bfs_version() -> int:
    return int(load().bfs_version())


def bfs_debug_bounds(reset: bool = False) -> tuple[int, bool]:
    """(first recorded out-of-range index word or 0, whether this library checks bounds)."""
    v = ctypes.c_uint64()
    c = ctypes.c_int()
    _check(load().bfs_debug_bounds(ctypes.byref(v), ctypes.byref(c), 1 if reset else 0), "bfs_debug_bounds")
    return v.value, bool(c.value)


def bfs_params_default() -> bfs_params:
    p = bfs_params()
    load().bfs_params_default(ctypes.byref(p))
    return p


def make_params(**kw) -> bfs_params:
    """Default parameters with the given fields replaced."""
    p = bfs_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"bfs_params has no field {k}")
        setattr(p, k, v)
    return p


class Graph:
    """A CSR graph resident on the current CUDA device (``bfs_graph*``)."""

    def __init__(self, handle: int, n: int, m: int):
        self.handle = handle
        self.n = n
        self.m = m

    def info(self) -> dict:
        n, m, mx, iso = (ctypes.c_int64() for _ in range(4))
        _check(load().bfs_graph_info(self.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(mx),
                                     ctypes.byref(iso)), "bfs_graph_info")
        return {"n": n.value, "m": m.value, "max_degree": mx.value, "isolated": iso.value}

    def free(self):
        if self.handle:
            load().bfs_graph_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bfs_graph_upload(row_ptr, col_idx, n: int | None = None, m: int | None = None, flags: int = 0,
                     row_ptr_bits: int | None = None) -> Graph:
    """Upload a CSR graph.  numpy arrays are host pointers, torch CUDA tensors device pointers."""
    lib = load()
    is_dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
    if not is_dev:
        row_ptr = np.ascontiguousarray(row_ptr)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        if row_ptr.dtype not in (np.int32, np.int64):
            row_ptr = row_ptr.astype(np.int64)
        bits = row_ptr.dtype.itemsize * 8
    else:
        bits = row_ptr.element_size() * 8
        flags |= BFS_DEVICE_PTRS
    if row_ptr_bits is not None and row_ptr_bits != bits:
        if is_dev:
            raise ValueError("convert device row_ptr to the requested width first")
        row_ptr = row_ptr.astype(np.int32 if row_ptr_bits == 32 else np.int64)
        bits = row_ptr_bits
    n = len(row_ptr) - 1 if n is None else n
    m = len(col_idx) if m is None else m
    h = ctypes.c_void_p()
    _check(lib.bfs_graph_upload(_ptr(row_ptr), bits, _ptr(col_idx) if m else None, n, m, flags, ctypes.byref(h)),
           "bfs_graph_upload")
    return Graph(h.value, n, m)


def bfs_graph_free(g: Graph):
    g.free()


def bfs_single(g: Graph, src: int, dist, stream=None):
    """Distances from ``src`` into ``dist`` (int32[n], device tensor or host numpy array)."""
    _check(load().bfs_single(g.handle, int(src), _ptr(dist), _stream_handle(stream)), "bfs_single")
    return dist


def bfs_single_ex(g: Graph, src: int, dist, params: bfs_params | None = None, stats: bool = False,
                  level_cap: int = 0, stream=None):
    """bfs_single with parameters; returns (stats dict or None, list of level dicts).

    Level records without ``stats`` come from the production (non-counting)
    kernel: direction, converted, frontier, found and ns; edges and unvisited
    are filled only with ``stats=True``."""
    st = bfs_stats() if stats else None
    lv = (bfs_level_stat * level_cap)() if level_cap > 0 else None
    rc = load().bfs_single_ex(g.handle, int(src), _ptr(dist), ctypes.byref(params) if params is not None else None,
                              ctypes.byref(st) if st is not None else None,
                              ctypes.cast(lv, ctypes.c_void_p) if lv is not None else None, level_cap,
                              _stream_handle(stream))
    _check(rc, "bfs_single_ex")
    levels = []
    if lv is not None:
        # every level (super-step under BFS_POLICY_LOCAL) has a non-empty frontier; unused entries stay zero
        nrec = (st.supersteps or st.levels) if st is not None else None
        nl = min(nrec, level_cap) if nrec is not None else next(
            (i for i in range(level_cap) if lv[i].frontier == 0), level_cap)
        levels = [lv[i].as_dict() for i in range(nl)]
    return (st.as_dict() if st is not None else None), levels


def bfs_single_async(g: Graph, src: int, dist, params: bfs_params | None = None, stream=None):
    """Enqueue one single-source query without waiting (``dist``: device or pinned host
    memory); ``bfs_single_wait`` reports a failed status of the queries since the last wait."""
    _check(load().bfs_single_async(g.handle, int(src), _ptr(dist),
                                   ctypes.byref(params) if params is not None else None, _stream_handle(stream)),
           "bfs_single_async")
    return dist


def bfs_single_wait(g: Graph) -> None:
    """Wait for g's enqueued single-source queries; raises BfsError with the first failed status."""
    _check(load().bfs_single_wait(g.handle), "bfs_single_wait")


def bfs_single_noalloc(row_ptr, col_idx, src: int, dist, stream=None):
    """Distances from ``src`` with no allocation: ``row_ptr`` (int32/int64),
    ``col_idx`` (int32) and ``dist`` (int32[n]) are torch CUDA tensors; the
    scratch is the library's static 64 MiB device array (see include/bfs.h)."""
    bits = row_ptr.element_size() * 8
    n = row_ptr.numel() - 1
    m = col_idx.numel()
    _check(load().bfs_single_noalloc(_ptr(row_ptr), bits, _ptr(col_idx) if m else None, n, m, int(src), _ptr(dist),
                                     _stream_handle(stream)), "bfs_single_noalloc")
    return dist


def bfs_multi(g: Graph, srcs, dist, dist_bits: int = 32, stream=None):
    """Distances from every source in ``srcs`` into ``dist`` ([k][n], uint8 or int32)."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    _check(load().bfs_multi(g.handle, _ptr(srcs), len(srcs), _ptr(dist), dist_bits, _stream_handle(stream)),
           "bfs_multi")
    return dist


def bfs_multi_ex(g: Graph, srcs, dist, dist_bits: int = 32, params: bfs_params | None = None, stream=None) -> dict:
    """bfs_multi with parameters; returns its counters."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    st = bfs_multi_stats()
    _check(load().bfs_multi_ex(g.handle, _ptr(srcs), len(srcs), _ptr(dist), dist_bits,
                               ctypes.byref(params) if params is not None else None, ctypes.byref(st),
                               _stream_handle(stream)), "bfs_multi_ex")
    return st.as_dict()


def bfs_parents(g: Graph, dist, parent, stream=None) -> None:
    """Parent array (BFS tree) of finished distances: first list neighbour one level closer."""
    _check(load().bfs_parents(g.handle, _ptr(dist), _ptr(parent), _stream_handle(stream)), "bfs_parents")


BFS_DUP_DEDUP = 0
BFS_DUP_EXPAND = 1


def bfs_single_nonatomic(g: Graph, src: int, dist, level_cap: int = 0, stats: bool = True, stream=None,
                         expand_duplicates: bool = False):
    """The paper's non-atomic top-down BFS (duplicates allowed); returns (totals or None, per-level list).
    ``expand_duplicates`` expands every appended entry again (the paper's variant, BFS_DUP_EXPAND)."""
    st = bfs_dup_stats() if stats else None
    lv = (bfs_dup_level * level_cap)() if level_cap > 0 else None
    mode = BFS_DUP_EXPAND if expand_duplicates else BFS_DUP_DEDUP
    _check(load().bfs_single_nonatomic_ex(g.handle, int(src), _ptr(dist), mode,
                                          ctypes.byref(st) if st is not None else None, lv, level_cap,
                                          _stream_handle(stream)), "bfs_single_nonatomic")
    levels = [] if lv is None else [x.as_dict() for x in lv]
    if st is not None:
        levels = levels[:st.levels]
    return (st.as_dict() if st is not None else None), levels


class GraphSet:
    """A set of small graphs resident on the device (``bfs_graphset*``)."""

    def __init__(self, handle: int, count: int, total_v: int):
        self.handle = handle
        self.count = count
        self.total_v = total_v

    def free(self):
        if self.handle:
            load().bfs_graphset_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bfs_graphset_upload(voff, eoff, row_ptr, col, flags: int = 0) -> GraphSet:
    """Upload concatenated graphs (host numpy arrays; layout as in include/bfs.h)."""
    voff = np.ascontiguousarray(voff, dtype=np.int64)
    eoff = np.ascontiguousarray(eoff, dtype=np.int64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().bfs_graphset_upload(_ptr(voff), _ptr(eoff), _ptr(row_ptr), _ptr(col) if len(col) else None,
                                      len(voff) - 1, flags, ctypes.byref(h)), "bfs_graphset_upload")
    return GraphSet(h.value, len(voff) - 1, int(voff[-1]))


def bfs_graphset_free(s: GraphSet):
    s.free()


def bfs_graphset_run(s: GraphSet, srcs, dist, params: bfs_params | None = None, stream=None) -> dict:
    """BFS of every graph from its source; distances into ``dist`` (int32[total vertices])."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    st = bfs_graphset_stats()
    _check(load().bfs_graphset_run(s.handle, _ptr(srcs), _ptr(dist), ctypes.byref(params) if params is not None else None,
                                   ctypes.byref(st), _stream_handle(stream)), "bfs_graphset_run")
    return st.as_dict()


class Server:
    """A serving loop over resident graphs (``bfs_server*``)."""

    def __init__(self, mem_budget: int, params: bfs_params | None = None):
        h = ctypes.c_void_p()
        _check(load().bfs_serve_create(int(mem_budget), ctypes.byref(params) if params is not None else None,
                                       ctypes.byref(h)), "bfs_serve_create")
        self.handle = h.value

    def add_graph(self, g: Graph) -> int:
        gid = ctypes.c_int32()
        _check(load().bfs_serve_add_graph(self.handle, g.handle, ctypes.byref(gid)), "bfs_serve_add_graph")
        return gid.value

    def submit(self, graph_id: int, src: int, dist_out) -> int:
        t = ctypes.c_uint64()
        _check(load().bfs_serve_submit(self.handle, int(graph_id), int(src), _ptr(dist_out), ctypes.byref(t)),
               "bfs_serve_submit")
        return t.value

    def poll(self, ticket: int):
        """None while running, else the query's stats dict."""
        done = ctypes.c_int()
        st = bfs_query_stats()
        _check(load().bfs_serve_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(st)), "bfs_serve_poll")
        return st.as_dict() if done.value else None

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        st = bfs_query_stats()
        _check(load().bfs_serve_wait(self.handle, ticket, int(timeout_us), ctypes.byref(st)), "bfs_serve_wait")
        return st.as_dict()

    def destroy(self):
        if self.handle:
            load().bfs_serve_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def bfs_serve_create(mem_budget: int, params: bfs_params | None = None) -> Server:
    return Server(mem_budget, params)


def bfs_serve_add_graph(srv: Server, g: Graph) -> int:
    return srv.add_graph(g)


def bfs_serve_submit(srv: Server, graph_id: int, src: int, dist_out) -> int:
    return srv.submit(graph_id, src, dist_out)


def bfs_serve_poll(srv: Server, ticket: int):
    return srv.poll(ticket)


def bfs_serve_wait(srv: Server, ticket: int, timeout_us: int = -1) -> dict:
    return srv.wait(ticket, timeout_us)


def bfs_serve_destroy(srv: Server):
    srv.destroy()


TUNABLE_FIELDS = ("policy", "alpha", "beta", "tau_inv", "relabel", "chunk", "small_max", "bu_thread_max",
                  "bu_warp_min", "bu_chunk", "threads_per_block", "blocks_per_sm", "local_levels", "local_threads")
TUNABLE_MULTI_FIELDS = ("ms_alpha", "ms_heavy_min", "ms_ring", "ms_lanes", "ms_relabel", "ms_degree_order")
TUNABLE_GRAPHSET_FIELDS = ("threads_per_block", "blocks_per_sm", "alpha", "beta")


def params_to_dict(p: bfs_params) -> dict:
    return {k: getattr(p, k) for k, _ in bfs_params._fields_ if k != "reserved"}


def bfs_tune(g: Graph, srcs, base: bfs_params | None = None):
    """Autotune single-source parameters on sample sources; returns (params, report dict)."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    out = bfs_params()
    rep = bfs_tune_report()
    _check(load().bfs_tune(g.handle, _ptr(srcs), len(srcs), ctypes.byref(base) if base is not None else None,
                           ctypes.byref(out), ctypes.byref(rep)), "bfs_tune")
    return out, rep.as_dict()


def bfs_tune_multi(g: Graph, srcs, dist_bits: int = 8, base: bfs_params | None = None):
    """Autotune multi-source (and serving-group) parameters on one call over ``srcs``; returns (params, report)."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    out = bfs_params()
    rep = bfs_tune_report()
    _check(load().bfs_tune_multi(g.handle, _ptr(srcs), len(srcs), dist_bits,
                                 ctypes.byref(base) if base is not None else None, ctypes.byref(out),
                                 ctypes.byref(rep)), "bfs_tune_multi")
    return out, rep.as_dict()


def bfs_tune_graphset(s: GraphSet, srcs, base: bfs_params | None = None):
    """Autotune graph-set launch parameters for one run over the set; returns (params, report)."""
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    out = bfs_params()
    rep = bfs_tune_report()
    _check(load().bfs_tune_graphset(s.handle, _ptr(srcs), ctypes.byref(base) if base is not None else None,
                                    ctypes.byref(out), ctypes.byref(rep)), "bfs_tune_graphset")
    return out, rep.as_dict()


def graph_class(n: int, m: int) -> str:
    """Key of the tuning table: the paper's degree classes (Section 3: average degree below 7
    is large-diameter) split further by size."""
    avg = m / max(n, 1)
    deg = "large_diameter" if avg < 7 else ("sparse" if avg < 24 else "dense")
    return f"{deg}_n2e{max(0, int(np.log2(max(n, 1))))}"


TUNED_TABLE = os.path.join(_HERE, "tuned.json")
_KIND_FIELDS = {"single": TUNABLE_FIELDS, "multi": TUNABLE_MULTI_FIELDS, "graphset": TUNABLE_GRAPHSET_FIELDS}


def table_key(kind: str, n: int = 0, m: int = 0) -> str:
    """Entry of the tuning table: graph sets have one entry, graphs one per class and kind."""
    return "graphset" if kind == "graphset" else f"{kind}/{graph_class(n, m)}"


def tune_table_store(path: str, kind: str, params: bfs_params, report: dict, n: int = 0, m: int = 0,
                     workload: str = "") -> dict:
    """Store tuned parameters of one kind ("single", "multi", "graphset") in the JSON table at ``path``."""
    import json
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    entry = {"params": {k: getattr(params, k) for k in _KIND_FIELDS[kind]}, "report": report, "workload": workload}
    table[table_key(kind, n, m)] = entry
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return entry


def tune_table_update(path: str, g: Graph, srcs) -> dict:
    """Tune g's single-source parameters and store them under its graph class."""
    params, rep = bfs_tune(g, srcs)
    return tune_table_store(path, "single", params, rep, g.n, g.m)


def tuned_params(path: str | None = None, g: Graph | None = None, kind: str = "single", n: int = 0,
                 m: int = 0) -> bfs_params:
    """Defaults overridden by the table entry of g's class and ``kind`` (defaults when absent)."""
    import json
    path = path or TUNED_TABLE
    if g is not None:
        n, m = g.n, g.m
    p = bfs_params_default()
    if os.path.exists(path):
        with open(path) as f:
            entry = json.load(f).get(table_key(kind, n, m))
        if entry:
            for k, v in entry["params"].items():
                setattr(p, k, v)
    return p
