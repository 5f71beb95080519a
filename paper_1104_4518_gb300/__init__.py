"""GB300 breadth-first search: Python binding of libbfs_gb300 (include/bfs.h).

Level-synchronous BFS where each level is a sparse matrix-sparse vector
product over the (select2nd, max) semiring (Buluc & Madduri, Sec. 3.2,
Algorithm 3), run by hand-written sm_103a kernels behind a C ABI.  This module
only marshals arguments: torch tensors supply device memory, torch streams
supply ordering, and every step of the traversal runs in the library's
kernels.  There is no CPU fallback: if the library is missing or cannot run,
the calls raise.

The function names are those of the C ABI.  Device tensors are passed as
device pointers; host (CPU) tensors or NumPy arrays select the library's
BFS_HOST_PTRS paths where the C ABI offers them.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BFS_BOUNDS_CHECK=1 in the environment selects the bounds-checking build
# (every device index checked, BFS_ERR_BOUNDS) for the whole process.
BOUNDS_CHECKED = os.environ.get("BFS_BOUNDS_CHECK", "0") == "1"
LIB_PATH = os.path.join(_HERE, "libbfs_gb300_checked.so" if BOUNDS_CHECKED else "libbfs_gb300.so")

BFS_OK = 0
BFS_ERR_INVALID_ARG = 1
BFS_ERR_INVALID_GRAPH = 2
BFS_ERR_OOM = 3
BFS_ERR_CUDA = 4
BFS_ERR_TIMEOUT = 5
BFS_ERR_UNSUPPORTED = 6
BFS_ERR_BOUNDS = 7

BFS_HOST_PTRS = 0x1
BFS_VALIDATE = 0x2
BFS_DIRECTED = 0x4
BFS_HOST_ASYNC = 0x8

BFS_VARIANT_TD_THREAD = 0
BFS_VARIANT_TD_WARP = 1
BFS_VARIANT_TD_BINNED = 2
BFS_VARIANT_PULL = 3
BFS_VARIANT_TILED = 4
BFS_NUM_VARIANTS = 5
VARIANT_NAMES = ("td_thread", "td_warp", "td_binned", "pull", "tiled")

BFS_SELECT_HEURISTIC = 0
BFS_SELECT_LEARNED = 1
BFS_SELECT_FORCED = 2
BFS_SELECT_SCHEDULE = 3

BFS_MLP_PARAMS = 5252
BFS_MLP_IN = 12
BFS_MLP_OUT = 4


class BfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bfs status {code}: {msg}")
        self.code = code


class bfs_level_stat(ctypes.Structure):
    _fields_ = [("frontier_count", ctypes.c_int64), ("frontier_edges", ctypes.c_int64),
                ("bin_count", ctypes.c_int64 * 3), ("unvisited_count", ctypes.c_int64),
                ("unvisited_edges", ctypes.c_int64), ("time_ns", ctypes.c_int64),
                ("variant", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bfs_tuning(ctypes.Structure):
    _fields_ = [("warp_degree", ctypes.c_int32), ("cta_degree", ctypes.c_int32),
                ("pull_thread_degree", ctypes.c_int32), ("chunk_degree", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("batch_topdown_limit", ctypes.c_int32), ("small_frontier", ctypes.c_int32),
                ("batch_width", ctypes.c_int32), ("narrow_edges", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class bfs_tile_info(ctypes.Structure):
    _fields_ = [("rb_bits", ctypes.c_int32), ("cb_bits", ctypes.c_int32), ("nrb", ctypes.c_int32),
                ("ncb", ctypes.c_int32), ("ntiles", ctypes.c_int64), ("nzc", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("tdir_jc", ctypes.c_void_p), ("tdir_ir", ctypes.c_void_p), ("jc", ctypes.c_void_p),
                ("cp", ctypes.c_void_p), ("ir", ctypes.c_void_p)]


class bfs_half_info(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("adj", ctypes.c_void_p)]


class bfs_opts(ctypes.Structure):
    _fields_ = [("selector", ctypes.c_int32), ("forced_variant", ctypes.c_int32),
                ("schedule", ctypes.POINTER(ctypes.c_int32)), ("schedule_len", ctypes.c_int32),
                ("max_stat_levels", ctypes.c_int32), ("stats", ctypes.POINTER(bfs_level_stat)),
                ("nlevels_out", ctypes.POINTER(ctypes.c_int32)), ("edges_out", ctypes.POINTER(ctypes.c_int64)),
                ("spin_limit", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def _declare(lib):
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    f32 = ctypes.c_float
    sig = {
        "bfs_graph_create": [vp, vp, i32, i64, u32, ctypes.POINTER(vp)],
        "bfs_graph_create_from_edges": [vp, vp, i64, i32, u32, vp, ctypes.POINTER(vp)],
        "bfs_graph_union": [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)],
        "bfs_graph_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "bfs_graph_csr": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)],
        "bfs_graph_copy_csr": [vp, vp, vp, u32],
        "bfs_run": [vp, i32, vp, vp, ctypes.POINTER(bfs_opts), vp],
        "bfs_run_batch": [vp, ctypes.POINTER(i32), i32, vp, vp, ctypes.POINTER(bfs_opts), vp],
        "bfs_run_ragged": [vp, ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.POINTER(vp),
                           ctypes.POINTER(bfs_opts), vp],
        "bfs_sync": [vp, vp],
        "bfs_run_static": [vp, vp, i32, i64, i32, vp, vp, vp],
        "bfs_graph_tiles": [vp, i32, i32, ctypes.POINTER(bfs_tile_info), vp],
        "bfs_spmsv_sorted": [vp, vp, i32, vp, vp, vp, ctypes.POINTER(i32), vp],
        "bfs_run_sorted": [vp, i32, vp, vp, vp],
        "bfs_graph_half": [vp, ctypes.POINTER(bfs_half_info), vp],
        "bfs_run_half": [vp, i32, vp, vp, vp],
        "bfs_set_tuning": [vp, ctypes.POINTER(bfs_tuning)],
        "bfs_get_tuning": [vp, ctypes.POINTER(bfs_tuning)],
        "bfs_autotune": [vp, ctypes.POINTER(i32), i32, ctypes.POINTER(bfs_tuning), vp],
        "bfs_mlp_forward": [vp, vp, i32, vp, vp],
        "bfs_mlp_loss_grad": [vp, vp, vp, i32, vp, vp, vp],
        "bfs_mlp_adam": [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp],
        "bfs_selector_train": [vp, vp, vp, i32, i32, f32, vp, vp],
        "bfs_selector_collect": [vp, ctypes.POINTER(i32), i32, i32, vp, vp, i32, ctypes.POINTER(i32), vp],
        "bfs_selector_set_params": [vp],
        "bfs_selector_load": [ctypes.c_char_p],
        "bfs_selector_save": [ctypes.c_char_p],
        "bfs_level_features": [i32, i64, i32, i64, i64, i64, i64, ctypes.POINTER(i64), ctypes.POINTER(f32)],
        "bfs_bounds_checked": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.bfs_graph_destroy.argtypes = [vp]
    lib.bfs_graph_destroy.restype = None
    lib.bfs_last_error.restype = ctypes.c_char_p
    lib.bfs_version.restype = ctypes.c_char_p


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
            l = ctypes.CDLL(LIB_PATH)
            _declare(l)
            _lib = l
    return _lib


def _check(code: int):
    if code != BFS_OK:
        raise BfsError(code, lib().bfs_last_error().decode(errors="replace"))


# ---------------- argument helpers ----------------

def _torch():
    import torch  # imported lazily so that CPU-only users of the inputs/oracle never need it
    return torch


def _ptr_and_host(a, dtype_name: str):
    """(pointer, is_host) of a contiguous torch tensor or NumPy array of the given dtype."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype_name) or not a.flags.c_contiguous:
            raise TypeError(f"expected a contiguous {dtype_name} array")
        return a.ctypes.data, True
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.dtype != getattr(torch, dtype_name) or not a.is_contiguous():
            raise TypeError(f"expected a contiguous torch.{dtype_name} tensor")
        return a.data_ptr(), not a.is_cuda
    raise TypeError(f"expected a torch tensor or NumPy array, got {type(a)}")


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Graph:
    """Owning handle of a bfs_graph (destroyed with the object)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("graph already destroyed")
        return self._h

    def info(self):
        n, nnz, parts = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().bfs_graph_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(parts)))
        return n.value, nnz.value, parts.value

    @property
    def n(self) -> int:
        return self.info()[0]

    @property
    def nnz(self) -> int:
        return self.info()[1]

    @property
    def parts(self) -> int:
        return self.info()[2]

    def destroy(self):
        if self._h:
            lib().bfs_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------- graph construction ----------------

def bfs_graph_create(offsets, adj, validate: bool = False, directed: bool = False) -> Graph:
    """Graph from a CSR (int64 offsets[n+1], int32 adj[nnz]) on device or host; with
    `directed`, row u lists the heads of the arcs u -> v (BFS_DIRECTED)."""
    po, ho = _ptr_and_host(offsets, "int64")
    pa, ha = _ptr_and_host(adj, "int32")
    if ho != ha:
        raise ValueError("offsets and adj must both be host or both be device memory")
    n = int(offsets.shape[0]) - 1
    nnz = int(adj.shape[0])
    flags = (BFS_HOST_PTRS if ho else 0) | (BFS_VALIDATE if validate else 0) | (BFS_DIRECTED if directed else 0)
    h = ctypes.c_void_p()
    _check(lib().bfs_graph_create(po, pa, n, nnz, flags, ctypes.byref(h)))
    return Graph(h)


def bfs_graph_create_from_edges(src, dst, n: int, stream=None, directed: bool = False) -> Graph:
    """Graph from an edge list (int32 src/dst) on device or host: undirected, or the
    arcs src -> dst with `directed` (BFS_DIRECTED)."""
    ps, hs = _ptr_and_host(src, "int32")
    pd, hd = _ptr_and_host(dst, "int32")
    if hs != hd:
        raise ValueError("src and dst must both be host or both be device memory")
    h = ctypes.c_void_p()
    flags = (BFS_HOST_PTRS if hs else 0) | (BFS_DIRECTED if directed else 0)
    _check(lib().bfs_graph_create_from_edges(ps, pd, int(src.shape[0]), int(n), flags,
                                             _stream_handle(stream), ctypes.byref(h)))
    return Graph(h)


def bfs_graph_union(graphs, stream=None) -> Graph:
    """Block-diagonal union of several graphs (for bfs_run_ragged)."""
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    h = ctypes.c_void_p()
    _check(lib().bfs_graph_union(arr, len(graphs), _stream_handle(stream), ctypes.byref(h)))
    return Graph(h)


def bfs_graph_copy_csr(g: Graph, device: bool = True):
    """Copy of the graph's CSR as (offsets int64[n+1], adj int32[nnz]) tensors."""
    torch = _torch()
    n, nnz, _ = g.info()
    dev = "cuda" if device else "cpu"
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    adj = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    _check(lib().bfs_graph_copy_csr(g.handle, off.data_ptr(), adj.data_ptr(), 0 if device else BFS_HOST_PTRS))
    return off, adj[:nnz]


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (only ever copied from)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _device_copy_to_host(ptr, count: int, typestr: str, view_dtype):
    torch = _torch()
    if count <= 0:
        return np.zeros(0, dtype=view_dtype)
    t = torch.as_tensor(_DeviceArray(ptr, count, typestr), device="cuda")
    return t.cpu().numpy().view(view_dtype).copy()


def bfs_graph_tiles(g: Graph, rb_bits: int = 0, cb_bits: int = 0, stream=None, host_copy: bool = True) -> dict:
    """The graph's 2D DCSC tiles (built when absent or when the bits differ; 0 = default).

    Returns the layout and, with host_copy, NumPy copies of tdir_jc, tdir_ir
    (int64), jc (uint16), cp (uint32) and ir (uint16)."""
    info = bfs_tile_info()
    _check(lib().bfs_graph_tiles(g.handle, int(rb_bits), int(cb_bits), ctypes.byref(info), _stream_handle(stream)))
    out = {f: getattr(info, f) for f in ("rb_bits", "cb_bits", "nrb", "ncb", "ntiles", "nzc", "nnz")}
    if host_copy:
        T, nzc, nnz = info.ntiles, info.nzc, info.nnz
        out["tdir_jc"] = _device_copy_to_host(info.tdir_jc, T + 1, "<i8", np.int64)
        out["tdir_ir"] = _device_copy_to_host(info.tdir_ir, T + 1, "<i8", np.int64)
        out["jc"] = _device_copy_to_host(info.jc, nzc, "<i2", np.uint16)
        out["cp"] = _device_copy_to_host(info.cp, nzc, "<i4", np.uint32)
        out["ir"] = _device_copy_to_host(info.ir, nnz, "<i2", np.uint16)
    return out


def _device_ptr(a, dtype_name: str, what: str) -> int:
    p, host = _ptr_and_host(a, dtype_name)
    if host:
        raise ValueError(f"{what} must be device memory")
    return p


def bfs_spmsv_sorted(g: Graph, frontier, out_idx, out_val, visited=None, stream=None) -> int:
    """One masked SpMSV step with sorted output (device tensors); returns the entry count.

    visited: an int32 device tensor holding the uint32 bitmap words, or None (no mask)."""
    nf = int(frontier.shape[0])
    pf = _device_ptr(frontier, "int32", "frontier")
    pv = 0 if visited is None else _device_ptr(visited, "int32", "visited")
    cnt = ctypes.c_int32()
    _check(lib().bfs_spmsv_sorted(g.handle, pf, nf, pv or None, _device_ptr(out_idx, "int32", "out_idx"),
                                  _device_ptr(out_val, "int32", "out_val"), ctypes.byref(cnt), _stream_handle(stream)))
    return cnt.value


def spmsv_sorted(g: Graph, frontier, visited=None, stream=None):
    """t = A (x) f masked by not(visited), as (indices ascending, values) device tensors."""
    torch = _torch()
    idx = torch.empty(g.n, dtype=torch.int32, device="cuda")
    val = torch.empty(g.n, dtype=torch.int32, device="cuda")
    cnt = bfs_spmsv_sorted(g, frontier, idx, val, visited, stream)
    return idx[:cnt], val[:cnt]


def bfs_run_sorted(g: Graph, source: int, parent_out, level_out, stream=None):
    """BFS of sorted-output SpMSV steps (device outputs int32[n])."""
    _check(lib().bfs_run_sorted(g.handle, int(source), _device_ptr(parent_out, "int32", "parent_out"),
                                _device_ptr(level_out, "int32", "level_out"), _stream_handle(stream)))


def run_sorted(g: Graph, source: int, stream=None):
    torch = _torch()
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    bfs_run_sorted(g, source, parent, level, stream)
    return parent, level


def bfs_graph_half(g: Graph, stream=None, host_copy: bool = True) -> dict:
    """The graph's symmetric half storage (row v: its entries above v), built on first use;
    with host_copy, NumPy copies of offsets (int64[n + 1]) and adj (int32[nnz])."""
    info = bfs_half_info()
    _check(lib().bfs_graph_half(g.handle, ctypes.byref(info), _stream_handle(stream)))
    out = {"nnz": info.nnz}
    if host_copy:
        out["offsets"] = _device_copy_to_host(info.offsets, g.n + 1, "<i8", np.int64)
        out["adj"] = _device_copy_to_host(info.adj, info.nnz, "<i4", np.int32)
    return out


def bfs_run_half(g: Graph, source: int, parent_out, level_out, stream=None):
    """BFS that reads only the half storage (device outputs int32[n])."""
    _check(lib().bfs_run_half(g.handle, int(source), _device_ptr(parent_out, "int32", "parent_out"),
                              _device_ptr(level_out, "int32", "level_out"), _stream_handle(stream)))


def run_half(g: Graph, source: int, stream=None):
    torch = _torch()
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    bfs_run_half(g, source, parent, level, stream)
    return parent, level


# ---------------- options ----------------

class RunOptions:
    """Python side of bfs_opts; keeps the buffers the C struct points into alive."""

    def __init__(self, selector: int = BFS_SELECT_HEURISTIC, forced_variant: int = 0, schedule=None,
                 stats_levels: int = 0, want_counts: bool = False, spin_limit: int = 0, host_outputs=False,
                 host_async=False):
        self.c = bfs_opts()
        self.c.selector = selector
        self.c.forced_variant = forced_variant
        self._schedule = None
        if schedule is not None:
            self._schedule = (ctypes.c_int32 * len(schedule))(*[int(v) for v in schedule])
            self.c.schedule = self._schedule
            self.c.schedule_len = len(schedule)
        self._stats = None
        if stats_levels > 0:
            self._stats = (bfs_level_stat * stats_levels)()
            self.c.stats = self._stats
            self.c.max_stat_levels = stats_levels
        self._nl = ctypes.c_int32(0)
        self._edges = ctypes.c_int64(0)
        if want_counts or stats_levels > 0:
            self.c.nlevels_out = ctypes.pointer(self._nl)
            self.c.edges_out = ctypes.pointer(self._edges)
        self.c.spin_limit = spin_limit
        self.c.flags = (BFS_HOST_PTRS if host_outputs else 0) | (BFS_HOST_ASYNC if host_outputs and host_async else 0)

    @property
    def nlevels(self) -> int:
        return self._nl.value

    @property
    def edges(self) -> int:
        return self._edges.value

    def stats(self) -> list[dict]:
        out = []
        if self._stats is None:
            return out
        for i in range(min(self.nlevels, len(self._stats))):
            s = self._stats[i]
            out.append({"frontier_count": s.frontier_count, "frontier_edges": s.frontier_edges,
                        "bin_count": list(s.bin_count), "unvisited_count": s.unvisited_count,
                        "unvisited_edges": s.unvisited_edges, "time_ns": s.time_ns, "variant": s.variant})
        return out


def _opts_ptr(opts):
    if opts is None:
        return None
    return ctypes.byref(opts.c)


# ---------------- traversals ----------------

def bfs_run(g: Graph, source: int, parent_out, level_out, opts: RunOptions | None = None, stream=None):
    """One BFS from `source` into parent_out / level_out (int32[n], device, or host with host_outputs)."""
    pp, hp = _ptr_and_host(parent_out, "int32")
    pl, hl = _ptr_and_host(level_out, "int32")
    if (hp or hl) and not (opts is not None and opts.c.flags & BFS_HOST_PTRS):
        raise ValueError("host outputs need RunOptions(host_outputs=True)")
    _check(lib().bfs_run(g.handle, int(source), pp, pl, _opts_ptr(opts), _stream_handle(stream)))


def bfs_run_batch(g: Graph, sources, parent_out, level_out, opts: RunOptions | None = None, stream=None):
    """BFS from k sources at once; outputs root-major int32[k][n]."""
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    pp, _ = _ptr_and_host(parent_out, "int32")
    pl, _ = _ptr_and_host(level_out, "int32")
    _check(lib().bfs_run_batch(g.handle, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(src.shape[0]),
                               pp, pl, _opts_ptr(opts), _stream_handle(stream)))


def bfs_run_ragged(u: Graph, sources, parent_outs, level_outs, opts: RunOptions | None = None, stream=None):
    """One traversal per part of a union graph; per-part outputs in local ids."""
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    pa = (ctypes.c_void_p * len(parent_outs))(*[_ptr_and_host(t, "int32")[0] for t in parent_outs])
    la = (ctypes.c_void_p * len(level_outs))(*[_ptr_and_host(t, "int32")[0] for t in level_outs])
    _check(lib().bfs_run_ragged(u.handle, src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), pa, la,
                                _opts_ptr(opts), _stream_handle(stream)))


def bfs_run_static(offsets, adj, source: int, parent_out, level_out, stream=None):
    """BFS that allocates nothing: CSR and outputs are caller device tensors; the
    library's scratch is a fixed static array (n <= 1,048,576, nnz <= 67,108,864).
    Synchronous; raises on a device-side timeout."""
    _check(lib().bfs_run_static(offsets.data_ptr(), adj.data_ptr(), int(offsets.shape[0]) - 1, int(adj.shape[0]),
                                int(source), parent_out.data_ptr(), level_out.data_ptr(), _stream_handle(stream)))


def bfs_sync(g: Graph, stream=None):
    """Waits for the stream; raises the device status of the last run on it."""
    _check(lib().bfs_sync(g.handle, _stream_handle(stream)))


def bfs_set_tuning(g: Graph, **knobs):
    t = bfs_get_tuning(g)
    for k, v in knobs.items():
        setattr(t, k, v)
    _check(lib().bfs_set_tuning(g.handle, ctypes.byref(t)))


def bfs_get_tuning(g: Graph) -> bfs_tuning:
    t = bfs_tuning()
    _check(lib().bfs_get_tuning(g.handle, ctypes.byref(t)))
    return t


def bfs_autotune(g: Graph, roots, stream=None) -> bfs_tuning:
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    t = bfs_tuning()
    _check(lib().bfs_autotune(g.handle, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(r.shape[0]),
                              ctypes.byref(t), _stream_handle(stream)))
    return t


def graph_class(g: Graph) -> str:
    """Cache key of a graph's tuning: the size class (log2 n, average degree)."""
    n, nnz, _ = g.info()
    import math
    return f"n2^{max(0, int(round(math.log2(max(n, 1)))))}-deg{int(round(nnz / max(n, 1)))}"


def bfs_autotune_cached(g: Graph, roots, cache_path: str, stream=None) -> bfs_tuning:
    """bfs_autotune with a JSON cache keyed by (graph class, GPU name): a hit sets the
    cached tuning on the graph without timing anything."""
    import json
    torch = _torch()
    key = f"{graph_class(g)}|{torch.cuda.get_device_name()}"
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        bfs_set_tuning(g, **cache[key])
        return bfs_get_tuning(g)
    t = bfs_autotune(g, roots, stream)
    cache[key] = t.as_dict()
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return t


# ---------------- selector network ----------------

def bfs_mlp_forward(params, X, Y, stream=None):
    _check(lib().bfs_mlp_forward(params.data_ptr(), X.data_ptr(), int(X.shape[0]), Y.data_ptr(),
                                 _stream_handle(stream)))


def bfs_mlp_loss_grad(params, X, T, grad, loss, stream=None):
    _check(lib().bfs_mlp_loss_grad(params.data_ptr(), X.data_ptr(), T.data_ptr(), int(X.shape[0]),
                                   grad.data_ptr(), loss.data_ptr() if loss is not None else None,
                                   _stream_handle(stream)))


def bfs_mlp_adam(params, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().bfs_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), int(t), lr, beta1,
                              beta2, eps, _stream_handle(stream)))


def bfs_selector_train(params, X, T, steps: int, lr: float = 1e-3, loss_history=None, stream=None):
    _check(lib().bfs_selector_train(params.data_ptr(), X.data_ptr(), T.data_ptr(), int(X.shape[0]), int(steps),
                                    float(lr), loss_history.data_ptr() if loss_history is not None else None,
                                    _stream_handle(stream)))


def bfs_selector_collect(g: Graph, roots, reps: int = 3, max_rows: int = 65536, stream=None):
    """Per-level training rows (features X [rows,12], log2 level-time targets T [rows,4])."""
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    X = np.zeros((max_rows, BFS_MLP_IN), dtype=np.float32)
    T = np.zeros((max_rows, BFS_MLP_OUT), dtype=np.float32)
    rows = ctypes.c_int32(0)
    _check(lib().bfs_selector_collect(g.handle, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(r.shape[0]),
                                      int(reps), X.ctypes.data, T.ctypes.data, max_rows, ctypes.byref(rows),
                                      _stream_handle(stream)))
    return X[:rows.value].copy(), T[:rows.value].copy()


def bfs_selector_set_params(params):
    """Sets (host float32[5252]) or clears (None) the learned selector network."""
    if params is None:
        _check(lib().bfs_selector_set_params(None))
        return
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if a.shape != (BFS_MLP_PARAMS,):
        raise ValueError("expected 5252 parameters")
    _check(lib().bfs_selector_set_params(a.ctypes.data))


def bfs_selector_load(path: str):
    _check(lib().bfs_selector_load(path.encode()))


def bfs_selector_save(path: str):
    _check(lib().bfs_selector_save(path.encode()))


def bfs_level_features(n, nnz, k, frontier_count, frontier_edges, unvisited_count, unvisited_edges, bins):
    b = (ctypes.c_int64 * 3)(*[int(x) for x in bins])
    out = (ctypes.c_float * 12)()
    _check(lib().bfs_level_features(int(n), int(nnz), int(k), int(frontier_count), int(frontier_edges),
                                    int(unvisited_count), int(unvisited_edges), b, out))
    return np.array(list(out), dtype=np.float32)


def bfs_version() -> str:
    return lib().bfs_version().decode()


def bfs_bounds_checked() -> bool:
    """True when the loaded library is the bounds-checking build."""
    return bool(lib().bfs_bounds_checked())


# ---------------- conveniences over the C ABI ----------------

def run(g: Graph, source: int, opts: RunOptions | None = None, stream=None):
    """Allocates device outputs and runs bfs_run; returns (parent, level) tensors."""
    torch = _torch()
    n = g.n
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs_run(g, source, parent, level, opts, stream)
    return parent, level


def run_batch(g: Graph, sources, opts: RunOptions | None = None, stream=None):
    torch = _torch()
    k, n = len(sources), g.n
    parent = torch.empty((k, n), dtype=torch.int32, device="cuda")
    level = torch.empty((k, n), dtype=torch.int32, device="cuda")
    bfs_run_batch(g, sources, parent, level, opts, stream)
    return parent, level
