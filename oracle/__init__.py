"""CPU oracle for the BFS library -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The library's product path never imports, links or
runs it, and it shares no code with the CUDA path (the seeded input generators
in `paper_1104_4518_gb300.inputs` are the only module both sides use, and they
hold none of the method's arithmetic).

Contents
  - `validate_edges`: an O(m) check of a BFS result against the edge list
    (distances and max-id parents), for sizes where building the oracle CSR
    would take minutes.
  - `csr`, `bfs`, `component_edges`, `level_stats`: ctypes wrappers over the
    plain serial C in `bfs_oracle.c` (definitions of Sec. 2.1 / Algorithm 1 and
    the max-id parent of Sec. 3.2 / Algorithm 3).
  - `spmsv_select2nd_max`, `bfs_spmsv`: Algorithm 3 on a single process written
    in pure Python (small inputs only): each level is the sparse matrix-sparse
    vector product over the (select2nd, max) semiring, masked by the parents
    vector, followed by the parent update and the frontier replacement.
  - `dcsc_tiles`: the 2D blocks of Sec. 3.2 in the doubly compressed sparse
    column form of Sec. 4.1 (arrays IR, JC, CP per block), for any block sizes.
  - `mlp` (separate module): the variant-selector network in float64 NumPy.
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
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles bfs_oracle.c (plain C, no GPU code) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_build_csr.restype = ctypes.c_int64
            lib.oracle_build_csr.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, i64p, i32p]
            lib.oracle_bfs.restype = ctypes.c_int32
            lib.oracle_bfs.argtypes = [i64p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p]
            lib.oracle_component_edges.restype = ctypes.c_int64
            lib.oracle_component_edges.argtypes = [i64p, i32p, ctypes.c_int32]
            lib.oracle_level_stats.restype = ctypes.c_int
            lib.oracle_level_stats.argtypes = [i64p, i32p, ctypes.c_int32, ctypes.c_int32, i64p, i64p]
            lib.oracle_build_digraph_csr.restype = ctypes.c_int64
            lib.oracle_build_digraph_csr.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, i64p, i32p]
            lib.oracle_bfs_directed.restype = ctypes.c_int32
            lib.oracle_bfs_directed.argtypes = [i64p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p]
            lib.oracle_out_edges.restype = ctypes.c_int64
            lib.oracle_out_edges.argtypes = [i64p, i32p, ctypes.c_int32]
            lib.oracle_validate_arcs.restype = ctypes.c_int64
            lib.oracle_validate_arcs.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p,
                                                 i32p, i32p, i64p]
            lib.oracle_validate_edges.restype = ctypes.c_int64
            lib.oracle_validate_edges.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p,
                                                  i32p, i32p, i64p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ct))


class CSR:
    """Oracle CSR: offsets int64[n+1], adj int32[nnz]."""

    def __init__(self, offsets: np.ndarray, adj: np.ndarray):
        self.offsets = offsets
        self.adj = adj

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def degree(self) -> np.ndarray:
        return np.diff(self.offsets)

    def row(self, v: int) -> np.ndarray:
        return self.adj[self.offsets[v]:self.offsets[v + 1]]


def csr(src: np.ndarray, dst: np.ndarray, n: int) -> CSR:
    """Symmetric, self-loop-free, deduplicated, row-sorted CSR (Sec. 4.1)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    offsets = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = _load().oracle_build_csr(_p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), m, n,
                                   _p(offsets, ctypes.c_int64), _p(adj, ctypes.c_int32))
    if nnz < 0:
        raise ValueError("oracle_build_csr: endpoint out of range")
    adj = adj[:nnz].copy() if nnz < 0.9 * adj.shape[0] else adj[:nnz]
    return CSR(offsets, adj)


def csr_of(g) -> CSR:
    """CSR of an `inputs.EdgeList`."""
    return csr(g.src, g.dst, g.n)


def bfs(g: CSR, s: int):
    """(level int32[n], parent int32[n], nlevels) of the BFS from s."""
    n = g.n
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    queue = np.empty(n, dtype=np.int32)
    nl = _load().oracle_bfs(_p(g.offsets, ctypes.c_int64), _p(g.adj, ctypes.c_int32), n, int(s),
                            _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32), _p(queue, ctypes.c_int32))
    if nl < 0:
        raise ValueError("oracle_bfs: bad source")
    return level, parent, int(nl)


def digraph_csr(src: np.ndarray, dst: np.ndarray, n: int) -> CSR:
    """Directed CSR: row u holds the heads of the arcs u -> v, sorted, repeats and
    self-loops dropped (the non-symmetric A of Sec. 3.2)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    offsets = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(max(m, 1), dtype=np.int32)
    nnz = _load().oracle_build_digraph_csr(_p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), m, n,
                                           _p(offsets, ctypes.c_int64), _p(adj, ctypes.c_int32))
    if nnz < 0:
        raise ValueError("oracle_build_digraph_csr: endpoint out of range")
    return CSR(offsets, adj[:nnz].copy())


def digraph_of(g) -> CSR:
    """Directed CSR of an `inputs.EdgeList` (arcs src -> dst)."""
    return digraph_csr(g.src, g.dst, g.n)


def bfs_directed(g: CSR, s: int):
    """(level, parent, nlevels) of the BFS from s along the arcs of a directed CSR:
    level = shortest directed path length, parent = largest in-neighbour one level up."""
    n = g.n
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    queue = np.empty(n, dtype=np.int32)
    nl = _load().oracle_bfs_directed(_p(g.offsets, ctypes.c_int64), _p(g.adj, ctypes.c_int32), n, int(s),
                                     _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32),
                                     _p(queue, ctypes.c_int32))
    if nl < 0:
        raise ValueError("oracle_bfs_directed: bad source")
    return level, parent, int(nl)


def out_edges(g: CSR, level: np.ndarray) -> int:
    """TEPS edge count of a directed traversal: arcs leaving reached vertices."""
    return int(_load().oracle_out_edges(_p(g.offsets, ctypes.c_int64), _p(level, ctypes.c_int32), g.n))


def bfs_many(g: CSR, sources, threads: int | None = None):
    """Runs `bfs` for every source on a thread pool (the C call drops the GIL)."""
    threads = threads or min(len(sources), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=max(threads, 1)) as ex:
        return list(ex.map(lambda s: bfs(g, int(s)), sources))


def component_edges(g: CSR, level: np.ndarray) -> int:
    """TEPS edge count: undirected edges inside the reached set (Sec. 6)."""
    return int(_load().oracle_component_edges(_p(g.offsets, ctypes.c_int64), _p(level, ctypes.c_int32), g.n))


def level_stats(g: CSR, level: np.ndarray, nlevels: int):
    """Per-level (frontier size, frontier degree sum) as two int64 arrays."""
    count = np.zeros(max(nlevels, 1), dtype=np.int64)
    edges = np.zeros(max(nlevels, 1), dtype=np.int64)
    _load().oracle_level_stats(_p(g.offsets, ctypes.c_int64), _p(level, ctypes.c_int32), g.n, nlevels,
                               _p(count, ctypes.c_int64), _p(edges, ctypes.c_int64))
    return count[:nlevels], edges[:nlevels]


def validate_edges(src, dst, n: int, s: int, level: np.ndarray, parent: np.ndarray):
    """Violations (a, b, c-parent, c-unreached) of a BFS result against an edge list.

    O(m + n) check that needs no CSR (see oracle_validate_edges in bfs_oracle.c):
    all four counts are zero exactly when `level` are the hop distances from s and
    `parent` follows the max-id rule.  The C loop drops the GIL, so several
    results can be validated on a thread pool.
    """
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    level = np.ascontiguousarray(level, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    best = np.empty(n, dtype=np.int32)
    bad = np.zeros(4, dtype=np.int64)
    r = _load().oracle_validate_edges(_p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), int(src.shape[0]), n, int(s),
                                      _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32), _p(best, ctypes.c_int32),
                                      _p(bad, ctypes.c_int64))
    if r < 0:
        raise ValueError("oracle_validate_edges: bad argument")
    return bad


def validate_arcs(src, dst, n: int, s: int, level: np.ndarray, parent: np.ndarray):
    """Violations (a, b, c, d) of a directed BFS result against the arc list src -> dst
    (see oracle_validate_arcs in bfs_oracle.c): all zero exactly when `level` are the
    directed distances from s and `parent` the largest in-neighbours one level up."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    level = np.ascontiguousarray(level, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    best = np.empty(n, dtype=np.int32)
    bad = np.zeros(4, dtype=np.int64)
    r = _load().oracle_validate_arcs(_p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), int(src.shape[0]), n, int(s),
                                     _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32), _p(best, ctypes.c_int32),
                                     _p(bad, ctypes.c_int64))
    if r < 0:
        raise ValueError("oracle_validate_arcs: bad argument")
    return bad


# ---------------- Algorithm 3 on one process, pure Python ----------------

def spmsv_select2nd_max(rows, x: dict) -> dict:
    """y = A (x) x over the (select2nd, max) semiring (Sec. 3.2).

    `rows[i]` lists the column indices j with A(i, j) != 0 (the matrix is taken
    as already transposed, as the paper assumes).  `x` maps the indices of the
    sparse vector's nonzeros to their values.  Multiplication selects the
    vector's value, addition keeps the maximum; y holds an entry for every row
    that meets at least one nonzero of x.
    """
    y = {}
    for i, cols in enumerate(rows):
        for j in cols:
            if j in x:
                val = x[j]
                if i not in y or val > y[i]:
                    y[i] = val
    return y


def mask_not(t: dict, parents) -> dict:
    """t (.) not(parents): keeps the entries of t whose vertex has no parent yet."""
    return {v: val for v, val in t.items() if parents[v] == -1}


def bfs_spmsv(rows, s: int):
    """Algorithm 3 with p = 1: returns (level, parent) as Python lists.

    f(s) <- s; while f is not empty: t <- A (x) f; t <- t (.) not(pi);
    pi <- pi + t (a masked assignment, since t only has entries where pi is
    empty); f <- t.  Frontier values are the vertices' own ids at every level,
    so t(v) is the largest frontier neighbour of v.
    """
    n = len(rows)
    parent = [-1] * n
    level = [-1] * n
    parent[s] = s
    level[s] = 0
    f = {s: s}
    k = 0
    while f:
        t = spmsv_select2nd_max(rows, f)
        t = mask_not(t, parent)
        for v, u in t.items():
            parent[v] = u
            level[v] = k + 1
        f = {v: v for v in t}
        k += 1
    return level, parent


# ---------------- 2D blocks in DCSC (Sec. 3.2, Sec. 4.1) ----------------

def dcsc_tiles(g: CSR, rows_per_block: int, cols_per_block: int) -> dict:
    """The entries of `g` split into a 2D grid of blocks, each in DCSC form.

    Entry (v, u) is "u in row v of g" (row v lists the candidate parents u of v,
    the transposed orientation Algorithm 3 multiplies with).  Block (rb, cb)
    holds the entries with v // rows_per_block == rb and u // cols_per_block ==
    cb; blocks are numbered t = rb * ncb + cb.  DCSC of a block (Sec. 4.1): JC
    lists the block's non-empty columns in ascending order, CP the start of
    each column's row ids, IR the row ids, ascending within a column; ids are
    local to the block (v mod rows_per_block, u mod cols_per_block).  Returned
    as flat arrays over all blocks in block order: tdir_jc / tdir_ir (first
    column / first entry of each block, plus one end entry), jc, cp (relative
    to the block's first entry) and ir.  A library sort orders the entries by
    (block, column, row); the rest follows the definition.
    """
    n = g.n
    nrb = (n + rows_per_block - 1) // rows_per_block
    ncb = (n + cols_per_block - 1) // cols_per_block
    T = nrb * ncb
    v = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.offsets))
    u = g.adj.astype(np.int64)
    t = (v // rows_per_block) * ncb + u // cols_per_block
    order = np.lexsort((v, u, t))
    v, u, t = v[order], u[order], t[order]
    ir = v % rows_per_block
    ul = u % cols_per_block
    new_col = np.ones(v.shape[0], dtype=bool)
    new_col[1:] = (t[1:] != t[:-1]) | (u[1:] != u[:-1])
    starts = np.nonzero(new_col)[0]
    tdir_ir = np.searchsorted(t, np.arange(T + 1), side="left").astype(np.int64)
    tdir_jc = np.searchsorted(t[starts], np.arange(T + 1), side="left").astype(np.int64)
    jc = ul[starts]
    cp = starts - tdir_ir[t[starts]]
    return {"nrb": nrb, "ncb": ncb, "ntiles": T, "nzc": int(starts.shape[0]), "tdir_jc": tdir_jc,
            "tdir_ir": tdir_ir, "jc": jc.astype(np.int64), "cp": cp.astype(np.int64), "ir": ir.astype(np.int64)}
