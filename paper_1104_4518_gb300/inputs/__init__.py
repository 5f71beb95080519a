"""Seeded synthetic inputs: edge lists and roots shaped like the paper's workloads.

The paper evaluates on R-MAT graphs with skewed degrees, edgefactor 16 and
(a, b, c, d) given as the Graph 500 values, symmetrised and randomly relabelled
(Sec. 6 and Sec. 4.4); this module also provides a high-diameter 3D grid (a
stand-in for the uk-union crawl, whose data is not available), Erdos-Renyi
graphs and small closed-form graphs for tests.

This module holds no traversal arithmetic: it only draws edge lists and roots,
so that the CPU oracle and the CUDA library can consume identical inputs
without sharing any of the method's code.  The heavy generators are plain C
(`gen.c`, pthreads), built on first use with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libbfsgen.so")
_lock = threading.Lock()
_lib = None

# Seed used for the relabelling permutation of a graph drawn with `seed`.
RELABEL_SEED_XOR = 0xA5A5A5A5A5A5A5A5

# R-MAT parameters of the paper's experiments (Sec. 6).  The printed values do
# not sum to one; a = 0.57 restores the Graph 500 set the text refers to.
RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compiles gen.c into libbfsgen.so (host code only, portable C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.gen_splitmix64_at.restype = ctypes.c_uint64
            lib.gen_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gen_rmat.restype = ctypes.c_int
            lib.gen_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, i32p, i32p]
            lib.gen_permutation.restype = ctypes.c_int
            lib.gen_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gen_apply_permutation.restype = ctypes.c_int
            lib.gen_apply_permutation.argtypes = [i32p, ctypes.c_int64, i32p, i32p]
            lib.gen_grid3d_edges.restype = ctypes.c_int64
            lib.gen_grid3d_edges.argtypes = [ctypes.c_int32]
            lib.gen_grid3d.restype = ctypes.c_int
            lib.gen_grid3d.argtypes = [ctypes.c_int32, i32p, i32p]
            lib.gen_er.restype = ctypes.c_int
            lib.gen_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gen_touched.restype = ctypes.c_int
            lib.gen_touched.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_int32, u8p]
            lib.gen_roots.restype = ctypes.c_int32
            lib.gen_roots.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gen_set_threads.restype = None
            lib.gen_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def splitmix64_at(seed: int, i: int) -> int:
    """The i-th output (i >= 0) of SplitMix64 seeded with `seed`."""
    return int(_load().gen_splitmix64_at(seed & 0xFFFFFFFFFFFFFFFF, i))


class EdgeList:
    """An undirected edge list on vertices 0..n-1 as two int32 arrays.

    Self-loops and repeated pairs may be present; CSR construction removes them.
    """

    def __init__(self, n: int, src: np.ndarray, dst: np.ndarray, name: str = ""):
        assert src.shape == dst.shape
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.name = name

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def __repr__(self) -> str:
        return f"EdgeList({self.name or 'graph'}, n={self.n}, m={self.m})"


def rmat(scale: int, edgefactor: int = 16, a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C,
         seed: int = 1, relabel: bool = True) -> EdgeList:
    """R-MAT graph with 2^scale vertices and edgefactor * 2^scale generated edges."""
    n = 1 << scale
    m = edgefactor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib = _load()
    if lib.gen_rmat(scale, m, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, _p32(src), _p32(dst)) != 0:
        raise ValueError("gen_rmat: bad arguments")
    if relabel:
        perm = permutation(n, seed ^ RELABEL_SEED_XOR)
        lib.gen_apply_permutation(_p32(perm), m, _p32(src), _p32(dst))
    return EdgeList(n, src, dst, f"rmat-s{scale}-ef{edgefactor}-a{a:g}-seed{seed}")


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded Fisher-Yates permutation of 0..n-1."""
    perm = np.empty(n, dtype=np.int32)
    _load().gen_permutation(n, seed & 0xFFFFFFFFFFFFFFFF, _p32(perm))
    return perm


def grid3d(N: int) -> EdgeList:
    """N^3 7-point grid, id = x + N*y + N*N*z, not relabelled."""
    lib = _load()
    m = int(lib.gen_grid3d_edges(N))
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if m and lib.gen_grid3d(N, _p32(src), _p32(dst)) != 0:
        raise ValueError("gen_grid3d: bad arguments")
    return EdgeList(N * N * N, src, dst, f"grid3d-{N}")


def erdos_renyi(n: int, avg_degree: float, seed: int) -> EdgeList:
    """G(n, m) with m = n * avg_degree / 2 uniform pairs."""
    m = int(n * avg_degree / 2)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if _load().gen_er(n, m, seed & 0xFFFFFFFFFFFFFFFF, _p32(src), _p32(dst)) != 0:
        raise ValueError("gen_er: bad arguments")
    return EdgeList(n, src, dst, f"er-{n}-d{avg_degree:g}-seed{seed}")


def touched(g: EdgeList) -> np.ndarray:
    """uint8[n]: 1 where the vertex has at least one non-loop edge."""
    h = np.empty(g.n, dtype=np.uint8)
    _load().gen_touched(_p32(g.src), _p32(g.dst), g.m, g.n, h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return h


def roots(g: EdgeList, k: int, seed: int) -> np.ndarray:
    """k distinct seeded roots of degree >= 1 (fewer if the graph has fewer)."""
    h = touched(g)
    out = np.empty(max(k, 0), dtype=np.int32)
    got = _load().gen_roots(h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), g.n, k,
                            seed & 0xFFFFFFFFFFFFFFFF, _p32(out))
    return out[:got].copy()


# ---------------- small closed-form graphs (tests) ----------------

def _el(n, pairs, name):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return EdgeList(n, pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32), name)


def path(n: int) -> EdgeList:
    return _el(n, [(i, i + 1) for i in range(n - 1)], f"path-{n}")


def star(n: int) -> EdgeList:
    """Centre 0 joined to leaves 1..n-1."""
    return _el(n, [(0, i) for i in range(1, n)], f"star-{n}")


def binary_tree(n: int) -> EdgeList:
    """Complete binary tree in heap order: i joined to (i-1)//2."""
    return _el(n, [((i - 1) // 2, i) for i in range(1, n)], f"bintree-{n}")


def cycle(n: int) -> EdgeList:
    return _el(n, [(i, (i + 1) % n) for i in range(n)], f"cycle-{n}")


def complete(n: int) -> EdgeList:
    return _el(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"complete-{n}")


def disjoint_union(graphs) -> tuple[EdgeList, np.ndarray]:
    """Block-diagonal union; returns the union and the vertex base of each part."""
    bases, src, dst, base = [], [], [], 0
    for g in graphs:
        bases.append(base)
        src.append(g.src.astype(np.int64) + base)
        dst.append(g.dst.astype(np.int64) + base)
        base += g.n
    if base > np.iinfo(np.int32).max:
        raise ValueError("union too large for int32 ids")
    s = np.concatenate(src) if src else np.empty(0, np.int64)
    d = np.concatenate(dst) if dst else np.empty(0, np.int64)
    return EdgeList(base, s.astype(np.int32), d.astype(np.int32), "union"), np.asarray(bases, dtype=np.int64)


# ---------------- the workloads of the evaluation ----------------

def workload_rmat(scale: int, n_roots: int, graph_seed: int, root_seed: int, edgefactor: int = 16):
    """R-MAT graph (A,B,C,D = .57,.19,.19,.05, relabelled) plus its seeded roots."""
    g = rmat(scale, edgefactor, seed=graph_seed)
    return g, roots(g, n_roots, root_seed)


def ragged_rmat(count: int = 32, seed: int = 5):
    """`count` R-MAT graphs (edgefactor 16) with scales drawn uniformly from 12..20, one
    seeded root each: the ragged batch of independent graphs."""
    rng = np.random.default_rng(seed)
    scales = rng.integers(12, 21, count)
    graphs = [rmat(int(sc), 16, seed=1000 * seed + i) for i, sc in enumerate(scales)]
    rts = [int(roots(g, 1, 7 + i)[0]) for i, g in enumerate(graphs)]
    return graphs, rts
