"""Pins for the oracle's CSR construction and for the seeded input generators."""
import numpy as np
import pytest

import oracle
from paper_1104_4518_gb300 import inputs


def set_csr(n, src, dst):
    """Naive CSR from Python sets: symmetric, no self-loops, no repeats, sorted rows."""
    rows = [set() for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            rows[u].add(v)
            rows[v].add(u)
    offsets = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        offsets[v + 1] = offsets[v] + len(rows[v])
    adj = np.array([u for v in range(n) for u in sorted(rows[v])], dtype=np.int32)
    return offsets, adj


@pytest.mark.parametrize("seed", range(10))
def test_csr_vs_set_builder(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(0, 5 * n))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    g = oracle.csr(src, dst, n)
    eo, ea = set_csr(n, src, dst)
    assert g.offsets.dtype == np.int64 and g.adj.dtype == np.int32
    assert np.array_equal(g.offsets, eo) and np.array_equal(g.adj, ea)


def test_csr_vs_scipy_on_rmat():
    sp = pytest.importorskip("scipy.sparse")
    el = inputs.rmat(11, 16, seed=7)
    g = oracle.csr_of(el)
    keep = el.src != el.dst
    r = np.concatenate([el.src[keep], el.dst[keep]])
    c = np.concatenate([el.dst[keep], el.src[keep]])
    A = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(el.n, el.n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    assert np.array_equal(g.offsets, A.indptr.astype(np.int64))
    assert np.array_equal(g.adj, A.indices.astype(np.int32))


def test_csr_empty_and_bad_input():
    g = oracle.csr(np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    assert g.offsets.tolist() == [0] * 6 and g.nnz == 0
    with pytest.raises(ValueError):
        oracle.csr(np.array([0], np.int32), np.array([5], np.int32), 5)


def test_component_edge_count_vs_unique_pairs():
    el = inputs.rmat(10, 16, seed=9)
    g = oracle.csr_of(el)
    s = int(inputs.roots(el, 1, 5)[0])
    level, _, _ = oracle.bfs(g, s)
    pairs = {(min(u, v), max(u, v)) for u, v in zip(el.src.tolist(), el.dst.tolist())
             if u != v and level[u] >= 0}
    assert oracle.component_edges(g, level) == len(pairs)


# ---------------- generators ----------------

def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014 reference generator).
    assert [inputs.splitmix64_at(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rmat_quadrant_frequencies():
    # scale 1: a single bit level, so the quadrant frequencies are (A, B, C, D) themselves
    m = 400_000
    g = inputs.rmat(1, m // 2, seed=3, relabel=False)
    freq = np.array([np.mean((g.src == i) & (g.dst == j)) for i, j in [(0, 0), (0, 1), (1, 0), (1, 1)]])
    exp = np.array([0.57, 0.19, 0.19, 0.05])
    assert np.all(np.abs(freq - exp) < 4 * np.sqrt(exp * (1 - exp) / m))


def test_rmat_deterministic_and_thread_independent():
    a = inputs.rmat(14, 16, seed=5)
    inputs._load().gen_set_threads(1)
    try:
        b = inputs.rmat(14, 16, seed=5)
    finally:
        inputs._load().gen_set_threads(0)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    c = inputs.rmat(14, 16, seed=6)
    assert not np.array_equal(a.src, c.src)
    assert a.m == 16 << 14 and a.src.min() >= 0 and a.src.max() < a.n


def test_permutation_is_permutation():
    p = inputs.permutation(100_003, 9)
    assert np.array_equal(np.sort(p), np.arange(100_003))
    assert not np.array_equal(p, np.arange(100_003))


def test_grid_edge_count_and_degrees():
    assert inputs._load().gen_grid3d_edges(128) == 6_242_304
    g = oracle.csr_of(inputs.grid3d(6))
    deg = g.degree()
    assert g.nnz == 2 * 3 * 36 * 5 and deg.max() == 6 and deg.min() == 3


def test_roots_distinct_with_edges():
    el = inputs.rmat(12, 16, seed=1)
    r = inputs.roots(el, 64, 101)
    h = inputs.touched(el)
    assert len(r) == 64 and len(set(r.tolist())) == 64 and (h[r] == 1).all()
    assert np.array_equal(r, inputs.roots(el, 64, 101))


def test_er_shape():
    el = inputs.erdos_renyi(1000, 8, seed=2)
    assert el.m == 4000 and el.src.max() < 1000
