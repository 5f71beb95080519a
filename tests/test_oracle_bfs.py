"""Pins for the CPU oracle's BFS: brute force, closed forms, invariants, library routines.

Nothing here compares the oracle with itself: distances come from Floyd-Warshall
or SciPy's csgraph, components from SciPy, and levels/parents of structured
graphs from their closed forms.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1104_4518_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def floyd_warshall(n, pairs):
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    for u, v in pairs:
        if u != v:
            D[u, v] = D[v, u] = 1.0
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def expected_from_distances(n, pairs, D, s):
    """Levels and max-id parents implied by a distance matrix (Sec. 2.1, Sec. 3.2)."""
    nbrs = [set() for _ in range(n)]
    for u, v in pairs:
        if u != v:
            nbrs[u].add(v)
            nbrs[v].add(u)
    level = np.array([int(D[s, v]) if np.isfinite(D[s, v]) else -1 for v in range(n)], dtype=np.int32)
    parent = np.full(n, -1, dtype=np.int32)
    parent[s] = s
    for v in range(n):
        if level[v] > 0:
            parent[v] = max(u for u in nbrs[v] if level[u] == level[v] - 1)
    return level, parent


def run_oracle(n, pairs, s):
    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    g = oracle.csr(pairs[:, 0].copy(), pairs[:, 1].copy(), n)
    level, parent, nl = oracle.bfs(g, s)
    return g, level, parent, nl


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_graphs_vs_floyd_warshall(n):
    all_pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(all_pairs)):
        pairs = [p for i, p in enumerate(all_pairs) if mask >> i & 1]
        D = floyd_warshall(n, pairs)
        for s in range(n):
            _, level, parent, nl = run_oracle(n, pairs if pairs else np.zeros((0, 2)), s)
            el, ep = expected_from_distances(n, pairs, D, s)
            assert np.array_equal(level, el), (n, pairs, s)
            assert np.array_equal(parent, ep), (n, pairs, s)
            assert nl == int(el.max()) + 1


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_vs_floyd_warshall(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 65))
    m = int(rng.integers(0, 3 * n))
    pairs = rng.integers(0, n, size=(m, 2))  # includes self-loops and repeats
    D = floyd_warshall(n, [tuple(p) for p in pairs])
    for s in rng.choice(n, size=min(n, 6), replace=False):
        _, level, parent, _ = run_oracle(n, pairs, int(s))
        el, ep = expected_from_distances(n, [tuple(p) for p in pairs], D, int(s))
        assert np.array_equal(level, el)
        assert np.array_equal(parent, ep)


def test_rmat_small_vs_floyd_warshall():
    g = inputs.rmat(6, 16, seed=11)
    pairs = list(zip(g.src.tolist(), g.dst.tolist()))
    D = floyd_warshall(g.n, pairs)
    for s in inputs.roots(g, 8, 12):
        _, level, parent, _ = run_oracle(g.n, pairs, int(s))
        el, ep = expected_from_distances(g.n, pairs, D, int(s))
        assert np.array_equal(level, el) and np.array_equal(parent, ep)


# ---------------- closed forms ----------------

def oracle_on(el, s):
    g = oracle.csr_of(el)
    level, parent, nl = oracle.bfs(g, s)
    return level, parent, nl


@pytest.mark.parametrize("n", [1, 2, 7, 100])
def test_path(n):
    level, parent, nl = oracle_on(inputs.path(n), 0)
    assert np.array_equal(level, np.arange(n))
    assert np.array_equal(parent, np.maximum(np.arange(n) - 1, 0))
    assert nl == n


def test_star_centre_and_leaf():
    n = 9
    level, parent, _ = oracle_on(inputs.star(n), 0)
    assert level[0] == 0 and (level[1:] == 1).all() and (parent == 0).all()
    level, parent, _ = oracle_on(inputs.star(n), 4)
    assert level[4] == 0 and level[0] == 1 and parent[0] == 4 and parent[4] == 4
    others = [v for v in range(1, n) if v != 4]
    assert (level[others] == 2).all() and (parent[others] == 0).all()


@pytest.mark.parametrize("n", [1, 2, 15, 31, 100])
def test_complete_binary_tree(n):
    level, parent, _ = oracle_on(inputs.binary_tree(n), 0)
    i = np.arange(n)
    assert np.array_equal(level, np.floor(np.log2(i + 1)).astype(np.int32))
    exp = np.maximum((i - 1) // 2, 0)
    assert np.array_equal(parent, exp)


@pytest.mark.parametrize("n", [3, 4, 9, 10, 64, 65])
def test_cycle_levels_and_tiebreak(n):
    level, parent, _ = oracle_on(inputs.cycle(n), 0)
    for v in range(1, n):
        d = min(v, n - v)
        assert level[v] == d
        if v < n - v:
            assert parent[v] == v - 1
        elif v > n - v:
            assert parent[v] == (v + 1) % n
        else:  # antipode of an even cycle: two parents one level up, the larger wins
            assert parent[v] == v + 1


@pytest.mark.parametrize("n", [2, 5, 17])
def test_complete_graph(n):
    for s in (0, n - 1):
        level, parent, _ = oracle_on(inputs.complete(n), s)
        exp = np.ones(n, dtype=np.int32)
        exp[s] = 0
        assert np.array_equal(level, exp) and (parent == s).all()


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_grid3d_corner(N):
    level, parent, _ = oracle_on(inputs.grid3d(N), 0)
    for v in range(N ** 3):
        x, y, z = v % N, (v // N) % N, v // (N * N)
        assert level[v] == x + y + z
        # the neighbours one level up are v-1 (x>0), v-N (y>0), v-N*N (z>0);
        # the largest id is the one with the smallest decrement
        if v == 0:
            assert parent[v] == 0
        elif x > 0:
            assert parent[v] == v - 1
        elif y > 0:
            assert parent[v] == v - N
        else:
            assert parent[v] == v - N * N


def test_disjoint_union_unreached():
    u, bases = inputs.disjoint_union([inputs.path(5), inputs.star(4), inputs.cycle(6)])
    level, parent, _ = oracle_on(u, int(bases[1]) + 2)
    inside = np.zeros(u.n, bool)
    inside[bases[1]:bases[1] + 4] = True
    assert (level[~inside] == -1).all() and (parent[~inside] == -1).all()
    assert (level[inside] >= 0).all()


def test_isolated_source():
    el = inputs.EdgeList(4, np.array([1], np.int32), np.array([2], np.int32))
    level, parent, nl = oracle_on(el, 0)
    assert level.tolist() == [0, -1, -1, -1] and parent.tolist() == [0, -1, -1, -1] and nl == 1


# ---------------- invariants and library routines at larger sizes ----------------

@pytest.mark.parametrize("scale,seed", [(10, 3), (12, 4), (13, 5)])
def test_rmat_invariants_and_scipy(scale, seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    el = inputs.rmat(scale, 16, seed=seed)
    g = oracle.csr_of(el)
    n = g.n
    A = sp.csr_matrix((np.ones(g.nnz), g.adj, g.offsets), shape=(n, n))
    ncomp, labels = csgraph.connected_components(A, directed=False)
    src_row = np.repeat(np.arange(n), g.degree())
    for s in inputs.roots(el, 4, seed + 100):
        level, parent, nl = oracle.bfs(g, int(s))
        dist = csgraph.shortest_path(A, method="D", unweighted=True, indices=int(s))
        exp = np.where(np.isfinite(dist), dist, -1).astype(np.int32)
        assert np.array_equal(level, exp)
        # reached set = connected component of s
        assert np.array_equal(level >= 0, labels == labels[s])
        # every edge's endpoint levels differ by at most one
        lu, lv = level[src_row], level[g.adj]
        assert (np.abs(lu - lv)[lu >= 0] <= 1).all()
        # parent one level up, adjacent, and the largest such neighbour
        reached = np.nonzero(level > 0)[0]
        assert (level[parent[reached]] == level[reached] - 1).all()
        cand = np.where(level[g.adj] == level[src_row] - 1, g.adj, -1)
        best = np.full(n, -1, dtype=np.int64)
        np.maximum.at(best, src_row, cand)
        assert np.array_equal(parent[reached], best[reached].astype(np.int32))
        assert parent[s] == s and (parent[level < 0] == -1).all()
        # frontier sizes sum to the reached count
        count, edges = oracle.level_stats(g, level, nl)
        assert count.sum() == (level >= 0).sum() and (count > 0).all()
        assert edges.sum() == g.degree()[level >= 0].sum()
        assert oracle.component_edges(g, level) * 2 == edges.sum()


# ---------------- Algorithm 3 form and the Fig. 3 worked example ----------------

def test_fig3_spmsv_worked_example():
    with open(os.path.join(GOLDEN, "fig3_spmsv.json")) as f:
        gold = json.load(f)
    x = {int(k): v for k, v in gold["frontier"].items()}
    y = oracle.spmsv_select2nd_max(gold["rows"], x)
    assert y == {int(k): v for k, v in gold["product_y"].items()}
    parents = [-1] * len(gold["rows"])
    for v in gold["visited"]:
        parents[v] = v
    t = oracle.mask_not(y, parents)
    assert t == {int(k): v for k, v in gold["masked_t"].items()}


@pytest.mark.parametrize("seed", range(8))
def test_algorithm3_form_matches_queue_bfs(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 200))
    m = int(rng.integers(0, 4 * n))
    pairs = rng.integers(0, n, size=(m, 2)).astype(np.int32)
    g = oracle.csr(pairs[:, 0].copy(), pairs[:, 1].copy(), n)
    rows = [g.row(v).tolist() for v in range(n)]
    for s in rng.choice(n, size=min(n, 4), replace=False):
        level, parent, _ = oracle.bfs(g, int(s))
        l3, p3 = oracle.bfs_spmsv(rows, int(s))
        assert level.tolist() == l3 and parent.tolist() == p3


def test_planted_min_id_parent_is_caught():
    """A plausible mistake (min instead of max in the parent rule) fails the cycle pin."""
    el = inputs.cycle(10)
    g = oracle.csr_of(el)
    level, parent, _ = oracle.bfs(g, 0)
    wrong = parent.copy()
    for v in range(1, 10):
        cands = [u for u in g.row(v) if level[u] == level[v] - 1]
        wrong[v] = min(cands)
    assert wrong[5] != 6 and parent[5] == 6


# ---------------- the edge-list validator ----------------

@pytest.mark.parametrize("seed", range(6))
def test_validator_accepts_floyd_warshall_results(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 60))
    pairs = rng.integers(0, n, size=(int(rng.integers(0, 3 * n)), 2))
    D = floyd_warshall(n, [tuple(p) for p in pairs])
    for s in range(min(n, 5)):
        el, ep = expected_from_distances(n, [tuple(p) for p in pairs], D, s)
        bad = oracle.validate_edges(pairs[:, 0], pairs[:, 1], n, s, el, ep)
        assert bad.sum() == 0


def test_validator_catches_planted_mistakes():
    el = inputs.rmat(10, 16, seed=21)
    g = oracle.csr_of(el)
    s = int(inputs.roots(el, 1, 22)[0])
    level, parent, _ = oracle.bfs(g, s)
    assert oracle.validate_edges(el.src, el.dst, el.n, s, level, parent).sum() == 0
    reached = np.nonzero(level > 1)[0]
    v = int(reached[0])
    lv = level.copy(); lv[v] += 1                     # a level one too large
    assert oracle.validate_edges(el.src, el.dst, el.n, s, lv, parent).sum() > 0
    lv = level.copy(); lv[v] -= 1                     # a level one too small
    assert oracle.validate_edges(el.src, el.dst, el.n, s, lv, parent).sum() > 0
    cands = [u for u in g.row(v) if level[u] == level[v] - 1]
    if len(cands) > 1:                                # a valid but non-maximal parent
        pv = parent.copy(); pv[v] = min(cands)
        assert oracle.validate_edges(el.src, el.dst, el.n, s, level, pv)[2] == 1
    un = np.nonzero(level < 0)[0]
    if un.size:                                        # an unreached vertex given a level
        lv = level.copy(); lv[un[0]] = 3
        assert oracle.validate_edges(el.src, el.dst, el.n, s, lv, parent).sum() > 0
    pv = parent.copy(); pv[s] = -1                     # the source's own parent
    assert oracle.validate_edges(el.src, el.dst, el.n, s, level, pv)[0] == 1
