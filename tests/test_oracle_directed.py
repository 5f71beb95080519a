"""Pins of the directed oracle (arcs u -> v; the traversal of Sec. 3.2 with a
non-symmetric A): shortest directed path lengths and the largest in-neighbour
one level up, checked against Floyd-Warshall on every digraph with 4 vertices
and on random digraphs, against closed forms, and against the undirected
oracle on symmetric digraphs.  A planted mistake (parents taken over the
out-arcs) is caught."""

import numpy as np
import pytest

import oracle


def fw_directed(n, arcs):
    """All-pairs shortest directed path lengths (np.inf when unreachable)."""
    d = np.full((n, n), np.inf)
    np.fill_diagonal(d, 0)
    for u, v in arcs:
        if u != v:
            d[u, v] = 1
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d


def expected(n, arcs, s, d, parent_over_out=False):
    """Levels and max-id parents from the distance matrix (the definitions)."""
    dist = d[s]
    level = np.where(np.isfinite(dist), dist, -1).astype(np.int32)
    parent = np.full(n, -1, np.int32)
    parent[s] = s
    for v in range(n):
        if v == s or level[v] < 0:
            continue
        if parent_over_out:  # the planted mistake: heads of v's own arcs
            cands = [w for (x, w) in arcs if x == v and level[w] == level[v] - 1]
        else:
            cands = [u for (u, w) in arcs if w == v and u != v and level[u] == level[v] - 1]
        parent[v] = max(cands)
    return level, parent


def run(n, arcs, s):
    src = np.array([a for a, _ in arcs], np.int32)
    dst = np.array([b for _, b in arcs], np.int32)
    g = oracle.digraph_csr(src, dst, n)
    lv, pa, _ = oracle.bfs_directed(g, s)
    return g, lv, pa


def test_every_digraph_on_4_vertices():
    n = 4
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    for mask in range(1 << len(pairs)):
        arcs = [p for i, p in enumerate(pairs) if (mask >> i) & 1]
        d = fw_directed(n, arcs)
        for s in range(n):
            _, lv, pa = run(n, arcs, s)
            el, ep = expected(n, arcs, s, d)
            assert np.array_equal(lv, el) and np.array_equal(pa, ep), (arcs, s)


def test_random_digraphs_against_floyd_warshall():
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(2, 49))
        m = int(rng.integers(0, 4 * n))
        arcs = [(int(a), int(b)) for a, b in zip(rng.integers(0, n, m), rng.integers(0, n, m))]
        d = fw_directed(n, arcs)
        for s in rng.integers(0, n, 3):
            _, lv, pa = run(n, arcs, int(s))
            el, ep = expected(n, arcs, int(s), d)
            assert np.array_equal(lv, el) and np.array_equal(pa, ep), (trial, int(s))


def test_closed_forms():
    n = 50
    path = [(v, v + 1) for v in range(n - 1)]
    _, lv, pa = run(n, path, 0)
    assert np.array_equal(lv, np.arange(n)) and np.array_equal(pa[1:], np.arange(n - 1)) and pa[0] == 0
    _, lv, pa = run(n, path, n - 1)  # nothing is reachable against the arcs
    assert (lv[:-1] == -1).all() and lv[-1] == 0 and (pa[:-1] == -1).all()
    cyc = path + [(n - 1, 0)]
    for s in (0, 17):
        _, lv, pa = run(n, cyc, s)
        v = np.arange(n)
        assert np.array_equal(lv, (v - s) % n)
        exp = (v - 1) % n
        exp[s] = s
        assert np.array_equal(pa, exp)
    out_star = [(0, v) for v in range(1, n)]
    _, lv, pa = run(n, out_star, 0)
    assert lv[0] == 0 and (lv[1:] == 1).all() and (pa == 0).all()
    _, lv, _ = run(n, out_star, 5)
    assert lv[5] == 0 and (np.delete(lv, 5) == -1).all()
    in_star = [(v, 0) for v in range(1, n)]
    _, lv, pa = run(n, in_star, 7)
    assert lv[7] == 0 and lv[0] == 1 and pa[0] == 7 and (np.delete(lv, [0, 7]) == -1).all()


def test_symmetric_digraph_equals_undirected_oracle():
    rng = np.random.default_rng(5)
    n, m = 300, 900
    a, b = rng.integers(0, n, m), rng.integers(0, n, m)
    src = np.concatenate([a, b]).astype(np.int32)
    dst = np.concatenate([b, a]).astype(np.int32)
    gd = oracle.digraph_csr(src, dst, n)
    gu = oracle.csr(a.astype(np.int32), b.astype(np.int32), n)
    assert np.array_equal(gd.offsets, gu.offsets) and np.array_equal(gd.adj, gu.adj)
    for s in range(0, n, 37):
        ld, pd, nd = oracle.bfs_directed(gd, s)
        lu, pu, nu = oracle.bfs(gu, s)
        assert np.array_equal(ld, lu) and np.array_equal(pd, pu) and nd == nu


def test_out_edges_counts_arcs_of_reached_vertices():
    rng = np.random.default_rng(8)
    n, m = 200, 700
    src, dst = rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32)
    g = oracle.digraph_csr(src, dst, n)
    lv, _, _ = oracle.bfs_directed(g, 3)
    assert oracle.out_edges(g, lv) == int(np.diff(g.offsets)[lv >= 0].sum())


def test_planted_direction_mistake_is_caught():
    """Parents chosen among out-neighbours instead of in-neighbours differ from the
    definition on some 4-vertex digraph, so the exhaustive pin would catch that bug."""
    n = 4
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    caught = False
    for mask in range(1 << len(pairs)):
        arcs = [p for i, p in enumerate(pairs) if (mask >> i) & 1]
        d = fw_directed(n, arcs)
        good = expected(n, arcs, 0, d)
        try:
            bad = expected(n, arcs, 0, d, parent_over_out=True)
        except ValueError:  # no out-neighbour one level up: the wrong rule has no answer at all
            caught = True
            break
        if not np.array_equal(good[1], bad[1]):
            caught = True
            break
    assert caught


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.digraph_csr(np.array([0], np.int32), np.array([5], np.int32), 3)
    g = oracle.digraph_csr(np.array([0], np.int32), np.array([1], np.int32), 3)
    with pytest.raises(ValueError):
        oracle.bfs_directed(g, 3)


def test_arc_validator_accepts_the_oracle_and_rejects_planted_mistakes():
    rng = np.random.default_rng(12)
    n, m = 400, 1600
    src, dst = rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32)
    g = oracle.digraph_csr(src, dst, n)
    for s in range(0, n, 53):
        lv, pa, _ = oracle.bfs_directed(g, s)
        assert oracle.validate_arcs(src, dst, n, s, lv, pa).sum() == 0
    s = int(src[0])
    lv, pa, _ = oracle.bfs_directed(g, s)
    reached = np.nonzero((lv > 0))[0]
    v = int(reached[len(reached) // 2])
    bad = lv.copy(); bad[v] += 1                       # a level too deep
    assert oracle.validate_arcs(src, dst, n, s, bad, pa).sum() > 0
    bad = lv.copy(); bad[v] = -1                        # a reached vertex dropped
    assert oracle.validate_arcs(src, dst, n, s, bad, pa).sum() > 0
    wrong = pa.copy()                                   # a smaller in-neighbour one level up, if any
    ins = [u for u, w in zip(src, dst) if w == v and u != v and lv[u] == lv[v] - 1]
    if len(set(ins)) > 1:
        wrong[v] = min(ins)
        assert oracle.validate_arcs(src, dst, n, s, lv, wrong)[2] == 1
    unreached = np.nonzero(lv < 0)[0]
    if unreached.size:
        wrong = pa.copy(); wrong[unreached[0]] = s       # an unreached vertex with a parent
        assert oracle.validate_arcs(src, dst, n, s, lv, wrong)[3] == 1
    # the undirected reading of the same arcs is not the directed result
    lu, pu, _ = oracle.bfs(oracle.csr(src, dst, n), s)
    assert oracle.validate_arcs(src, dst, n, s, lu, pu).sum() > 0
