"""The sorted-output SpMSV (bfs_spmsv_sorted) and the BFS built from its steps
(bfs_run_sorted), against the oracle.

- Fig. 3's matrix and frontier give the hand-derived product y and masked t of
  tests/golden/fig3_spmsv.json, indices ascending.
- On R-MAT, directed R-MAT and grid graphs, random frontiers (with repeats)
  and random visited masks give oracle.spmsv_select2nd_max masked by
  oracle.mask_not entry for entry, with strictly ascending indices.
- bfs_run_sorted gives the oracle's levels and parents on undirected, directed
  and grid graphs, including vertices it cannot reach.
- An empty frontier gives an empty t; a frontier id outside [0, n) is an
  argument error.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def out_rows_csr(in_rows):
    """CSR (int64 offsets, int32 adj) of the out-rows of the matrix whose rows are in_rows."""
    n = len(in_rows)
    out = [[] for _ in range(n)]
    for i, cols in enumerate(in_rows):
        for j in cols:
            out[j].append(i)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in out])
    adj = np.array([v for r in out for v in sorted(r)], np.int32)
    return off, adj


def bitmap(n, vertices):
    words = np.zeros((n + 31) // 32, np.uint32)
    for v in vertices:
        words[v >> 5] |= np.uint32(1 << (v & 31))
    return torch.from_numpy(words.view(np.int32)).cuda()


def device_ids(ids):
    return torch.tensor(np.asarray(ids, np.int32), dtype=torch.int32, device="cuda")


def expected(in_rows, frontier, visited):
    y = oracle.spmsv_select2nd_max(in_rows, {int(u): int(u) for u in frontier})
    pi = [-1] * len(in_rows)
    for v in visited:
        pi[v] = 0
    t = oracle.mask_not(y, pi)
    keys = sorted(t)
    return keys, [t[k] for k in keys]


def check_step(g, in_rows, frontier, visited):
    n = len(in_rows)
    idx, val = bfs.spmsv_sorted(g, device_ids(frontier), None if visited is None else bitmap(n, visited))
    keys, vals = expected(in_rows, frontier, visited or [])
    got_i, got_v = idx.cpu().numpy(), val.cpu().numpy()
    assert np.all(np.diff(got_i) > 0), "indices not strictly ascending"
    assert got_i.tolist() == keys and got_v.tolist() == vals


def test_fig3_product_and_masked_step():
    """Fig. 3's matrix has a diagonal entry A(3, 3), a self-loop the library does
    not store; it only touches row 3, which the golden's mask removes, so the
    masked step matches the golden exactly and the product everywhere but y(3)
    (the largest off-diagonal frontier entry of row 3, 0)."""
    gold = json.load(open(os.path.join(HERE, "golden", "fig3_spmsv.json")))
    rows = [[j for j in r if j != i] for i, r in enumerate(gold["rows"])]
    off, adj = out_rows_csr(rows)
    g = bfs.bfs_graph_create(off, adj, directed=True)
    frontier = [int(k) for k in gold["frontier"]]
    idx, val = bfs.spmsv_sorted(g, device_ids(frontier))
    want = {int(k): v for k, v in gold["product_y"].items()}
    want[3] = 0
    assert idx.cpu().tolist() == sorted(want) and val.cpu().tolist() == [want[k] for k in sorted(want)]
    idx, val = bfs.spmsv_sorted(g, device_ids(frontier), bitmap(len(rows), gold["visited"]))
    want = {int(k): v for k, v in gold["masked_t"].items()}
    assert idx.cpu().tolist() == sorted(want) and val.cpu().tolist() == [want[k] for k in sorted(want)]
    g.destroy()


def test_random_steps_match_the_oracle():
    rng = np.random.default_rng(91)
    el = inputs.rmat(11, 8, seed=92)
    og = oracle.csr_of(el)
    rows = [og.row(v).tolist() for v in range(og.n)]
    g = device_graph_from_edges(el)
    for k in (1, 7, 300, 5000):
        frontier = rng.integers(0, og.n, k)  # repeats included
        visited = rng.choice(og.n, int(rng.integers(0, og.n)), replace=False).tolist()
        check_step(g, rows, frontier, visited)
        check_step(g, rows, frontier, None)
    g.destroy()
    # directed: t(v) is the largest frontier tail of an arc into v
    el = inputs.rmat(10, 8, seed=93)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    in_rows = oracle.digraph_csr(el.dst, el.src, el.n)
    rows = [in_rows.row(v).tolist() for v in range(el.n)]
    for k in (3, 200):
        frontier = rng.integers(0, el.n, k)
        check_step(g, rows, frontier, rng.choice(el.n, 100, replace=False).tolist())
    g.destroy()
    # a grid: rows of 3 to 6 entries, frontier a diagonal plane
    el = inputs.grid3d(12)
    og = oracle.csr_of(el)
    rows = [og.row(v).tolist() for v in range(og.n)]
    g = device_graph_from_edges(el)
    plane = [x + 12 * y + 144 * z for x in range(12) for y in range(12) for z in range(12) if x + y + z == 9]
    check_step(g, rows, plane, [v for v in range(og.n) if (v % 12) + (v // 12 % 12) + v // 144 < 9])
    g.destroy()


def test_empty_frontier_and_bad_ids():
    el = inputs.rmat(8, 8, seed=94)
    g = device_graph_from_edges(el)
    idx, val = bfs.spmsv_sorted(g, device_ids([]))
    assert idx.numel() == 0 and val.numel() == 0
    with pytest.raises(bfs.BfsError) as e:
        bfs.spmsv_sorted(g, device_ids([0, el.n + 3]))
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    with pytest.raises(bfs.BfsError) as e:
        bfs.run_sorted(g, el.n)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    g.destroy()


def test_sorted_bfs_matches_the_oracle():
    el, roots = inputs.workload_rmat(14, 4, graph_seed=95, root_seed=195)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    leaf = int(np.nonzero(np.diff(og.offsets) == 1)[0][0])  # a degree-1 root, possibly outside the large component
    for s in [int(r) for r in roots] + [leaf]:
        parent, level = bfs.run_sorted(g, s)
        assert_same(oracle.bfs(og, s), (level.cpu().numpy(), parent.cpu().numpy()), f"rmat14 root {s}")
    g.destroy()
    el = inputs.grid3d(16)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    parent, level = bfs.run_sorted(g, 0)
    assert_same(oracle.bfs(og, 0), (level.cpu().numpy(), parent.cpu().numpy()), "grid 16^3")
    g.destroy()
    el = inputs.rmat(12, 8, seed=96)
    dg = oracle.digraph_of(el)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    outdeg = np.diff(dg.offsets)
    for s in [int(r) for r in inputs.roots(el, 12, 196) if outdeg[r] > 0][:3]:
        parent, level = bfs.run_sorted(g, s)
        assert_same(oracle.bfs_directed(dg, s), (level.cpu().numpy(), parent.cpu().numpy()), f"directed root {s}")
    g.destroy()


def test_sorted_bfs_at_scale_20():
    el, roots = inputs.workload_rmat(20, 2, graph_seed=97, root_seed=197)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    for s in roots:
        parent, level = bfs.run_sorted(g, int(s))
        assert_same(oracle.bfs(og, int(s)), (level.cpu().numpy(), parent.cpu().numpy()), f"rmat20 root {s}")
    g.destroy()
