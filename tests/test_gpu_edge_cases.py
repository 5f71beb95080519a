"""Degenerate inputs on the GPU, against the oracle: a graph without edges, a
one-vertex graph, self-loops and repeated pairs only, ragged unions whose parts
are single vertices or edgeless, and the batched traversal on all of them."""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu

SELECTORS = [bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC)] + [
    bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v) for v in range(bfs.BFS_NUM_VARIANTS)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def check(el, roots):
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    for s in roots:
        ref = oracle.bfs(og, int(s))
        for opts in SELECTORS:
            parent, level = bfs.run(g, int(s), opts)
            assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"{el.name} root {s}")
    parent, level = bfs.run_batch(g, [int(s) for s in roots])
    bfs.bfs_sync(g)
    for i, s in enumerate(roots):
        assert_same(oracle.bfs(og, int(s)), (level[i].cpu().numpy(), parent[i].cpu().numpy()), f"batched {s}")
    g.destroy()


def empty(n):
    return inputs.EdgeList(n, np.zeros(0, np.int32), np.zeros(0, np.int32))


def test_graph_without_edges():
    check(empty(100), [0, 5, 99])
    check(empty(33), [32])  # a partial last bitmap word


def test_one_vertex():
    check(empty(1), [0])


def test_self_loops_and_repeats_only():
    src = np.array([0, 1, 0, 1, 0, 2, 2], np.int32)
    dst = np.array([0, 1, 1, 0, 1, 2, 2], np.int32)
    el = inputs.EdgeList(3, src, dst)
    g = device_graph_from_edges(el)
    assert g.nnz == 2  # the single edge 0-1, stored in both rows
    g.destroy()
    check(el, [0, 1, 2])


def test_ragged_with_degenerate_parts():
    parts_el = [empty(1), inputs.path(2), empty(3), inputs.star(5), inputs.path(1)]
    parts = [device_graph_from_edges(el) for el in parts_el]
    u = bfs.bfs_graph_union(parts)
    roots = [0, 1, 2, 0, 0]
    levels = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in parts_el]
    parents = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in parts_el]
    bfs.bfs_run_ragged(u, roots, parents, levels)
    bfs.bfs_sync(u)
    for el, s, lv, pa in zip(parts_el, roots, levels, parents):
        assert_same(oracle.bfs(oracle.csr_of(el), s), (lv.cpu().numpy(), pa.cpu().numpy()), f"part {el.name}")


@pytest.mark.parametrize("directed", [False, True])
def test_csr_builder_when_the_last_pair_repeats(directed):
    """Edge lists whose largest (u, v) pair occurs several times, with isolated vertices
    after the last non-empty row: the device CSR equals the oracle's row for row."""
    rng = np.random.default_rng(9)
    for n, m in ((3, 0), (50, 80), (1000, 3000)):
        src = rng.integers(0, n // 2 + 1, m).astype(np.int32)
        dst = rng.integers(0, n // 2 + 1, m).astype(np.int32)
        hi = np.int32(n // 2)
        src = np.concatenate([src, [hi, hi, 0, hi - 1, hi - 1]]).astype(np.int32)  # the last pairs repeat
        dst = np.concatenate([dst, [hi - 1, hi - 1, 0, hi, hi]]).astype(np.int32)
        og = oracle.digraph_csr(src, dst, n) if directed else oracle.csr(src, dst, n)
        g = bfs.bfs_graph_create_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n,
                                            directed=directed)
        off, adj = bfs.bfs_graph_copy_csr(g)
        assert np.array_equal(off.cpu().numpy(), og.offsets), (n, m)
        assert np.array_equal(adj.cpu().numpy(), og.adj), (n, m)
        g.destroy()
