"""Symmetric half storage (bfs_graph_half) and the BFS that reads only it
(bfs_run_half), against the oracle.

- The half rows equal the oracle CSR's rows cut to their entries above the
  diagonal, and hold half its entries.
- bfs_run_half gives the oracle's levels and parents on R-MAT (large-component
  roots and a degree-1 root), a 3D grid, a star from its centre (every parent
  found by the push from below) and from a leaf, a path from either end (all
  parents below, or all above), and R-MAT at scale 20.
- A directed graph has no half storage (BFS_ERR_UNSUPPORTED).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def check_bfs(el, roots, what):
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    for s in roots:
        parent, level = bfs.run_half(g, int(s))
        assert_same(oracle.bfs(og, int(s)), (level.cpu().numpy(), parent.cpu().numpy()), f"{what} root {s}")
    g.destroy()


def test_half_rows_are_the_upper_triangle():
    for el in (inputs.rmat(12, 16, seed=101), inputs.grid3d(9), inputs.star(50)):
        og = oracle.csr_of(el)
        g = device_graph_from_edges(el)
        h = bfs.bfs_graph_half(g)
        rows = [og.row(v)[og.row(v) > v] for v in range(og.n)]
        want_off = np.zeros(og.n + 1, np.int64)
        want_off[1:] = np.cumsum([len(r) for r in rows])
        assert h["nnz"] * 2 == len(og.adj)
        assert np.array_equal(h["offsets"], want_off)
        assert np.array_equal(h["adj"], np.concatenate(rows).astype(np.int32))
        g.destroy()


def test_half_storage_bfs_matches_the_oracle():
    el, roots = inputs.workload_rmat(14, 4, graph_seed=102, root_seed=202)
    leaf = int(np.nonzero(np.diff(oracle.csr_of(el).offsets) == 1)[0][0])
    check_bfs(el, [int(r) for r in roots] + [leaf], "rmat14")
    check_bfs(inputs.grid3d(16), [0, 16 ** 3 - 1], "grid 16^3")
    check_bfs(inputs.star(300), [0, 7, 299], "star")
    check_bfs(inputs.path(200), [0, 199, 77], "path")


def test_half_storage_bfs_at_scale_20():
    el, roots = inputs.workload_rmat(20, 2, graph_seed=103, root_seed=203)
    check_bfs(el, roots, "rmat20")


def test_directed_graphs_have_no_half_storage():
    el = inputs.rmat(8, 8, seed=104)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    with pytest.raises(bfs.BfsError) as e:
        bfs.run_half(g, 0)
    assert e.value.code == bfs.BFS_ERR_UNSUPPORTED
    g.destroy()
