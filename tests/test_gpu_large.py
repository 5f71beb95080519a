"""Full-size checks in the benchmark's launch configurations.

At these sizes the oracle's CSR build would take minutes, so results are checked
with the oracle's O(m) edge-list validator (`oracle.validate_edges`): zero
violations means the levels are the hop distances and the parents follow the
max-id rule, exactly.  Inputs come from the seeded generators; nothing from the
CUDA path is used as an expected value.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _validate_rows(el, roots, levels, parents):
    def one(i):
        return oracle.validate_edges(el.src, el.dst, el.n, int(roots[i]), levels[i], parents[i])

    with ThreadPoolExecutor(max_workers=min(len(roots), os.cpu_count() or 1)) as ex:
        bad = list(ex.map(one, range(len(roots))))
    for i, b in enumerate(bad):
        assert b.sum() == 0, (int(roots[i]), b.tolist())


def test_rmat26_single_root_bench_configuration():
    """R-MAT scale 26 (67 M vertices, 2.1 G CSR entries), graph seed 3 / roots 103, heuristic selector."""
    el, roots = inputs.workload_rmat(26, 64, graph_seed=3, root_seed=103)
    g = device_graph_from_edges(el)
    picks = [int(roots[0]), int(roots[len(roots) // 2])]
    levels, parents = [], []
    for s in picks:
        parent, level = bfs.run(g, s)
        bfs.bfs_sync(g)
        levels.append(level.cpu().numpy())
        parents.append(parent.cpu().numpy())
    g.destroy()
    _validate_rows(el, picks, levels, parents)


def test_rmat24_batched_64_roots():
    """64 roots in one batched traversal with 64-bit words on R-MAT scale 24 (graph seed 4 /
    roots 104): every row validated; four traversals of 16-bit words give the same rows."""
    el, roots = inputs.workload_rmat(24, 64, graph_seed=4, root_seed=104)
    g = device_graph_from_edges(el)
    parent, level = bfs.run_batch(g, [int(s) for s in roots])
    bfs.bfs_set_tuning(g, batch_width=16)
    p2, l2 = bfs.run_batch(g, [int(s) for s in roots])
    bfs.bfs_sync(g)
    assert torch.equal(parent, p2) and torch.equal(level, l2)
    del p2, l2
    lv, pa = level.cpu().numpy(), parent.cpu().numpy()
    del parent, level
    g.destroy()
    _validate_rows(el, roots, lv, pa)


def test_grid256_closed_form():
    """The 256^3 grid from the corner (766 levels): level = x + y + z, parent by the max-id rule."""
    N = 256
    el = inputs.grid3d(N)
    g = device_graph_from_edges(el)
    parent, level = bfs.run(g, 0)
    bfs.bfs_sync(g)
    level, parent = level.cpu().numpy(), parent.cpu().numpy()
    v = np.arange(N ** 3, dtype=np.int64)
    x, y, z = v % N, (v // N) % N, v // (N * N)
    assert np.array_equal(level, (x + y + z).astype(np.int32))
    exp = np.where(x > 0, v - 1, np.where(y > 0, v - N, v - N * N))
    exp[0] = 0
    assert np.array_equal(parent, exp.astype(np.int32))
