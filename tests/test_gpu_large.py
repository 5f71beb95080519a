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


def test_rmat26_single_root_and_batched_bench_configuration():
    """R-MAT scale 26 (67 M vertices, 2.1 G CSR entries), graph seed 3 / roots 103: two single-root
    traversals (heuristic selector) and the bench's 64-root batched traversal.  The batched rows of
    those two roots equal the single-root results on the device, and the last batched row is
    validated on its own."""
    el, roots = inputs.workload_rmat(26, 64, graph_seed=3, root_seed=103)
    g = device_graph_from_edges(el)
    picks = [0, len(roots) // 2]
    levels, parents, singles = [], [], []
    for i in picks:
        parent, level = bfs.run(g, int(roots[i]))
        bfs.bfs_sync(g)
        singles.append((parent, level))
    pb, lb = bfs.run_batch(g, [int(r) for r in roots])
    bfs.bfs_sync(g)
    for i, (parent, level) in zip(picks, singles):
        assert torch.equal(pb[i], parent) and torch.equal(lb[i], level), f"batched row {i}"
        levels.append(level.cpu().numpy())
        parents.append(parent.cpu().numpy())
    last = len(roots) - 1
    levels.append(lb[last].cpu().numpy())
    parents.append(pb[last].cpu().numpy())
    del pb, lb, singles
    g.destroy()
    _validate_rows(el, [int(roots[i]) for i in picks + [last]], levels, parents)


def test_directed_rmat22_validated():
    """Directed R-MAT scale 22 (the generated pairs read as arcs, 67 M of them): two single-root
    traversals and a 16-root batched traversal, validated arc by arc (`oracle.validate_arcs`)."""
    el = inputs.rmat(22, 16, seed=33)
    outdeg = np.bincount(el.src[el.src != el.dst], minlength=el.n)
    roots = [int(r) for r in inputs.roots(el, 64, 34) if outdeg[r] > 0][:16]
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    rows = []
    for s in roots[:2]:
        parent, level = bfs.run(g, s)
        bfs.bfs_sync(g)
        rows.append((s, level.cpu().numpy(), parent.cpu().numpy()))
    pb, lb = bfs.run_batch(g, roots)
    bfs.bfs_sync(g)
    rows.append((roots[-1], lb[-1].cpu().numpy(), pb[-1].cpu().numpy()))
    assert np.array_equal(lb[0].cpu().numpy(), rows[0][1]) and np.array_equal(pb[0].cpu().numpy(), rows[0][2])
    g.destroy()

    def one(r):
        s, lv, pa = r
        return oracle.validate_arcs(el.src, el.dst, el.n, s, lv, pa)

    with ThreadPoolExecutor(max_workers=len(rows)) as ex:
        for (s, lv, _), b in zip(rows, ex.map(one, rows)):
            assert b.sum() == 0, (s, b.tolist())
            assert (lv > 0).sum() > 1000  # a real traversal, not a trivial one


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
