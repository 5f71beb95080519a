"""GPU parity of the batched (8- to 64-root bitset) and ragged (union of graphs) traversals:
every output row equals the oracle's BFS from that root, bit for bit."""
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


def check_batch(el, roots, td_limit=None, width=None):
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    if td_limit is not None:
        bfs.bfs_set_tuning(g, batch_topdown_limit=td_limit)
    if width is not None:
        bfs.bfs_set_tuning(g, batch_width=width)
        assert bfs.bfs_get_tuning(g).batch_width == width
    parent, level = bfs.run_batch(g, list(roots))
    bfs.bfs_sync(g)
    parent, level = parent.cpu().numpy(), level.cpu().numpy()
    refs = oracle.bfs_many(og, roots)
    for i, (s, ref) in enumerate(zip(roots, refs)):
        assert_same(ref, (level[i], parent[i]), f"{el.name} batch row {i} root {s}")
    return g


@pytest.mark.parametrize("width", [8, 16, 32, 64])
@pytest.mark.parametrize("td_limit", [None, 1, 1 << 30])
def test_batch_s16_64_roots(td_limit, width):
    el, roots = inputs.workload_rmat(16, 64, graph_seed=1, root_seed=101)
    check_batch(el, roots, td_limit, width)


@pytest.mark.parametrize("width", [8, 64])
def test_batch_ragged_sizes_and_repeats(width):
    el = inputs.rmat(13, 16, seed=8)
    r = inputs.roots(el, 70, 9)
    roots = list(r[:65]) + [int(r[0]), int(r[0])] + [0]  # 68 roots: several chunks, repeated roots, a maybe-isolated one
    check_batch(el, roots, width=width)
    check_batch(el, roots[:1], width=width)


@pytest.mark.parametrize("width", [8, 16, 64])
def test_batch_closed_forms(width):
    check_batch(inputs.grid3d(12), [0, 5, 1727, 100], width=width)
    check_batch(inputs.star(70000), [0, 1, 2], width=width)
    check_batch(inputs.path(3000), list(range(0, 3000, 97)), width=width)


def test_batch_width_default_and_rejects():
    g = device_graph_from_edges(inputs.path(100))
    assert bfs.bfs_get_tuning(g).batch_width == 64
    bfs.bfs_set_tuning(g, batch_width=12)  # not a word width: the default applies
    assert bfs.bfs_get_tuning(g).batch_width == 64
    g.destroy()


def test_batch_s22_64_roots():
    el, roots = inputs.workload_rmat(22, 64, graph_seed=2, root_seed=102)
    check_batch(el, roots)


def test_batch_host_outputs():
    el = inputs.rmat(12, 16, seed=2)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    roots = inputs.roots(el, 5, 1)
    level = np.empty((5, el.n), np.int32)
    parent = np.empty((5, el.n), np.int32)
    bfs.bfs_run_batch(g, roots, parent, level, bfs.RunOptions(host_outputs=True))
    for i, s in enumerate(roots):
        assert_same(oracle.bfs(og, int(s)), (level[i], parent[i]))


def ragged_workload(count=32, seed=5):
    """`count` R-MAT graphs with scales drawn uniformly from 12..20, one root each."""
    return inputs.ragged_rmat(count, seed)


def test_ragged_32_graphs():
    graphs, roots = ragged_workload()
    parts = [device_graph_from_edges(el) for el in graphs]
    u = bfs.bfs_graph_union(parts)
    assert u.parts == 32 and u.n == sum(el.n for el in graphs)
    levels = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in graphs]
    parents = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in graphs]
    bfs.bfs_run_ragged(u, roots, parents, levels)
    bfs.bfs_sync(u)
    for el, s, lv, pa in zip(graphs, roots, levels, parents):
        og = oracle.csr_of(el)
        assert_same(oracle.bfs(og, s), (lv.cpu().numpy(), pa.cpu().numpy()), f"ragged {el.name}")
    # forced variants give the same result
    for v in range(4):
        bfs.bfs_run_ragged(u, roots, parents, levels, bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v))
        bfs.bfs_sync(u)
        og = oracle.csr_of(graphs[3])
        assert_same(oracle.bfs(og, roots[3]), (levels[3].cpu().numpy(), parents[3].cpu().numpy()))


def test_ragged_rejects_source_outside_part():
    parts = [device_graph_from_edges(inputs.path(10)), device_graph_from_edges(inputs.path(5))]
    u = bfs.bfs_graph_union(parts)
    outs = [torch.empty(10, dtype=torch.int32, device="cuda"), torch.empty(5, dtype=torch.int32, device="cuda")]
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run_ragged(u, [0, 5], outs, outs)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG


def test_batch_unaligned_outputs_and_odd_n():
    """The output transpose takes its scalar path for n not a multiple of 4 and for output
    rows that do not start on a 16-byte boundary; results are the same."""
    for n_extra in (0, 1, 2, 3):
        el = inputs.rmat(11, 16, seed=30 + n_extra)
        if n_extra:
            el, _ = inputs.disjoint_union([el, inputs.path(n_extra + 1)])
        og = oracle.csr_of(el)
        g = device_graph_from_edges(el)
        roots = [int(r) for r in inputs.roots(el, 9, 4)]
        n = el.n
        buf = torch.empty(2 * (len(roots) * n + 1), dtype=torch.int32, device="cuda")
        level = buf[1:1 + len(roots) * n]  # 4-byte aligned, not 16-byte aligned
        parent = buf[2 + len(roots) * n:2 + 2 * len(roots) * n]
        bfs.bfs_run_batch(g, roots, parent, level)
        bfs.bfs_sync(g)
        lv = level.view(len(roots), n).cpu().numpy()
        pa = parent.view(len(roots), n).cpu().numpy()
        for i, s in enumerate(roots):
            assert_same(oracle.bfs(og, s), (lv[i], pa[i]), f"n={n} root {s}")
        g.destroy()
