"""Seeded differential fuzzing on the GPU: small random graphs with many self-loops
and repeated pairs, undirected and directed, sizes around bitmap-word boundaries;
random roots, random per-level variant schedules, random batched word widths and
top-down limits, random ragged unions.  Every output is compared with the oracle,
bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def random_graph(rng):
    n = int(rng.choice([1, 2, 31, 32, 33, 63, 64, 65, int(rng.integers(2, 3000))]))
    m = int(rng.integers(0, 6 * n + 2))
    hub = rng.random() < 0.3
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if hub and m:  # a vertex with a long row (chunked above 1024 entries)
        k = int(rng.integers(1, m + 1))
        src[:k] = int(rng.integers(0, n))
    if m and rng.random() < 0.5:  # repeats and loops
        r = int(rng.integers(1, m + 1))
        src = np.concatenate([src, src[:r], dst[:r // 2 + 1]])
        dst = np.concatenate([dst, dst[:r], dst[:r // 2 + 1]])
    return n, src.astype(np.int32), dst.astype(np.int32)


@pytest.mark.parametrize("directed", [False, True])
def test_fuzz_single_root_and_schedules(directed):
    rng = np.random.default_rng(1000 + int(directed))
    for case in range(400):
        n, src, dst = random_graph(rng)
        og = oracle.digraph_csr(src, dst, n) if directed else oracle.csr(src, dst, n)
        ref_bfs = oracle.bfs_directed if directed else oracle.bfs
        g = bfs.bfs_graph_create_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n,
                                            directed=directed)
        off, adj = bfs.bfs_graph_copy_csr(g)
        assert np.array_equal(off.cpu().numpy(), og.offsets) and np.array_equal(adj.cpu().numpy(), og.adj), case
        for s in rng.integers(0, n, 2):
            sched = [int(x) for x in rng.integers(0, bfs.BFS_NUM_VARIANTS, int(rng.integers(1, 12)))]
            opts = bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE, schedule=sched)
            parent, level = bfs.run(g, int(s), opts)
            assert_same(ref_bfs(og, int(s)), (level.cpu().numpy(), parent.cpu().numpy()),
                        f"case {case} n={n} root {s} schedule {sched}")
        g.destroy()


@pytest.mark.parametrize("directed", [False, True])
def test_fuzz_batched(directed):
    rng = np.random.default_rng(2000 + int(directed))
    for case in range(200):
        n, src, dst = random_graph(rng)
        og = oracle.digraph_csr(src, dst, n) if directed else oracle.csr(src, dst, n)
        ref_bfs = oracle.bfs_directed if directed else oracle.bfs
        g = bfs.bfs_graph_create_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n,
                                            directed=directed)
        width = int(rng.choice([8, 16, 32, 64]))
        limit = int(rng.choice([1, 2, 16, 1 << 30]))
        bfs.bfs_set_tuning(g, batch_width=width, batch_topdown_limit=limit)
        k = int(rng.integers(1, 80))
        roots = [int(x) for x in rng.integers(0, n, k)]
        parent, level = bfs.run_batch(g, roots)
        bfs.bfs_sync(g)
        pa, lv = parent.cpu().numpy(), level.cpu().numpy()
        for i, s in enumerate(roots):
            assert_same(ref_bfs(og, s), (lv[i], pa[i]), f"case {case} n={n} width {width} limit {limit} row {i}")
        g.destroy()


def test_fuzz_ragged():
    rng = np.random.default_rng(3000)
    for case in range(60):
        parts_el = []
        for _ in range(int(rng.integers(1, 12))):
            n, src, dst = random_graph(rng)
            parts_el.append(inputs.EdgeList(n, src, dst))
        parts = [bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(),
                                                 el.n) for el in parts_el]
        u = bfs.bfs_graph_union(parts)
        roots = [int(rng.integers(0, el.n)) for el in parts_el]
        levels = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in parts_el]
        parents = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in parts_el]
        v = int(rng.integers(0, bfs.BFS_NUM_VARIANTS + 1))
        opts = None if v == bfs.BFS_NUM_VARIANTS else bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v)
        bfs.bfs_run_ragged(u, roots, parents, levels, opts)
        bfs.bfs_sync(u)
        for el, s, lv, pa in zip(parts_el, roots, levels, parents):
            assert_same(oracle.bfs(oracle.csr_of(el), s), (lv.cpu().numpy(), pa.cpu().numpy()), f"case {case}")
        for p in parts:
            p.destroy()
        u.destroy()
