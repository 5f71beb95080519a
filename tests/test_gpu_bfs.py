"""GPU parity of the library against the CPU oracle: CSR builder, single-root BFS,
every forced variant, selectors, statistics, edge cases and error codes.

All comparisons are bit-exact (integer outputs)."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import (assert_same, check_roots, device_graph_from_edges, device_graph_from_oracle_csr,
                         require_cuda, run_gpu)
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL_FORCED = tuple((bfs.BFS_SELECT_FORCED, v) for v in range(bfs.BFS_NUM_VARIANTS))
ALL_SELECTORS = ((bfs.BFS_SELECT_HEURISTIC, 0),) + ALL_FORCED


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


# ---------------- K1: device CSR builder ----------------

def csr_equal(el):
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    off, adj = bfs.bfs_graph_copy_csr(g, device=False)
    assert g.n == og.n and g.nnz == og.nnz
    assert np.array_equal(off.numpy(), og.offsets)
    assert np.array_equal(adj.numpy(), og.adj)


@pytest.mark.parametrize("seed", range(6))
def test_csr_builder_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 6 * n))
    el = inputs.EdgeList(n, rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32))
    csr_equal(el)


@pytest.mark.parametrize("make", [lambda: inputs.path(1), lambda: inputs.star(70000), lambda: inputs.complete(90),
                                  lambda: inputs.grid3d(20), lambda: inputs.rmat(16, 16, seed=1),
                                  lambda: inputs.EdgeList(5, np.zeros(0, np.int32), np.zeros(0, np.int32)),
                                  lambda: inputs.EdgeList(3, np.array([1, 1], np.int32), np.array([1, 1], np.int32))])
def test_csr_builder_shapes(make):
    csr_equal(make())


def test_csr_builder_rmat_s22():
    csr_equal(inputs.rmat(22, 16, seed=2))


def test_csr_builder_rejects_bad_endpoint():
    src = torch.tensor([0, 5], dtype=torch.int32, device="cuda")
    dst = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_create_from_edges(src, dst, 5)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG


# ---------------- single-root BFS ----------------

@pytest.mark.parametrize("make,roots", [
    (lambda: inputs.path(1000), [0, 500, 999]),
    (lambda: inputs.star(100_000), [0, 7]),  # centre degree above the chunk threshold
    (lambda: inputs.binary_tree(4095), [0, 4094]),
    (lambda: inputs.cycle(1001), [0, 3]),
    (lambda: inputs.cycle(1000), [0]),
    (lambda: inputs.complete(200), [0, 199]),
    (lambda: inputs.grid3d(16), [0, 4095]),
])
def test_closed_form_graphs(make, roots):
    check_roots(make(), roots, selectors=ALL_SELECTORS)


def test_disjoint_union_and_isolated_source():
    u, bases = inputs.disjoint_union([inputs.path(37), inputs.star(33), inputs.cycle(40)])
    el = inputs.EdgeList(u.n + 5, u.src, u.dst)  # five isolated vertices at the end
    check_roots(el, [int(bases[1]) + 3, u.n + 2, 0], selectors=ALL_SELECTORS)


@pytest.mark.parametrize("seed", range(8))
def test_random_graphs(seed):
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(1, 5000))
    m = int(rng.integers(0, 8 * n))
    el = inputs.EdgeList(n, rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32))
    roots = rng.choice(n, size=min(n, 3), replace=False)
    check_roots(el, roots, selectors=ALL_SELECTORS)


def test_rmat_s16_sixteen_roots_all_variants():
    """R-MAT scale 16, edgefactor 16, seeded graph 1 / roots 101 (the small evaluation workload)."""
    el, roots = inputs.workload_rmat(16, 16, graph_seed=1, root_seed=101)
    check_roots(el, roots, selectors=ALL_SELECTORS)


def test_rmat_s22_sixty_four_roots():
    """R-MAT scale 22, 64 roots (graph seed 2, roots 102), heuristic selector; variants on a few roots."""
    el, roots = inputs.workload_rmat(22, 64, graph_seed=2, root_seed=102)
    g, og, refs = check_roots(el, roots)
    for s, ref in list(zip(roots, refs))[:3]:
        for sel, var in ALL_FORCED:
            got = run_gpu(g, int(s), bfs.RunOptions(selector=sel, forced_variant=var))
            assert_same(ref, got, f"s22 root {s} variant {var}")


def test_grid_128_corner():
    """3D 7-point grid 128^3 from the corner: 382 levels, level = x + y + z."""
    el = inputs.grid3d(128)
    g, og, refs = check_roots(el, [0], selectors=((bfs.BFS_SELECT_HEURISTIC, 0), (bfs.BFS_SELECT_FORCED, 0),
                                                  (bfs.BFS_SELECT_FORCED, 3)))
    assert refs[0][2] == 382


def test_graph_from_csr_matches_from_edges():
    el = inputs.rmat(14, 16, seed=9)
    og = oracle.csr_of(el)
    g1 = device_graph_from_oracle_csr(og)
    g2 = device_graph_from_edges(el)
    s = int(inputs.roots(el, 1, 3)[0])
    assert_same(oracle.bfs(og, s), run_gpu(g1, s))
    assert_same(oracle.bfs(og, s), run_gpu(g2, s))


def test_stats_match_oracle_level_counts():
    el, roots = inputs.workload_rmat(16, 4, graph_seed=1, root_seed=101)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    for s in roots:
        level, parent, nl = oracle.bfs(og, int(s))
        count, edges = oracle.level_stats(og, level, nl)
        opts = bfs.RunOptions(stats_levels=64)
        bfs.run(g, int(s), opts)
        st = opts.stats()
        assert len(st) == nl
        deg = og.degree()
        for k in range(nl):
            assert st[k]["frontier_count"] == count[k]
            assert st[k]["frontier_edges"] == edges[k]
            fk = level == k
            d = deg[fk]
            assert st[k]["bin_count"] == [int((d <= 32).sum()), int(((d > 32) & (d <= 1024)).sum()),
                                          int((d > 1024).sum())]
            assert st[k]["unvisited_count"] == og.n - count[:k + 1].sum()
            assert st[k]["unvisited_edges"] == og.nnz - edges[:k + 1].sum()
            assert 0 <= st[k]["variant"] < 4 and st[k]["time_ns"] > 0


def test_schedule_selector():
    el, roots = inputs.workload_rmat(16, 2, graph_seed=1, root_seed=101)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    for s in roots:
        ref = oracle.bfs(og, int(s))
        sched = [0, 2, 3, 3, 1, 0, 2]
        opts = bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE, schedule=sched, stats_levels=64)
        got = run_gpu(g, int(s), opts)
        assert_same(ref, got)
        for k, st in enumerate(opts.stats()):
            if k < len(sched):
                assert st["variant"] == sched[k]


def test_host_outputs():
    el = inputs.rmat(14, 16, seed=3)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    s = int(inputs.roots(el, 1, 4)[0])
    level = np.empty(el.n, np.int32)
    parent = np.empty(el.n, np.int32)
    bfs.bfs_run(g, s, parent, level, bfs.RunOptions(host_outputs=True))
    assert_same(oracle.bfs(og, s), (level, parent))


def test_deterministic_repeat_and_streams():
    el = inputs.rmat(16, 16, seed=1)
    g = device_graph_from_edges(el)
    s = int(inputs.roots(el, 1, 5)[0])
    a = run_gpu(g, s)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        parent, level = bfs.run(g, s, stream=side)
    bfs.bfs_sync(g, side)
    assert np.array_equal(a[0], level.cpu().numpy()) and np.array_equal(a[1], parent.cpu().numpy())


# ---------------- errors ----------------

def test_invalid_arguments():
    el = inputs.path(10)
    g = device_graph_from_edges(el)
    out = torch.empty(10, dtype=torch.int32, device="cuda")
    for s in (-1, 10):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_run(g, s, out, out)
        assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run(g, 0, out, out, bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=7))
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    with pytest.raises(bfs.BfsError):
        bfs.bfs_run_batch(g, [], out, out)


@pytest.mark.parametrize("bad", ["unsorted", "asymmetric", "loop", "range", "offsets"])
def test_validation_rejects_malformed_csr(bad):
    off = np.array([0, 2, 4, 6], np.int64)
    adj = np.array([1, 2, 0, 2, 0, 1], np.int32)  # triangle
    if bad == "unsorted":
        adj = np.array([2, 1, 0, 2, 0, 1], np.int32)
    elif bad == "asymmetric":
        off = np.array([0, 2, 3, 5], np.int64)
        adj = np.array([1, 2, 0, 0, 1], np.int32)  # 1 lacks 2
    elif bad == "loop":
        adj = np.array([0, 1, 0, 2, 0, 1], np.int32)
    elif bad == "range":
        adj = np.array([1, 3, 0, 2, 0, 1], np.int32)
    elif bad == "offsets":
        off = np.array([0, 4, 2, 6], np.int64)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_create(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda(), validate=True)
    assert e.value.code == bfs.BFS_ERR_INVALID_GRAPH
    good = bfs.bfs_graph_create(torch.from_numpy(np.array([0, 2, 4, 6], np.int64)).cuda(),
                                torch.from_numpy(np.array([1, 2, 0, 2, 0, 1], np.int32)).cuda(), validate=True)
    assert good.nnz == 6


def test_device_wait_limit_returns_timeout_and_recovers():
    """A spin limit of one poll makes the grid barrier give up: the kernel returns
    BFS_ERR_TIMEOUT through the status word instead of waiting, and the next run works."""
    el = inputs.rmat(12, 16, seed=4)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    s = int(inputs.roots(el, 1, 6)[0])
    parent, level = bfs.run(g, s, bfs.RunOptions(spin_limit=1))
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_sync(g)
    assert e.value.code == bfs.BFS_ERR_TIMEOUT
    assert_same(oracle.bfs(og, s), run_gpu(g, s))


# ---------------- autotuner ----------------

def test_autotune_keeps_results_and_caches(tmp_path):
    el, roots = inputs.workload_rmat(16, 4, graph_seed=1, root_seed=101)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    cache = str(tmp_path / "tuning.json")
    t = bfs.bfs_autotune_cached(g, roots[:2], cache)
    assert t.warp_degree in (8, 16, 32, 64) and 1 <= t.pull_thread_degree <= 4 and t.chunk_degree >= 1024
    assert t.alpha > 0 and t.beta > 0 and t.batch_topdown_limit >= 1
    for s in roots:
        assert_same(oracle.bfs(og, int(s)), run_gpu(g, int(s)))
    # a second graph of the same class takes the cached tuning without timing
    g2 = device_graph_from_edges(el)
    t2 = bfs.bfs_autotune_cached(g2, roots[:2], cache)
    assert t2.as_dict() == t.as_dict()
    parent, level = bfs.run_batch(g2, [int(s) for s in roots])
    bfs.bfs_sync(g2)
    for i, s in enumerate(roots):
        assert_same(oracle.bfs(og, int(s)), (level[i].cpu().numpy(), parent[i].cpu().numpy()))


@pytest.mark.parametrize("narrow_edges,ctas_per_sm", [(-1, 0), (1 << 30, 0), (0, 1), (1 << 30, 1)])
def test_narrow_levels_and_grid_sizes(narrow_edges, ctas_per_sm):
    """The narrow_edges knob decides which levels run on half the CTAs (never: -1; every
    level: 1 << 30) and ctas_per_sm the persistent grid's size (two CTAs per SM, or one);
    every variant and the learned selector, on R-MAT and on a grid, give the oracle's
    results bit for bit; a default run on the same graph follows (the grid size changes
    back, and with it the barrier's base)."""
    wpath = os.path.join(os.path.dirname(bfs.__file__), "selector_weights.bin")
    bfs.bfs_selector_load(wpath)
    try:
        for el, roots in ((inputs.rmat(15, 16, seed=81), None), (inputs.grid3d(24), [0])):
            if roots is None:
                roots = [int(r) for r in inputs.roots(el, 3, 181)]
            og = oracle.csr_of(el)
            g = device_graph_from_edges(el)
            bfs.bfs_set_tuning(g, narrow_edges=narrow_edges, ctas_per_sm=ctas_per_sm)
            refs = oracle.bfs_many(og, roots)
            opts = [bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v)
                    for v in range(bfs.BFS_NUM_VARIANTS)]
            opts += [bfs.RunOptions(), bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED)]
            for s, ref in zip(roots, refs):
                for o in opts:
                    parent, level = bfs.run(g, s, o)
                    bfs.bfs_sync(g)
                    assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()),
                                f"narrow {narrow_edges}, {ctas_per_sm} CTAs per SM, root {s}")
            bfs.bfs_set_tuning(g, narrow_edges=0, ctas_per_sm=0)
            parent, level = bfs.run(g, roots[0])
            bfs.bfs_sync(g)
            assert_same(refs[0], (level.cpu().numpy(), parent.cpu().numpy()), "default after narrow runs")
            g.destroy()
    finally:
        bfs.bfs_selector_set_params(None)
