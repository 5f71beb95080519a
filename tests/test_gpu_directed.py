"""GPU parity on directed graphs (BFS_DIRECTED): levels = shortest directed path
lengths and parents = largest in-neighbour one level up, bit-identical to the
directed oracle under every selector, for the batched traversal, from a CSR or
from an arc list, including a hub whose out-row is split into chunks after a
pull level discovered it."""
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


def digraph(src, dst, n):
    return bfs.bfs_graph_create_from_edges(torch.from_numpy(np.asarray(src, np.int32)).cuda(),
                                           torch.from_numpy(np.asarray(dst, np.int32)).cuda(), n, directed=True)


def selectors(nlev_hint=8):
    yield "heuristic", bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC, want_counts=True)
    for v in range(bfs.BFS_NUM_VARIANTS):
        yield f"forced {bfs.VARIANT_NAMES[v]}", bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v,
                                                                want_counts=True)
    # pull then top-down: vertices claimed by the pull are expanded top-down next
    sched = [bfs.BFS_VARIANT_TD_BINNED if k % 2 == 0 else bfs.BFS_VARIANT_PULL for k in range(nlev_hint * 4)]
    yield "alternating", bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE, schedule=sched, want_counts=True)


def check_all(el, roots):
    og = oracle.digraph_of(el)
    g = digraph(el.src, el.dst, el.n)
    assert g.nnz == og.nnz
    for s in roots:
        ref = oracle.bfs_directed(og, int(s))
        for name, opts in selectors():
            parent, level = bfs.run(g, int(s), opts)
            assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"{el.name} root {s} {name}")
            assert opts.edges == oracle.out_edges(og, ref[0]), name
    return g


def test_directed_rmat_and_er_all_selectors():
    el = inputs.rmat(14, 8, seed=21)
    check_all(el, [int(r) for r in inputs.roots(el, 4, 22)])
    er = inputs.erdos_renyi(1 << 13, 3, seed=23)
    check_all(er, [int(r) for r in inputs.roots(er, 4, 24)])


def test_directed_learned_selector():
    el = inputs.rmat(13, 16, seed=25)
    og = oracle.digraph_of(el)
    g = digraph(el.src, el.dst, el.n)
    rng = np.random.default_rng(3)
    bfs.bfs_selector_set_params((0.3 * rng.standard_normal(bfs.BFS_MLP_PARAMS)).astype(np.float32))
    try:
        for s in inputs.roots(el, 3, 26):
            parent, level = bfs.run(g, int(s), bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED))
            assert_same(oracle.bfs_directed(og, int(s)), (level.cpu().numpy(), parent.cpu().numpy()))
    finally:
        bfs.bfs_selector_set_params(None)


def test_directed_closed_forms():
    n = 3000
    v = np.arange(n)
    g = digraph(v[:-1], v[1:], n)  # path 0 -> 1 -> ... -> n-1
    parent, level = bfs.run(g, 0)
    assert np.array_equal(level.cpu().numpy(), v) and np.array_equal(parent.cpu().numpy()[1:], v[:-1])
    parent, level = bfs.run(g, n - 1)  # nothing reachable against the arcs
    lv = level.cpu().numpy()
    assert lv[-1] == 0 and (lv[:-1] == -1).all()
    g = digraph(v, (v + 1) % n, n)  # cycle
    for s in (0, 1234):
        parent, level = bfs.run(g, s)
        assert np.array_equal(level.cpu().numpy(), (v - s) % n)
        exp = (v - 1) % n
        exp[s] = s
        assert np.array_equal(parent.cpu().numpy(), exp)
    g = digraph(np.zeros(n - 1, np.int32), v[1:], n)  # out-star: 0 -> everything
    parent, level = bfs.run(g, 0)
    assert (level.cpu().numpy()[1:] == 1).all() and (parent.cpu().numpy() == 0).all()
    parent, level = bfs.run(g, 7)
    lv = level.cpu().numpy()
    assert lv[7] == 0 and (np.delete(lv, 7) == -1).all()


def test_directed_from_csr_equals_from_arcs_and_validation():
    el = inputs.rmat(12, 8, seed=27)
    og = oracle.digraph_of(el)
    off = torch.from_numpy(og.offsets).cuda()
    adj = torch.from_numpy(og.adj).cuda()
    g1 = bfs.bfs_graph_create(off, adj, validate=True, directed=True)
    g2 = digraph(el.src, el.dst, el.n)
    for s in inputs.roots(el, 3, 28):
        p1, l1 = bfs.run(g1, int(s))
        p2, l2 = bfs.run(g2, int(s))
        assert torch.equal(p1, p2) and torch.equal(l1, l2)
    # an asymmetric CSR is not an undirected graph
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_create(off, adj, validate=True)
    assert e.value.code == bfs.BFS_ERR_INVALID_GRAPH
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_union([g1])
    assert e.value.code == bfs.BFS_ERR_UNSUPPORTED


@pytest.mark.parametrize("width", [8, 64])
@pytest.mark.parametrize("td_limit", [None, 1, 1 << 30])
def test_directed_batched(width, td_limit):
    el = inputs.rmat(13, 8, seed=29)
    og = oracle.digraph_of(el)
    g = digraph(el.src, el.dst, el.n)
    bfs.bfs_set_tuning(g, batch_width=width)
    if td_limit is not None:
        bfs.bfs_set_tuning(g, batch_topdown_limit=td_limit)
    roots = [int(r) for r in inputs.roots(el, 20, 30)] + [0]
    parent, level = bfs.run_batch(g, roots)
    bfs.bfs_sync(g)
    pa, lv = parent.cpu().numpy(), level.cpu().numpy()
    for i, s in enumerate(roots):
        assert_same(oracle.bfs_directed(og, s), (lv[i], pa[i]), f"row {i} root {s}")


def test_directed_hub_found_by_pull_then_expanded_in_chunks():
    """0 -> A (2000 vertices), every A -> H, the first ten of A -> H2, H -> B (5000
    vertices), H2 -> D (3000 vertices), every B -> C (one vertex each).  A pull
    level finds H through a long in-row and H2 through a short one; their
    out-rows (above the 1024-arc chunk size) must then be expanded top-down."""
    nA, nB, nD = 2000, 5000, 3000
    A = 1 + np.arange(nA)
    H, H2 = 1 + nA, 2 + nA
    B = H2 + 1 + np.arange(nB)
    C = B[-1] + 1 + np.arange(nB)
    D = C[-1] + 1 + np.arange(nD)
    n = int(D[-1]) + 1
    src = np.concatenate([np.zeros(nA), A, A[:10], np.full(nB, H), np.full(nD, H2), B]).astype(np.int32)
    dst = np.concatenate([A, np.full(nA, H), np.full(10, H2), B, D, C]).astype(np.int32)
    perm = np.random.default_rng(31).permutation(src.shape[0])
    src, dst = src[perm], dst[perm]
    og = oracle.digraph_csr(src, dst, n)
    ref = oracle.bfs_directed(og, 0)
    assert ref[0][H] == 2 and ref[0][H2] == 2 and ref[0][B[0]] == 3 and ref[0][D[0]] == 3
    g = digraph(src, dst, n)
    td, pull = bfs.BFS_VARIANT_TD_BINNED, bfs.BFS_VARIANT_PULL
    for sched in ([td, pull, td, td, td], [td, pull, bfs.BFS_VARIANT_TD_WARP, pull, td],
                  [td, pull, bfs.BFS_VARIANT_TD_THREAD, td, td]):
        parent, level = bfs.run(g, 0, bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE, schedule=sched))
        assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"schedule {sched}")
    # batched: level 1 (A, 2000 vertices) pulls, level 2 ({H, H2}) goes top-down
    bfs.bfs_set_tuning(g, batch_topdown_limit=1000)
    for width in (8, 64):
        bfs.bfs_set_tuning(g, batch_width=width)
        parent, level = bfs.run_batch(g, [0, 0])
        bfs.bfs_sync(g)
        for i in range(2):
            assert_same(ref, (level[i].cpu().numpy(), parent[i].cpu().numpy()), f"batched row {i} width {width}")
