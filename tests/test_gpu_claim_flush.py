"""Top-down levels that claim more vertices than a CTA's claim buffers hold:
the CTA flushes its buffers before a chunk item or a binned tile could
overflow them, and whatever still overflows goes to the queue directly.  The
graph makes every CTA claim several thousand vertices from chunk items in one
level: root 0 joins 64 hubs (ids 1..64), and each of 2^21 leaves joins two
distinct hubs, i mod 64 and (7 i + 3) mod 64, so a hub row holds about 65,000
leaves (64 chunk items) and, on 304 CTAs, each CTA claims about 6,900 leaves at
level 1 against 6,144 buffer entries.  Each leaf is offered by two chunk items,
usually on different CTAs, and must take the larger hub as parent.  Levels and
parents equal the oracle's for every top-down variant forced at every level,
the heuristic, and the batched traversal (whose top-down chunk loop flushes
the same way)."""
import numpy as np
import pytest

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu

HUBS, LEAVES = 64, 1 << 21


def hub_graph():
    i = np.arange(LEAVES, dtype=np.int64)
    leaf = (1 + HUBS + i).astype(np.int32)
    h1 = (1 + i % HUBS).astype(np.int32)
    h2 = (1 + (7 * i + 3) % HUBS).astype(np.int32)
    src = np.concatenate([np.zeros(HUBS, np.int32), leaf, leaf])
    dst = np.concatenate([np.arange(1, HUBS + 1, dtype=np.int32), h1, h2])
    return inputs.EdgeList(1 + HUBS + LEAVES, src, dst), np.maximum(h1, h2)


@pytest.fixture(scope="module")
def case():
    require_cuda()
    el, want_parent = hub_graph()
    og = oracle.csr_of(el)
    ref = oracle.bfs(og, 0)
    lv, pa = ref[0], ref[1]
    # the closed form, so that the oracle itself is pinned here too
    assert lv[0] == 0 and (lv[1:HUBS + 1] == 1).all() and (lv[HUBS + 1:] == 2).all()
    assert (pa[1:HUBS + 1] == 0).all() and np.array_equal(pa[HUBS + 1:], want_parent)
    g = device_graph_from_edges(el)
    yield g, ref
    g.destroy()


@pytest.mark.parametrize("variant", [bfs.BFS_VARIANT_TD_THREAD, bfs.BFS_VARIANT_TD_WARP, bfs.BFS_VARIANT_TD_BINNED])
def test_forced_top_down_with_full_claim_buffers(case, variant):
    g, ref = case
    parent, level = bfs.run(g, 0, bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=variant))
    bfs.bfs_sync(g)
    assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), bfs.VARIANT_NAMES[variant])


def test_heuristic(case):
    g, ref = case
    parent, level = bfs.run(g, 0)
    bfs.bfs_sync(g)
    assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), "heuristic")


def test_batched_top_down_with_full_claim_buffers(case):
    g, ref = case
    bfs.bfs_set_tuning(g, batch_topdown_limit=1 << 30)  # every level top-down
    try:
        parent, level = bfs.run_batch(g, [0, 0, 0])
        bfs.bfs_sync(g)
    finally:
        bfs.bfs_set_tuning(g, batch_topdown_limit=0)
    for r in range(3):
        assert_same(ref, (level[r].cpu().numpy(), parent[r].cpu().numpy()), f"batched row {r}")
