"""Cases of the bounds-checking build, run in a child process of
test_gpu_bounds.py with BFS_BOUNDS_CHECK=1 (the library choice is per process).

    python tests/bounds_child.py parity     # well-formed graphs: bit-identical to the oracle, no false alarm
    python tests/bounds_child.py malformed  # bad ids and offsets: BFS_ERR_BOUNDS, then a clean run

The malformed cases run only when the loaded library reports that it is the
bounds-checking build: through the normal build those inputs would read and
write outside the arrays.  Every bad id is planted where the traversal reads
it on its first level (the last entry of a row, which keeps the row sorted):
a row of the source for the top-down variants, a row of an unvisited vertex
for the pull variant, whose first probe loads the last entries of a row; the
tiled variant's tile builder reads every id and rejects the graph.
Prints one line per case and exits non-zero on the first failure.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_1104_4518_gb300 as bfs  # noqa: E402
from gpu_helpers import assert_same, device_graph_from_edges  # noqa: E402
from paper_1104_4518_gb300 import inputs  # noqa: E402

FORCED = [bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v) for v in range(bfs.BFS_NUM_VARIANTS)]


def say(msg):
    print(msg, flush=True)


def parity():
    """Well-formed graphs through the checked build: every selector, the batched,
    ragged, directed and static entry points, bit-identical to the oracle."""
    wpath = os.path.join(ROOT, "paper_1104_4518_gb300", "selector_weights.bin")
    el = inputs.rmat(14, 16, seed=61)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    roots = [int(r) for r in inputs.roots(el, 4, 62)]
    refs = oracle.bfs_many(og, roots)
    sels = [bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC)] + FORCED
    if os.path.exists(wpath):
        bfs.bfs_selector_load(wpath)
        sels.append(bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED))
    for s, ref in zip(roots, refs):
        for o in sels:
            parent, level = bfs.run(g, s, o)
            bfs.bfs_sync(g)
            assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"rmat14 root {s}")
    say("single-source rmat14: ok")
    broots = [int(r) for r in inputs.roots(el, 40, 63)]
    brefs = oracle.bfs_many(og, broots)
    for width in (64, 8):
        for td in (None, 1):
            bfs.bfs_set_tuning(g, batch_width=width)
            if td is not None:
                bfs.bfs_set_tuning(g, batch_topdown_limit=td)
            parent, level = bfs.run_batch(g, broots)
            bfs.bfs_sync(g)
            pa, lv = parent.cpu().numpy(), level.cpu().numpy()
            for i, ref in enumerate(brefs):
                assert_same(ref, (lv[i], pa[i]), f"batched width {width} td {td} row {i}")
    g.destroy()
    say("batched rmat14: ok")
    st = inputs.star(5000)  # a row of 4,999 entries: chunk items in both kernels
    og = oracle.csr_of(st)
    g = device_graph_from_edges(st)
    for s in (0, 1, 4999):
        for o in FORCED:
            parent, level = bfs.run(g, s, o)
            bfs.bfs_sync(g)
            assert_same(oracle.bfs(og, s), (level.cpu().numpy(), parent.cpu().numpy()), f"star root {s}")
    parent, level = bfs.run_batch(g, [0, 1, 4999])
    bfs.bfs_sync(g)
    for i, s in enumerate((0, 1, 4999)):
        assert_same(oracle.bfs(og, s), (level[i].cpu().numpy(), parent[i].cpu().numpy()), f"star batched {s}")
    g.destroy()
    say("star 5000: ok")
    dl = inputs.rmat(13, 8, seed=64)
    dg = oracle.digraph_of(dl)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(dl.src).cuda(), torch.from_numpy(dl.dst).cuda(), dl.n,
                                        directed=True)
    droots = [int(r) for r in inputs.roots(dl, 3, 65)]
    for s in droots:
        for o in [bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC)] + FORCED:
            parent, level = bfs.run(g, s, o)
            bfs.bfs_sync(g)
            assert_same(oracle.bfs_directed(dg, s), (level.cpu().numpy(), parent.cpu().numpy()), f"directed {s}")
    parent, level = bfs.run_batch(g, droots)
    bfs.bfs_sync(g)
    for i, s in enumerate(droots):
        assert_same(oracle.bfs_directed(dg, s), (level[i].cpu().numpy(), parent[i].cpu().numpy()),
                    f"directed batched {s}")
    g.destroy()
    say("directed rmat13: ok")
    parts_el = [inputs.rmat(sc, 8, seed=70 + sc) for sc in (9, 11, 10)]
    parts = [device_graph_from_edges(p) for p in parts_el]
    u = bfs.bfs_graph_union(parts)
    proots = [int(inputs.roots(p, 1, 80 + i)[0]) for i, p in enumerate(parts_el)]
    levels = [torch.empty(p.n, dtype=torch.int32, device="cuda") for p in parts_el]
    parents = [torch.empty(p.n, dtype=torch.int32, device="cuda") for p in parts_el]
    bfs.bfs_run_ragged(u, proots, parents, levels)
    bfs.bfs_sync(u)
    for p, s, lv, pa in zip(parts_el, proots, levels, parents):
        assert_same(oracle.bfs(oracle.csr_of(p), s), (lv.cpu().numpy(), pa.cpu().numpy()), f"ragged {p.name}")
    say("ragged union: ok")
    el = inputs.rmat(12, 16, seed=66)
    og = oracle.csr_of(el)
    off, adj = torch.from_numpy(og.offsets).cuda(), torch.from_numpy(og.adj).cuda()
    parent = torch.empty(el.n, dtype=torch.int32, device="cuda")
    level = torch.empty_like(parent)
    for s in [int(r) for r in inputs.roots(el, 3, 67)]:
        bfs.bfs_run_static(off, adj, s, parent, level)
        assert_same(oracle.bfs(og, s), (level.cpu().numpy(), parent.cpu().numpy()), f"static {s}")
    say("static entry: ok")


def expect_bounds(fn, site_words, what):
    try:
        fn()
    except bfs.BfsError as e:
        if e.code != bfs.BFS_ERR_BOUNDS:
            raise AssertionError(f"{what}: status {e.code}, expected BFS_ERR_BOUNDS: {e}")
        msg = str(e)
        if site_words and site_words not in msg:
            raise AssertionError(f"{what}: message {msg!r} does not name {site_words!r}")
        say(f"{what}: BFS_ERR_BOUNDS ({msg.split(': ', 1)[-1]})")
        return
    raise AssertionError(f"{what}: no error reported")


def malformed():
    if not bfs.bfs_bounds_checked():
        raise SystemExit("refusing to run malformed graphs through a library without bounds checks")
    el = inputs.rmat(12, 8, seed=68)
    og = oracle.csr_of(el)
    n = og.n
    deg = np.diff(og.offsets)
    s, x = [int(v) for v in np.nonzero(deg >= 2)[0][:2]]
    # top-down: the last entry of the source's row points past the vertices
    adj_td = og.adj.copy()
    adj_td[og.offsets[s + 1] - 1] = n + 5
    # pull: the last entry of an unvisited vertex's row (x != s) likewise
    adj_pull = og.adj.copy()
    adj_pull[og.offsets[x + 1] - 1] = n + 7
    # top-down, negative id: the first entry of the source's row
    adj_neg = og.adj.copy()
    adj_neg[og.offsets[s]] = -3
    off = torch.from_numpy(og.offsets).cuda()

    for name, adj_h, variants, site in (
            ("id n+5 in the source row", adj_td, range(3), "top-down adjacency id"),
            ("id -3 in the source row", adj_neg, range(3), "top-down adjacency id"),
            ("id n+7 in an unvisited row", adj_pull, [bfs.BFS_VARIANT_PULL], "pull adjacency id"),
            ("id n+7 in an unvisited row", adj_pull, [bfs.BFS_VARIANT_TILED], "tile adjacency id")):
        g = bfs.bfs_graph_create(off, torch.from_numpy(adj_h).cuda())  # no BFS_VALIDATE
        for v in variants:
            o = bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v)

            def one(o=o):
                bfs.run(g, s, o)
                bfs.bfs_sync(g)
            expect_bounds(one, site, f"{name}, {bfs.VARIANT_NAMES[v]}")
        g.destroy()

    # batched: top-down from one root vertex, and pull at level 0 (40 distinct roots, limit 1)
    g = bfs.bfs_graph_create(off, torch.from_numpy(adj_td).cuda())

    def batched_td():
        bfs.run_batch(g, [s, s])
        bfs.bfs_sync(g)
    expect_bounds(batched_td, "batched top-down adjacency id", "batched, id n+5 in the source row")
    g.destroy()
    g = bfs.bfs_graph_create(off, torch.from_numpy(adj_pull).cuda())
    bfs.bfs_set_tuning(g, batch_topdown_limit=1)
    broots = [int(r) for r in inputs.roots(el, 40, 69) if int(r) != x][:32]

    def batched_pull():
        bfs.run_batch(g, broots)
        bfs.bfs_sync(g)
    expect_bounds(batched_pull, "batched pull adjacency id", "batched, id n+7 in an unvisited row")
    g.destroy()

    # row offsets: checked where the graph is created
    bad_off = og.offsets.copy()
    bad_off[10] = bad_off[11] + 3
    expect_bounds(lambda: bfs.bfs_graph_create(torch.from_numpy(bad_off).cuda(), torch.from_numpy(og.adj).cuda()),
                  "row offsets", "decreasing row offsets at create")
    bad_end = og.offsets.copy()
    bad_end[-1] -= 1
    expect_bounds(lambda: bfs.bfs_graph_create(torch.from_numpy(bad_end).cuda(), torch.from_numpy(og.adj).cuda()),
                  "row offsets", "offsets[n] != nnz at create")

    # the static entry point: offsets checked per call, ids in the kernel
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty_like(parent)
    expect_bounds(lambda: bfs.bfs_run_static(torch.from_numpy(bad_off).cuda(), torch.from_numpy(og.adj).cuda(), s,
                                             parent, level), "row offsets", "static, decreasing row offsets")
    expect_bounds(lambda: bfs.bfs_run_static(off, torch.from_numpy(adj_td).cuda(), s, parent, level),
                  "top-down adjacency id", "static, id n+5 in the source row")

    # the device and the library stay usable: a clean graph after the errors
    g = bfs.bfs_graph_create(off, torch.from_numpy(og.adj).cuda())
    ref = oracle.bfs(og, s)
    for o in [bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC)] + FORCED:
        parent, level = bfs.run(g, s, o)
        bfs.bfs_sync(g)
        assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), "clean run after the errors")
    parent, level = bfs.run_batch(g, [s, x])
    bfs.bfs_sync(g)
    assert_same(ref, (level[0].cpu().numpy(), parent[0].cpu().numpy()), "clean batched run after the errors")
    bfs.bfs_run_static(off, torch.from_numpy(og.adj).cuda(), s, parent[0], level[0])
    assert_same(ref, (level[0].cpu().numpy(), parent[0].cpu().numpy()), "clean static run after the errors")
    g.destroy()
    say("clean runs after the errors: ok")


if __name__ == "__main__":
    if not torch.cuda.is_available():
        raise SystemExit("needs a CUDA device")
    if not bfs.bfs_bounds_checked():
        raise SystemExit("BFS_BOUNDS_CHECK=1 must select the bounds-checking library")
    {"parity": parity, "malformed": malformed}[sys.argv[1]]()
    say("done")
