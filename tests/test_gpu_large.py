"""Full-size checks in the benchmark's launch configurations.

Every root of the scale-26 benchmark is validated, and the scale-24 batched
traversal row by row; the selector's held-out graphs run under the learned
selector.

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


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1104_4518_gb300",
                       "selector_weights.bin")


class Validations:
    """Runs `oracle.validate_edges` on host copies of GPU results, a bounded number at
    a time on a thread pool (the C validator drops the GIL), and collects failures."""

    def __init__(self, el, workers=None):
        self.el = el
        self.workers = workers or min(16, os.cpu_count() or 1)
        self.ex = ThreadPoolExecutor(max_workers=self.workers)
        self.pending = []
        self.checked = 0

    def submit(self, what, root, level, parent):
        if len(self.pending) >= 2 * self.workers:
            self._drain(self.workers)
        lv = level.cpu().numpy() if isinstance(level, torch.Tensor) else level
        pa = parent.cpu().numpy() if isinstance(parent, torch.Tensor) else parent
        fut = self.ex.submit(oracle.validate_edges, self.el.src, self.el.dst, self.el.n, int(root), lv, pa)
        self.pending.append((what, fut))

    def _drain(self, keep=0):
        while len(self.pending) > keep:
            what, fut = self.pending.pop(0)
            bad = fut.result()
            assert bad.sum() == 0, (what, bad.tolist())
            self.checked += 1

    def finish(self):
        try:
            self._drain()
        finally:
            self.ex.shutdown()
        return self.checked


def _validate_rows(el, roots, levels, parents):
    v = Validations(el, workers=min(len(roots), os.cpu_count() or 1))
    for i in range(len(roots)):
        v.submit(f"row {i}", roots[i], levels[i], parents[i])
    v.finish()


@pytest.fixture(scope="module")
def rmat26():
    """The scale-26 benchmark graph (67 M vertices, 2.1 G CSR entries; graph seed 3,
    roots 103) on the device, built by the library's CSR builder."""
    el, roots = inputs.workload_rmat(26, 64, graph_seed=3, root_seed=103)
    g = device_graph_from_edges(el)
    yield el, [int(r) for r in roots], g
    g.destroy()


def test_rmat26_every_bench_root_and_the_batched_traversal(rmat26):
    """All 64 benchmark roots at scale 26, heuristic selector (the benchmark's launch
    configuration): every result validated edge by edge against the oracle's rule.
    The benchmark's 64-root batched traversal of the same roots gives the same rows,
    bit for bit, compared on the device."""
    el, roots, g = rmat26
    pb, lb = bfs.run_batch(g, roots)
    bfs.bfs_sync(g)
    val = Validations(el)
    deep = 0
    for i, s in enumerate(roots):
        parent, level = bfs.run(g, s)
        bfs.bfs_sync(g)
        assert torch.equal(pb[i], parent) and torch.equal(lb[i], level), f"batched row {i} (root {s})"
        deep += int(level.max().item() >= 3)
        val.submit(f"root {s}", s, level, parent)
    del pb, lb
    assert val.finish() == 64
    assert deep >= 60  # real traversals of the large component, not trivial ones


def test_rmat26_forced_variants_schedules_and_learned_selector(rmat26):
    """At scale 26, four benchmark roots under every forced variant, a random per-level
    schedule and the learned selector with the shipped weights: each result is
    bit-identical to the heuristic run of the same root, and those runs are validated
    edge by edge against the oracle's rule."""
    el, roots, g = rmat26
    picks = roots[:4]
    val = Validations(el)
    rng = np.random.default_rng(26)
    bfs.bfs_selector_load(WEIGHTS)
    try:
        for s in picks:
            parent, level = bfs.run(g, s)
            bfs.bfs_sync(g)
            val.submit(f"heuristic root {s}", s, level, parent)
            runs = [(f"forced {v}", bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v))
                    for v in range(bfs.BFS_NUM_VARIANTS)]
            runs.append(("schedule", bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE,
                                                    schedule=rng.integers(0, bfs.BFS_NUM_VARIANTS, 16))))
            runs.append(("learned", bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED)))
            for name, o in runs:
                p2, l2 = bfs.run(g, s, o)
                bfs.bfs_sync(g)
                assert torch.equal(p2, parent) and torch.equal(l2, level), (name, s)
    finally:
        bfs.bfs_selector_set_params(None)
    assert val.finish() == len(picks)


def test_rmat26_learned_selector_beats_the_heuristic(rmat26):
    """On the scale-26 benchmark graph, the 64 bench roots traversed with the learned
    selector (shipped weights) take less device time than with the fixed-threshold
    heuristic: alternating rounds, the median of three for each.  (The network
    keeps pull one level longer where the heuristic's exit threshold leaves it
    early, and runs the last levels thread-per-vertex.)"""
    _, roots, g = rmat26
    n = g.info()[0]
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_selector_load(WEIGHTS)
    try:
        times = {bfs.BFS_SELECT_HEURISTIC: [], bfs.BFS_SELECT_LEARNED: []}
        for rnd in range(4):
            for sel in times:
                o = bfs.RunOptions(selector=sel)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for s in roots:
                    bfs.bfs_run(g, s, parent, level, o)
                e1.record()
                torch.cuda.synchronize()
                if rnd > 0:  # the first round warms up
                    times[sel].append(e0.elapsed_time(e1))
        heur, learned = (float(np.median(times[s])) for s in (bfs.BFS_SELECT_HEURISTIC, bfs.BFS_SELECT_LEARNED))
        print(f"\nscale 26, 64 roots: heuristic {heur:.2f} ms, learned {learned:.2f} ms")
        assert learned < heur, (learned, heur)
    finally:
        bfs.bfs_selector_set_params(None)


def test_heldout_rmat25_learned_selector():
    """The selector's held-out R-MAT graph (scale 25, edgefactor 16, graph seed 7,
    8 roots of seed 107) traversed with the learned selector and the shipped weights:
    every result validated edge by edge against the oracle's rule."""
    el = inputs.rmat(25, 16, seed=7)
    roots = [int(r) for r in inputs.roots(el, 8, 107)]
    g = device_graph_from_edges(el)
    bfs.bfs_selector_load(WEIGHTS)
    val = Validations(el)
    try:
        for s in roots:
            o = bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED, want_counts=True)
            parent, level = bfs.run(g, s, o)
            bfs.bfs_sync(g)
            assert o.nlevels >= 3
            val.submit(f"learned root {s}", s, level, parent)
    finally:
        bfs.bfs_selector_set_params(None)
        g.destroy()
    assert val.finish() == len(roots)


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


@pytest.mark.parametrize("selector", ["heuristic", "learned"])
def test_grid256_closed_form(selector):
    """The 256^3 grid from the corner (766 levels; the selector's held-out grid):
    level = x + y + z and the max-id parent, under the heuristic and under the learned
    selector with the shipped weights."""
    N = 256
    el = inputs.grid3d(N)
    g = device_graph_from_edges(el)
    learned = selector == "learned"
    if learned:
        bfs.bfs_selector_load(WEIGHTS)
    try:
        parent, level = bfs.run(g, 0, bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED) if learned else None)
        bfs.bfs_sync(g)
    finally:
        if learned:
            bfs.bfs_selector_set_params(None)
        g.destroy()
    level, parent = level.cpu().numpy(), parent.cpu().numpy()
    v = np.arange(N ** 3, dtype=np.int64)
    x, y, z = v % N, (v // N) % N, v // (N * N)
    assert np.array_equal(level, (x + y + z).astype(np.int32))
    exp = np.where(x > 0, v - 1, np.where(y > 0, v - N, v - N * N))
    exp[0] = 0
    assert np.array_equal(parent, exp.astype(np.int32))


@pytest.mark.parametrize("ef", [4, 8, 16, 32, 64])
def test_degree_sweep_graphs_validated(ef):
    """The graphs of the average-degree sweep (`paper_1104_4518_gb300.sweep`: R-MAT with
    2^27 generated edges, edgefactor ef, scale 27 - log2 ef, graph seed 40 + ef, roots
    seed 140 + ef): the first sweep root under the heuristic and the learned selector,
    and the first two rows of the batched traversal of the sweep's 16 roots, validated
    edge by edge against the oracle's rule."""
    from paper_1104_4518_gb300 import sweep

    scale = sweep.LOG2_EDGES - int(np.log2(ef))
    el = inputs.rmat(scale, ef, seed=40 + ef)
    roots = [int(r) for r in inputs.roots(el, 16, 140 + ef)]
    g = device_graph_from_edges(el)
    val = Validations(el)
    bfs.bfs_selector_load(WEIGHTS)
    try:
        for sel in (bfs.BFS_SELECT_HEURISTIC, bfs.BFS_SELECT_LEARNED):
            parent, level = bfs.run(g, roots[0], bfs.RunOptions(selector=sel))
            bfs.bfs_sync(g)
            val.submit(f"ef {ef} selector {sel}", roots[0], level, parent)
        pb, lb = bfs.run_batch(g, roots)
        bfs.bfs_sync(g)
        for i in range(2):
            val.submit(f"ef {ef} batched row {i}", roots[i], lb[i], pb[i])
        del pb, lb
    finally:
        bfs.bfs_selector_set_params(None)
        g.destroy()
    assert val.finish() == 4
