"""The library's 2D DCSC tiles (bfs_graph_tiles) and the tiled variant, against the oracle.

- The tiles built on the device equal `oracle.dcsc_tiles` array for array, for
  several row / column block sizes, on undirected and directed graphs (the
  directed tiles are those of the in-rows, the transpose).
- BFS_VARIANT_TILED forced at every level, and mixed into schedules, gives the
  oracle's levels and parents bit for bit, for several tile layouts, including
  layouts where a graph has a single tile or thousands.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu

TILED = bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=bfs.BFS_VARIANT_TILED)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def assert_tiles_equal(got, ref):
    assert got["ntiles"] == ref["ntiles"] and got["nzc"] == ref["nzc"]
    for key in ("tdir_jc", "tdir_ir", "jc", "cp", "ir"):
        assert np.array_equal(got[key].astype(np.int64), ref[key]), key


@pytest.mark.parametrize("rb_bits,cb_bits", [(5, 5), (8, 6), (6, 12), (16, 16), (10, 16)])
def test_tiles_equal_the_oracle_dcsc(rb_bits, cb_bits):
    el = inputs.rmat(13, 16, seed=31)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    got = bfs.bfs_graph_tiles(g, rb_bits, cb_bits)
    g.destroy()
    assert got["rb_bits"] == rb_bits and got["cb_bits"] == cb_bits
    assert_tiles_equal(got, oracle.dcsc_tiles(og, 1 << rb_bits, 1 << cb_bits))


def test_directed_tiles_are_those_of_the_in_rows():
    el = inputs.rmat(12, 8, seed=32)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    got = bfs.bfs_graph_tiles(g, 7, 9)
    g.destroy()
    in_rows = oracle.digraph_csr(el.dst, el.src, el.n)  # row v lists the tails u of the arcs u -> v
    assert_tiles_equal(got, oracle.dcsc_tiles(in_rows, 1 << 7, 1 << 9))


def test_default_layout_and_rebuild():
    el = inputs.rmat(14, 16, seed=33)
    g = device_graph_from_edges(el)
    d = bfs.bfs_graph_tiles(g, host_copy=False)
    assert d["cb_bits"] == 16 and 8 <= d["rb_bits"] <= 16 and d["nnz"] == g.info()[1]
    again = bfs.bfs_graph_tiles(g, 5, 7, host_copy=False)
    assert again["rb_bits"] == 5 and again["cb_bits"] == 7 and again["nrb"] == (1 << 14) // 32
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_tiles(g, 17, 0)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    g.destroy()


@pytest.mark.parametrize("layout", [None, (5, 5), (8, 16), (12, 6), (16, 16)])
def test_tiled_variant_matches_the_oracle(layout):
    el, roots = inputs.workload_rmat(14, 6, graph_seed=34, root_seed=134)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    if layout is not None:
        bfs.bfs_graph_tiles(g, *layout, host_copy=False)
    refs = oracle.bfs_many(og, roots)
    for s, ref in zip(roots, refs):
        parent, level = bfs.run(g, int(s), TILED)
        bfs.bfs_sync(g)
        assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"tiled, layout {layout}, root {s}")
    g.destroy()


def test_tiled_variant_in_schedules_and_on_grids_and_directed_graphs():
    rng = np.random.default_rng(35)
    # a 3D grid: long thin frontiers, many levels, a single column block
    el = inputs.grid3d(20)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    ref = oracle.bfs(og, 0)
    for opts in (TILED, bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE,
                                       schedule=[int(x) for x in rng.integers(0, bfs.BFS_NUM_VARIANTS, 40)])):
        parent, level = bfs.run(g, 0, opts)
        bfs.bfs_sync(g)
        assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), "grid 20^3")
    g.destroy()
    # directed R-MAT: the tiles are the in-rows, the next level's degrees the out-rows
    el = inputs.rmat(12, 8, seed=36)
    dg = oracle.digraph_of(el)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n,
                                        directed=True)
    bfs.bfs_graph_tiles(g, 6, 8, host_copy=False)
    outdeg = np.diff(dg.offsets)
    for s in [int(r) for r in inputs.roots(el, 20, 136) if outdeg[r] > 0][:4]:
        ref = oracle.bfs_directed(dg, s)
        for opts in (TILED, bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE,
                                           schedule=[int(x) for x in rng.integers(0, bfs.BFS_NUM_VARIANTS, 12)])):
            parent, level = bfs.run(g, s, opts)
            bfs.bfs_sync(g)
            assert_same(ref, (level.cpu().numpy(), parent.cpu().numpy()), f"directed root {s}")
    g.destroy()
