"""Shared helpers of the GPU parity tests: build graphs both ways, compare with the oracle."""
import numpy as np
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from paper_1104_4518_gb300 import inputs


def require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    bfs.lib()


def device_graph_from_edges(el: inputs.EdgeList) -> bfs.Graph:
    """Graph built by the library's device CSR builder from a host edge list copied to the GPU."""
    src = torch.from_numpy(el.src).cuda()
    dst = torch.from_numpy(el.dst).cuda()
    g = bfs.bfs_graph_create_from_edges(src, dst, el.n)
    torch.cuda.synchronize()
    return g


def device_graph_from_oracle_csr(g: oracle.CSR, validate=True) -> bfs.Graph:
    return bfs.bfs_graph_create(torch.from_numpy(g.offsets).cuda(), torch.from_numpy(g.adj).cuda(),
                                validate=validate)


def run_gpu(g: bfs.Graph, s: int, opts=None):
    """(level, parent) as NumPy arrays."""
    parent, level = bfs.run(g, s, opts)
    bfs.bfs_sync(g)
    return level.cpu().numpy(), parent.cpu().numpy()


def assert_same(ref, got, what=""):
    level_ref, parent_ref = ref[0], ref[1]
    level_got, parent_got = got
    if not np.array_equal(level_ref, level_got):
        bad = np.nonzero(level_ref != level_got)[0]
        raise AssertionError(f"{what}: {bad.size} level mismatches, first at v={bad[0]}: "
                             f"oracle {level_ref[bad[0]]} gpu {level_got[bad[0]]}")
    if not np.array_equal(parent_ref, parent_got):
        bad = np.nonzero(parent_ref != parent_got)[0]
        raise AssertionError(f"{what}: {bad.size} parent mismatches, first at v={bad[0]}: "
                             f"oracle {parent_ref[bad[0]]} gpu {parent_got[bad[0]]} (level {level_ref[bad[0]]})")


def check_roots(el, roots, selectors=((bfs.BFS_SELECT_HEURISTIC, 0),), via_edges=True, oracle_csr=None):
    """Runs the GPU BFS for every root and selector and compares with the oracle bit for bit."""
    og = oracle_csr if oracle_csr is not None else oracle.csr_of(el)
    g = device_graph_from_edges(el) if via_edges else device_graph_from_oracle_csr(og)
    refs = oracle.bfs_many(og, roots)
    for (sel, var) in selectors:
        for s, ref in zip(roots, refs):
            opts = bfs.RunOptions(selector=sel, forced_variant=var, want_counts=True)
            parent, level = bfs.run(g, int(s), opts)
            got = (level.cpu().numpy(), parent.cpu().numpy())
            assert_same(ref, got, f"{el.name} root {s} selector {sel}/{var}")
            assert opts.nlevels == ref[2]
            assert opts.edges == oracle.component_edges(og, ref[0])
    return g, og, refs
