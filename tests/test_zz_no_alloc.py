"""bfs_run_static: the BFS entry point that allocates nothing.

Some callers of this library cannot call cudaMalloc (a plug-in or a real-time
loop that must not trigger an allocation's device synchronisation or risk its
failure, or a process whose device memory is reserved up front by another
allocator).  For them bfs_run_static keeps all scratch of a traversal in a
fixed static array inside the library; the caller passes only the CSR and the
outputs.  These tests call it through the C ABI twice in a row, on two
different graphs, and compare each result with the allocating entry point
bfs_run and with the CPU oracle (the outputs are integers, so both comparisons
are exact); a third case fills the array to its vertex limit.  They need no
state from other tests and pass alone in a fresh process as well as after the
suite.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")


def _check_against_bfs_run_and_oracle(el, source):
    og = oracle.csr_of(el)
    off, adj = torch.from_numpy(og.offsets).cuda(), torch.from_numpy(og.adj).cuda()
    n = el.n
    parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    level = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    bfs.bfs_run_static(off, adj, source, parent, level)
    got = (parent.cpu().numpy(), level.cpu().numpy())
    g = bfs.bfs_graph_create(off, adj)
    ref_parent, ref_level = bfs.run(g, source)
    bfs.bfs_sync(g)
    g.destroy()
    assert np.array_equal(got[0], ref_parent.cpu().numpy()) and np.array_equal(got[1], ref_level.cpu().numpy())
    o_level, o_parent, _ = oracle.bfs(og, source)
    assert np.array_equal(got[1], o_level) and np.array_equal(got[0], o_parent)
    assert (got[1] >= 0).sum() > 1
    return off, adj, parent, level


def test_static_entry_point_matches_bfs_run_and_the_oracle_on_two_calls_in_a_row():
    _require_cuda()
    first = inputs.rmat(16, 16, seed=1)
    second = inputs.grid3d(24)  # a different shape, many levels
    for el, s in ((first, int(inputs.roots(first, 1, 101)[0])), (second, 0)):
        _check_against_bfs_run_and_oracle(el, s)


def test_static_entry_point_at_its_vertex_limit_allocates_nothing():
    """R-MAT scale 20 (n = 1,048,576, the array's vertex limit; about 31 M CSR
    entries).  After a first call, a second call leaves the device's free memory
    unchanged, and its result still matches bfs_run and the oracle."""
    _require_cuda()
    el = inputs.rmat(20, 16, seed=20)
    s = int(inputs.roots(el, 1, 120)[0])
    off, adj, parent, level = _check_against_bfs_run_and_oracle(el, s)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    parent.fill_(7)
    level.fill_(7)
    torch.cuda.synchronize()
    bfs.bfs_run_static(off, adj, s, parent, level)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    o_level, o_parent, _ = oracle.bfs(oracle.CSR(off.cpu().numpy(), adj.cpu().numpy()), s)
    assert np.array_equal(level.cpu().numpy(), o_level) and np.array_equal(parent.cpu().numpy(), o_parent)


def test_static_entry_point_rejects_sizes_beyond_its_scratch():
    _require_cuda()
    n = (1 << 20) + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    adj = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run_static(off, adj, 0, out, out)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG and "static scratch" in str(e.value)
