"""bfs_run_static: the BFS entry point that allocates nothing.

Some callers of this library cannot call cudaMalloc (a plug-in or a real-time
loop that must not trigger an allocation's device synchronisation or risk its
failure, or a process whose device memory is reserved up front by another
allocator).  For them bfs_run_static keeps all scratch of a traversal in a
fixed static array inside the library; the caller passes only the CSR and the
outputs.  This test calls it through the C ABI twice in a row, on two different
graphs, and compares each result with the allocating entry point bfs_run (the
outputs are integers, so the comparison is exact).  It needs no state from
other tests and passes alone in a fresh process as well as after the suite.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


def _csr_on_device(el):
    og = oracle.csr_of(el)
    return torch.from_numpy(og.offsets).cuda(), torch.from_numpy(og.adj).cuda()


def _static_and_reference(el, source):
    off, adj = _csr_on_device(el)
    n = el.n
    parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    level = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    bfs.bfs_run_static(off, adj, source, parent, level)
    g = bfs.bfs_graph_create(off, adj)
    ref_parent, ref_level = bfs.run(g, source)
    bfs.bfs_sync(g)
    return (parent.cpu().numpy(), level.cpu().numpy()), (ref_parent.cpu().numpy(), ref_level.cpu().numpy())


def test_static_entry_point_matches_bfs_run_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    first = inputs.rmat(16, 16, seed=1)
    second = inputs.grid3d(24)  # a different shape, many levels
    for el, s in ((first, int(inputs.roots(first, 1, 101)[0])), (second, 0)):
        got, ref = _static_and_reference(el, s)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        assert (got[1] >= 0).sum() > 1


def test_static_entry_point_rejects_sizes_beyond_its_scratch():
    n = (1 << 20) + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    adj = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run_static(off, adj, 0, out, out)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG and "static scratch" in str(e.value)
