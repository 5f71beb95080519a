"""Host outputs of bfs_run: synchronous (BFS_HOST_PTRS) and asynchronous
(BFS_HOST_PTRS | BFS_HOST_ASYNC, double-buffered staging on the device and a
copy stream).  Several traversals are enqueued back to back, each into its own
pinned host arrays, and after bfs_sync every array equals the oracle's result
bit for bit; synchronous and asynchronous calls may be mixed on one stream."""
import numpy as np
import pytest
import torch

import oracle
import paper_1104_4518_gb300 as bfs
from gpu_helpers import assert_same, device_graph_from_edges, require_cuda
from paper_1104_4518_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def test_async_host_outputs_of_back_to_back_traversals():
    el, roots = inputs.workload_rmat(16, 7, graph_seed=71, root_seed=171)
    og = oracle.csr_of(el)
    g = device_graph_from_edges(el)
    n = el.n
    outs = [(torch.full((n,), 9, dtype=torch.int32).pin_memory(), torch.full((n,), 9, dtype=torch.int32).pin_memory())
            for _ in roots]
    ao = bfs.RunOptions(host_outputs=True, host_async=True)
    so = bfs.RunOptions(host_outputs=True)
    for i, (s, (hp, hl)) in enumerate(zip(roots, outs)):
        bfs.bfs_run(g, int(s), hp, hl, so if i == 3 else ao)  # one synchronous call in the middle
    bfs.bfs_sync(g)
    refs = oracle.bfs_many(og, roots)
    for s, ref, (hp, hl) in zip(roots, refs, outs):
        assert_same(ref, (hl.numpy(), hp.numpy()), f"host outputs, root {s}")
    # pageable host arrays work too (the copies are then staged by the driver)
    hp, hl = np.full(n, 9, np.int32), np.full(n, 9, np.int32)
    bfs.bfs_run(g, int(roots[0]), hp, hl, ao)
    bfs.bfs_sync(g)
    assert_same(refs[0], (hl, hp), "pageable host outputs")
    g.destroy()
