"""Host logic of the multi-GPU benchmark path (independent replicas), run as two gloo
ranks on the CPU: the timed-region length is the maximum over ranks, the traversed
edges are summed, and each rank draws its own seeded roots."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, e = bench.aggregate(1.5 + rank, 1000 * (rank + 1))
    wl = dict(bench.WORKLOADS["rmat16"])
    wl["scale"] = 10
    _, roots = bench.make_workload(wl, rank)
    out[rank] = (t, e, roots.tolist(), bench.dist_env())
    bench.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        t, e, roots, env = res[rank]
        assert t == pytest.approx(2.5)  # max over ranks
        assert e == 3000  # sum over ranks
        assert env == (rank, world, rank)
    assert res[0][2] != res[1][2]  # each replica draws its own roots
    assert len(set(res[0][2])) == len(res[0][2])
