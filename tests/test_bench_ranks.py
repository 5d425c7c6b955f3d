"""Host logic of bench.py's multi-GPU mode on CPU ranks (gloo, world size 2):
every rank times its own independent suspension (seed = rank) and the job
time is the maximum over ranks; the aggregate counts all ranks' work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1004_1932_b300 import inputs
    elapsed = 1.5 + rank                       # rank 1 is the slow one
    out[rank] = (bench.reduce_max(elapsed), bench.rank_seed(rank),
                 float(inputs.paper_scale(16, seed=bench.rank_seed(rank)).x0[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_max_time_and_distinct_systems():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5          # max over ranks, seen by every rank
    assert res[0][1] != res[1][1]                 # distinct seeds
    assert res[0][2] != res[1][2]                 # hence distinct suspensions


def test_reduce_max_without_process_group():
    import bench
    assert bench.reduce_max(3.25) == 3.25
