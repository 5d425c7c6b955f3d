"""One suspension split by target rows, on the GPU.

The pair-sum kernel computes each rank's row block with the unsharded run's
i-blocks, j-split and j-order, and the ranks all-gather the packed records
after every evaluation, so every rank's dumbbells must follow the unsharded
grid path bit for bit:

* several shards in one process on one GPU (records exchanged by device
  copies), FP32C and FP64, RPY and Oseen, ragged last blocks;
* two processes on one GPU exchanging through gloo (host copies): the
  multi-process form of the path, with its collective.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1004_1932_b300 import dbs, inputs, shard

pytestmark = pytest.mark.gpu


def _reference(s, precision, steps):
    with dbs.Suspension.from_inputs(s, precision=precision) as h:
        h.step(steps)
        return h.positions()


@pytest.mark.parametrize("S,precision,mob,nranks", [(300, "fp32c", "rpy", 2), (2049, "fp32c", "rpy", 3),
                                                    (700, "fp64", "oseen", 2), (8193, "fp32c", "oseen", 4),
                                                    (33, "fp32c", "rpy", 2)])
def test_local_shards_are_bit_identical_to_unsharded(S, precision, mob, nranks):
    import torch
    torch.cuda.set_device(0)
    s = inputs.make_suspension(S, seed=40 + S, density=0.002, mobility=mob)
    steps = 60
    ref = _reference(s, precision, steps)
    stream = torch.cuda.Stream()
    shards = [shard.Shard(s, nranks, r, precision=precision, stream=stream) for r in range(nranks)]
    try:
        assert [(sh.row0, sh.row1) for sh in shards] == shards[0].blocks
        shard.step(shards, steps, shard.LocalExchange())
        stream.synchronize()
        for sh in shards:
            assert sh.h.get_time()[0] == steps
            assert np.array_equal(sh.positions(), ref[2 * sh.row0:2 * sh.row1])
    finally:
        for sh in shards:
            sh.close()


def test_sharded_handle_refuses_plain_steps():
    s = inputs.make_suspension(100, seed=3, density=0.002)
    with dbs.Suspension.from_inputs(s) as h:
        h.shard_set(2, 0)
        with pytest.raises(dbs.DbsError) as ei:
            h.step(1)
        assert ei.value.status == dbs.E_STATE


def _free_port():
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    p = sk.getsockname()[1]
    sk.close()
    return p


def _rank(rank, world, port, S, steps, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s = inputs.make_suspension(S, seed=77, density=0.002)
    sh = shard.Shard(s, world, rank)
    shard.step([sh], steps, shard.GroupExchange())
    sh.stream.synchronize()
    out[rank] = (sh.row0, sh.row1, sh.positions().tobytes())
    sh.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_exchange_through_gloo():
    S, steps, world = 1500, 40, 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, S, steps, out), nprocs=world, join=True)
        res = dict(out)
    import torch
    torch.cuda.set_device(0)
    ref = _reference(inputs.make_suspension(S, seed=77, density=0.002), "fp32c", steps)
    covered = 0
    for r in range(world):
        r0, r1, xb = res[r]
        x = np.frombuffer(xb, dtype=np.float64).reshape(-1, 3)
        assert np.array_equal(x, ref[2 * r0:2 * r1])
        covered += r1 - r0
    assert covered == S
