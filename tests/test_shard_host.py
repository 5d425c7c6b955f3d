"""Host logic of one suspension split by target rows (no GPU).

* The row blocks of dbs_shard_rows: contiguous, covering [0, S) once, aligned
  to the pair-sum kernel's i-blocks, balanced to one i-block; too many ranks
  for the i-blocks is refused.
* The record all-gather on CPU ranks (gloo, world size 2 and 3): every rank
  fills its own block of a byte buffer and leaves garbage elsewhere; after the
  exchange every rank holds every block, bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1004_1932_b300 import dbs, shard


@pytest.mark.parametrize("S,bt", [(1, 32), (31, 32), (32, 32), (33, 32), (1000, 32), (2048, 32),
                                  (2049, 256), (8192, 256), (8193, 512), (32768, 512), (300, 128)])
def test_row_blocks_partition_the_suspension(S, bt):
    nb = -(-S // bt)
    for nranks in range(1, min(nb, 9) + 1):
        blocks = shard.all_blocks(S, bt, nranks)
        assert blocks[0][0] == 0 and blocks[-1][1] == S
        for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
            assert a1 == b0                          # contiguous
        nblk = [-(-(r1 - r0) // bt) for r0, r1 in blocks]
        assert all(k > 0 for k in nblk) and max(nblk) - min(nblk) <= 1
        assert all(r0 % bt == 0 for r0, _ in blocks)   # i-block aligned
    with pytest.raises(dbs.DbsError):
        shard.shard_rows(S, bt, nb + 1, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, S, rb, bt, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    blocks = shard.all_blocks(S, bt, world)
    rng = np.random.default_rng(rank + 100)
    buf = torch.from_numpy(rng.integers(0, 256, size=S * rb, dtype=np.uint8))   # garbage
    r0, r1 = blocks[rank]
    own = np.random.default_rng(7 + rank).integers(0, 256, size=(r1 - r0) * rb, dtype=np.uint8)
    buf[r0 * rb:r1 * rb] = torch.from_numpy(own)
    shard.gather_blocks(buf, blocks, rank, rb)
    out[rank] = buf.numpy().tobytes()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,S,bt", [(2, 100, 32), (3, 1000, 32), (2, 2049, 256)])
def test_record_gather_on_cpu_ranks(world, S, bt):
    rb = 48
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, S, rb, bt, out), nprocs=world, join=True)
        res = dict(out)
    blocks = shard.all_blocks(S, bt, world)
    expect = np.empty(S * rb, dtype=np.uint8)
    for r, (r0, r1) in enumerate(blocks):
        expect[r0 * rb:r1 * rb] = np.random.default_rng(7 + r).integers(0, 256, size=(r1 - r0) * rb,
                                                                       dtype=np.uint8)
    for r in range(world):
        assert res[r] == expect.tobytes()
