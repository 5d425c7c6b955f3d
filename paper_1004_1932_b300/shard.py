"""One suspension split by target rows over several ranks.

The pair sum of Eq. (3b) splits by target rows: a sphere's velocity needs every
record but only its own dumbbell's state.  Each rank holds a full copy of the
suspension (a grid-path handle of libdbs) and computes the Heun evaluations
(Sec. IV) of one contiguous block of dumbbells (``dbs_shard_set``); after
every evaluation the ranks all-gather the packed records of their blocks into
every rank's record buffer (``dbs_shard_buffers``), so that the next evaluation
again sees all S records.  The j-order, the j-split and the i-blocks of every
sum are those of the unsharded grid path, so each rank's rows are
bit-identical to an unsharded run.

Exchanges (argument marshalling and collectives only; the arithmetic is in the
library's kernels):

* ``GroupExchange`` -- one shard per process over a ``torch.distributed``
  group.  NCCL gathers the device buffers directly (stream-ordered on the
  current stream, no host synchronisation); other backends (gloo) go through
  host copies.  Blocks are padded to the largest for the gather.
* ``LocalExchange`` -- several shards of one process on one device (device
  copies): the in-process form, used to check bit-identity on one GPU.
"""
from __future__ import annotations

import ctypes

from . import dbs


def shard_rows(S: int, rows_per_block: int, nranks: int, rank: int) -> tuple[int, int]:
    """Row block [row0, row1) of rank ``rank`` (``dbs_shard_rows``, host only)."""
    r0, r1 = ctypes.c_int64(), ctypes.c_int64()
    rc = dbs.load().dbs_shard_rows(ctypes.c_int64(int(S)), ctypes.c_int32(int(rows_per_block)),
                                   ctypes.c_int32(int(nranks)), ctypes.c_int32(int(rank)),
                                   ctypes.byref(r0), ctypes.byref(r1))
    if rc != dbs.OK:
        raise dbs.DbsError(rc, "dbs_shard_rows")
    return r0.value, r1.value


def all_blocks(S: int, rows_per_block: int, nranks: int) -> list[tuple[int, int]]:
    return [shard_rows(S, rows_per_block, nranks, r) for r in range(nranks)]


class Shard:
    """Rank ``rank``'s part of a suspension split over ``nranks`` ranks.  Its
    evaluations and exchanges run on one torch stream (``stream``, or a new one:
    the legacy default stream is not used, because the library would then run on
    a private stream that the exchange's copies do not wait for)."""

    def __init__(self, susp, nranks: int, rank: int, precision: str = "fp32c", stream=None,
                 device: int = -1):
        import torch
        dev = torch.device("cuda", device if device >= 0 else torch.cuda.current_device())
        if stream is None or int(stream.cuda_stream) == 0:
            stream = torch.cuda.Stream(device=dev)
        self.stream = stream
        self.device_index = dev.index
        self.h = dbs.Suspension.from_inputs(susp, precision=precision, stream=stream, device=dev.index)
        self.S = susp.S
        self.rank, self.nranks = rank, nranks
        self.row0, self.row1 = self.h.shard_set(nranks, rank)
        self.rows_per_block = self.h.get_launch()["bt"]
        self.blocks = all_blocks(self.S, self.rows_per_block, nranks)
        self.buf_a, self.buf_b, self.record_bytes = self.h.shard_buffers()

    def close(self):
        self.h.close()

    def positions(self):
        """FP64 positions [2 (row1 - row0), 3] of this rank's dumbbells."""
        return self.h.positions()[2 * self.row0:2 * self.row1]


def step(shards, n: int, exchange) -> None:
    """n Heun steps of the shards (this process's part of the split): every
    evaluation on every local shard, then the exchange of the buffer it wrote,
    all in order on the shards' one stream."""
    import torch
    stream = shards[0].stream
    if any(s.stream.cuda_stream != stream.cuda_stream for s in shards):
        raise ValueError("the shards of one process must share one stream")
    with torch.cuda.stream(stream):
        for _ in range(n):
            for s in shards:
                s.h.shard_eval(0)
            exchange([s.buf_b for s in shards], shards)
            for s in shards:
                s.h.shard_eval(1)
            exchange([s.buf_a for s in shards], shards)


def _device_bytes(ptr: int, nbytes: int, device_index: int):
    import torch
    view = dbs.DeviceView(ptr, (nbytes,), device_index=device_index, typestr="|u1")
    return torch.as_tensor(view, device=torch.device("cuda", device_index))


class LocalExchange:
    """All shards of one split held by this process on one device: copy every
    shard's block into every other shard's buffer (on the shards' stream)."""

    def __call__(self, ptrs, shards):
        rb = shards[0].record_bytes
        total = shards[0].S * rb
        bufs = [_device_bytes(p, total, s.device_index) for p, s in zip(ptrs, shards)]
        for src, s in zip(bufs, shards):
            lo, hi = s.row0 * rb, s.row1 * rb
            for dst in bufs:
                if dst is not src:
                    dst[lo:hi].copy_(src[lo:hi])


def gather_blocks(buf, blocks, rank: int, record_bytes: int, group=None) -> None:
    """All-gather of the row blocks of ``buf`` (a uint8 tensor of S records,
    device or host) over ``group``: afterwards every rank's ``buf`` holds every
    rank's block.  Blocks are padded to the largest for the gather."""
    import torch
    import torch.distributed as dist
    world = len(blocks)
    rb = record_bytes
    per = max(r1 - r0 for r0, r1 in blocks) * rb
    r0, r1 = blocks[rank]
    send = torch.zeros(per, dtype=torch.uint8, device=buf.device)
    send[:(r1 - r0) * rb].copy_(buf[r0 * rb:r1 * rb])
    if buf.is_cuda and dist.get_backend(group) == "nccl":
        out = torch.empty(world * per, dtype=torch.uint8, device=buf.device)
        dist.all_gather_into_tensor(out, send, group=group)
        parts = [out[q * per:(q + 1) * per] for q in range(world)]
    else:
        parts = [torch.empty(per, dtype=torch.uint8, device=send.device) for _ in range(world)]
        dist.all_gather(parts, send, group=group)
    for q, (q0, q1) in enumerate(blocks):
        if q != rank:
            buf[q0 * rb:q1 * rb].copy_(parts[q][:(q1 - q0) * rb])


class GroupExchange:
    """One shard per process over a ``torch.distributed`` group (rank r holds
    block r).  NCCL: device buffers gathered in place on the shard's stream.
    Other backends: the buffer goes through host memory (the shard's stream is
    synchronised first)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.group = group
        self.nccl = dist.get_backend(group) == "nccl"

    def __call__(self, ptrs, shards):
        (ptr,), (s,) = ptrs, shards
        rb = s.record_bytes
        dev_buf = _device_bytes(ptr, s.S * rb, s.device_index)
        if self.nccl:
            gather_blocks(dev_buf, s.blocks, s.rank, rb, self.group)
            return
        s.stream.synchronize()
        host = dev_buf.cpu()
        gather_blocks(host, s.blocks, s.rank, rb, self.group)
        dev_buf.copy_(host.to(dev_buf.device))
        s.stream.synchronize()
