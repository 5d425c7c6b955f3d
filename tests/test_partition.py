"""Independent systems over ranks (host logic, no GPU).

* LPT: every system on exactly one rank; the makespan within Graham's bound
  (4/3 - 1/(3m)) of the brute-force optimum on small instances, and on the
  benchmark ensemble's costs within the list-scheduling bound
  total / m + (1 - 1/m) largest, and no worse than a round-robin split.
* The assignment is a pure function of the inputs: on CPU ranks (gloo, world
  size 2) each rank computes it alone, and all ranks agree; their shares
  cover every system once.
* Online routing of a request stream keeps the ranks' assigned work within one
  request of each other.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1004_1932_b300 import inputs, partition


def _ensemble_costs(count=256, steps=1000):
    return [partition.pair_work(int(S), steps) for S in inputs.ensemble_sizes(count)]


def _optimum(costs, nranks):
    """Brute-force optimal makespan (small instances)."""
    import itertools
    best = float("inf")
    for a in itertools.product(range(nranks), repeat=len(costs)):
        best = min(best, max(partition.loads(costs, a, nranks)))
    return best


@pytest.mark.parametrize("nranks", [2, 3, 4])
def test_lpt_is_within_graham_bound_of_the_optimum(nranks):
    rng = np.random.default_rng(nranks)
    cases = [[5.0] * 7, [3.0, 3.0, 2.0, 2.0, 2.0], list(rng.uniform(1, 100, size=8)),
             [float(S) ** 2 for S in inputs.ensemble_sizes(9, seed=nranks)]]
    for costs in cases:
        a = partition.lpt(costs, nranks)
        ms = max(partition.loads(costs, a, nranks))
        assert ms <= partition.lpt_bound(_optimum(costs, nranks), nranks) * (1 + 1e-12)


@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 8])
def test_lpt_on_the_benchmark_ensemble(nranks):
    costs = _ensemble_costs()
    a = partition.lpt(costs, nranks)
    assert len(a) == len(costs) and all(0 <= r < nranks for r in a)
    ld = partition.loads(costs, a, nranks)
    assert max(ld) <= partition.list_bound(costs, nranks) * (1 + 1e-12)
    rr = [i % nranks for i in range(len(costs))]
    assert max(ld) <= max(partition.loads(costs, rr, nranks)) * (1 + 1e-12)


def test_lpt_small_cases():
    assert max(partition.loads([3, 3, 2, 2, 2], partition.lpt([3, 3, 2, 2, 2], 2), 2)) == 7
    assert partition.lpt([], 3) == []
    with pytest.raises(ValueError):
        partition.lpt([1.0], 0)


def test_route_stream_balances_work():
    trace = inputs.request_trace(500)
    costs = [partition.pair_work(S, n) for _, S, n, _ in trace]
    for nranks in (2, 4):
        r = partition.route_stream(costs, nranks)
        ld = partition.loads(costs, r, nranks)
        assert max(ld) - min(ld) <= max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = _ensemble_costs()
    a = partition.lpt(costs, world)
    t = torch.tensor(a, dtype=torch.int64)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out[rank] = ([p.tolist() for p in parts], [i for i, r in enumerate(a) if r == rank])
    dist.destroy_process_group()


def test_ranks_agree_on_the_assignment():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    gathered0, mine0 = res[0]
    gathered1, mine1 = res[1]
    assert gathered0[0] == gathered0[1] == gathered1[0] == gathered1[1]
    assert sorted(mine0 + mine1) == list(range(256)) and not set(mine0) & set(mine1)
