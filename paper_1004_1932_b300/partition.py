"""Independent systems spread over ranks (one GPU each), with no collective on
the data path.

Every rank computes the same assignment from the same inputs and runs only its
own share: an ensemble of suspensions is split by longest-processing-time-first
(LPT) list scheduling on the pair work S^2 x steps of each member (the pair sum
of Eq. (3b) costs N(N - 1) terms per evaluation); a request stream is routed on
arrival to the rank with the least work assigned so far.  A system's result
does not depend on the rank it lands on: each rank runs the single-GPU path.
"""
from __future__ import annotations

import heapq


def pair_work(S: int, steps: int) -> float:
    """Pair terms of `steps` Heun steps of S dumbbells (two evaluations per step)."""
    N = 2 * S
    return 2.0 * N * (N - 1) * steps


def lpt(costs, nranks: int) -> list[int]:
    """Rank of every item: items in decreasing cost (ties: lower index first), each
    to the rank with the least load so far (ties: lower rank).  Deterministic."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(nranks)]
    out = [0] * len(costs)
    for i in order:
        load, r = heapq.heappop(heap)
        out[i] = r
        heapq.heappush(heap, (load + costs[i], r))
    return out


def loads(costs, assign, nranks: int) -> list[float]:
    tot = [0.0] * nranks
    for c, r in zip(costs, assign):
        tot[r] += c
    return tot


def lpt_bound(optimum: float, nranks: int) -> float:
    """Graham's bound on the LPT makespan: (4/3 - 1/(3 m)) times the optimum."""
    return (4.0 / 3.0 - 1.0 / (3.0 * nranks)) * optimum


def list_bound(costs, nranks: int) -> float:
    """Bound of any greedy list schedule: total / m + (1 - 1/m) max item."""
    return sum(costs) / nranks + (1.0 - 1.0 / nranks) * max(costs, default=0.0)


def route_stream(costs, nranks: int) -> list[int]:
    """Online routing of requests in arrival order: each to the rank with the least
    work assigned so far (ties: lower rank)."""
    tot = [0.0] * nranks
    out = []
    for c in costs:
        r = min(range(nranks), key=lambda q: (tot[q], q))
        out.append(r)
        tot[r] += c
    return out
