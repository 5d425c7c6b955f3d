"""Serving engine: continuous batching under a device-memory budget.

* A request gives the same final positions alone and in a mix with other
  requests that arrive before, during and after it (within the trajectory
  tolerance 1e-4 ell), and the same as a plain suspension handle stepped alone.
* With a budget that holds one request at a time, requests queue and all
  complete with the same results.
* Queued and running requests can be cancelled; their memory is released.
"""
import numpy as np
import pytest

from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu


def _susp(S, seed, mob="rpy", lam=0.2):
    return inputs.make_suspension(S, seed=seed, density=0.002, mobility=mob, lam=lam)


def _drain(eng, max_ticks=10000):
    for _ in range(max_ticks):
        a, q = eng.tick()
        if a == 0 and q == 0:
            return
    raise AssertionError("engine did not drain")


def _alone(s, steps):
    with dbs.Suspension.from_inputs(s) as h:
        h.step(steps)
        return h.positions()


def test_request_alone_and_in_mix():
    A = _susp(200, 1)
    ref = _alone(A, 700)
    with dbs.Engine(block_steps=128) as eng:
        ra = eng.submit_inputs(A, 700)
        _drain(eng)
        st, x_alone, lat = eng.poll(ra)
        assert st == dbs.REQ_DONE and lat > 0
    with dbs.Engine(block_steps=128) as eng:
        early = [eng.submit_inputs(_susp(S, 10 + S, mob), n)
                 for S, n, mob in ((16, 300, "oseen"), (900, 500, "rpy"), (2500, 200, "rpy"))]
        eng.tick()
        eng.tick()
        ra = eng.submit_inputs(A, 700)                    # arrives while others run
        eng.tick()
        late = [eng.submit_inputs(_susp(64, 77), 1000)]
        _drain(eng)
        st, x_mix, _ = eng.poll(ra)
        assert st == dbs.REQ_DONE
        for rid in early + late:
            assert eng.poll(rid)[0] == dbs.REQ_DONE
    assert np.abs(x_alone - ref).max() <= 1e-4 * A.ell
    assert np.abs(x_mix - ref).max() <= 1e-4 * A.ell


def test_budget_admits_one_at_a_time():
    systems = [_susp(S, 30 + S) for S in (100, 120, 90)]
    budget = max(dbs.request_bytes(s.S) for s in systems) + 1024
    refs = [_alone(s, 300) for s in systems]
    with dbs.Engine(hbm_budget_bytes=budget, block_steps=100) as eng:
        ids = [eng.submit_inputs(s, 300) for s in systems]
        a, q = eng.tick()
        assert a == 1 and q == 2
        _drain(eng)
        for rid, ref, s in zip(ids, refs, systems):
            st, x, _ = eng.poll(rid)
            assert st == dbs.REQ_DONE
            assert np.abs(x - ref).max() <= 1e-4 * s.ell


def test_cancel_queued_and_running():
    with dbs.Engine(max_active=1, block_steps=50) as eng:
        r1 = eng.submit_inputs(_susp(40, 5), 10000)
        r2 = eng.submit_inputs(_susp(40, 6), 10000)
        eng.tick()
        assert eng.poll(r1)[0] == dbs.REQ_RUNNING and eng.poll(r2)[0] == dbs.REQ_PENDING
        eng.cancel(r2)
        eng.cancel(r1)
        assert eng.poll(r1)[0] == dbs.REQ_CANCELLED and eng.poll(r2)[0] == dbs.REQ_CANCELLED
        a, q = eng.tick()
        assert a == 0 and q == 0
