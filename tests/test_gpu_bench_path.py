"""GPU parity of the benchmark's exact path against the FP64 oracle.

The benchmark times the paper-scale suspension (S = 512 dumbbells, N = 1024
spheres, density 0.002, lambda = 0.2, RPY, FP32 pair math with FP64 state,
seed 0) on the cooperative path, whose spring force and self term are FP32 and
whose critical-path Heun update runs on a double-single copy of the positions.
These tests run that configuration, at the split the autotuner picks (4
dumbbells per CTA) and at 8 and 16, and compare element by element with the
oracle's Heun integration (Sec. IV, Eqs. (3), (4)):

* positions after 1000 Heun steps within 1e-4 ell;
* the stroke-averaged centres (Eqs. (6b), (7b)) of the first two periods
  within 1e-4 ell of the oracle's period averages.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu

S_BENCH = 512
STEPS = 1000          # one stroke period (T = 1, dt = 1e-3)


@functools.lru_cache(maxsize=None)
def _oracle_two_periods():
    s = inputs.paper_scale(S_BENCH, seed=0, mobility="rpy")
    x1 = oracle.heun(s.x0, 0, STEPS, dt=s.dt, mobility=oracle.RPY, **s.phys())
    _, avg = oracle.heun_period_avg(s.x0, 0, STEPS, 2, dt=s.dt, mobility=oracle.RPY, **s.phys())
    return s, x1, avg


@pytest.mark.slow
@pytest.mark.parametrize("T", [4, 8, 16])
def test_benchmark_path_follows_oracle_1000_steps(T):
    s, x_ref, _ = _oracle_two_periods()
    with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
        h.set_path("coop")
        h.set_chunks(T)
        assert h.get_launch()["bt"] == T
        h.step(STEPS)
        x = h.positions()
        assert h.get_time()[0] == STEPS
    err = np.abs(x - x_ref).max()
    assert err <= 1e-4 * s.ell, err


@pytest.mark.slow
def test_benchmark_path_period_averages_follow_oracle():
    s, _, avg_ref = _oracle_two_periods()
    with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
        h.set_path("coop")
        h.set_chunks(4)
        h.enable_period_average(STEPS, max_periods=2)
        h.step(2 * STEPS)
        assert h.period_count() == 2
        got = h.period_averages(0, 2)
    assert got.shape == avg_ref.shape
    err = np.abs(got - avg_ref).max()
    assert err <= 1e-4 * s.ell, err
