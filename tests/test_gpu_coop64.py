"""GPU parity of the cooperative path in FP64 (all-FP64 plain method, Sec. IV).

The FP64 cooperative kernel runs up to 1024 Heun steps per launch over one CTA
per 1, 2 or 4 dumbbells, exchanging FP64 records whose lowest significand bits
carry the evaluation's parity bit.  The checks:

* trajectories follow the FP64 oracle within the FP64 trajectory tolerance of
  the grid path (1e-10 ell), from one dumbbell to 592 (one CTA per SM at 4
  dumbbells each), under both mobilities, including the S = 16 Oseen system
  (side 8, seed 0, 1000 steps) that the benchmark times;
* they agree with the grid path's FP64 run to 1e-11 ell, and the velocities the
  grid path computes afterwards from the records the cooperative launch left
  behind agree with the grid run's;
* every split (1, 2, 4 dumbbells per CTA) gives the same trajectory;
* runs longer than one launch continue the clock and the step counter, stroke
  averages match the oracle's, and a tag counter about to wrap changes nothing;
* an RPY overlap, more than 592 dumbbells and additive noise are refused or
  reported, and a launch in a shape the kernel was not built for is refused;
  the handle stays usable.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}
TOL = 1e-10      # FP64 trajectory tolerance against the oracle (ell units), as the grid path


def _handle(s, precision="fp64"):
    return dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                          mobility=s.mobility, precision=precision, lam=s.lam, phi=s.phi)


def _susp(S, mob, seed):
    if S > 40:
        return inputs.make_suspension(S, seed=seed, density=0.002, mobility=mob)
    return inputs.make_suspension(S, seed=seed, side=8.0, mobility=mob)


@pytest.mark.parametrize("S,mob,nsteps", [(1, "rpy", 1000), (2, "oseen", 1000), (16, "rpy", 1000),
                                          (31, "oseen", 500), (149, "rpy", 200), (300, "oseen", 100),
                                          (592, "rpy", 20)])
def test_coop64_follows_oracle(S, mob, nsteps):
    s = _susp(S, mob, S + 3)
    ref = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[mob], **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        assert h.get_path()[0] == "coop"
        h.step(nsteps)
        x = h.positions()
        assert h.get_time()[0] == nsteps
    assert np.abs(x - ref).max() <= TOL * s.ell


def test_coop64_small_system_of_the_benchmark():
    s = inputs.small_fp64_oseen(seed=0)
    ref = oracle.heun(s.x0, 0, 1000, dt=s.dt, mobility=oracle.OSEEN, **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        assert h.get_launch()["bt"] == 1 and h.get_launch()["grid"] == 16
        h.step(1000)
        x = h.positions()
        n, t = h.get_time()
    assert n == 1000 and t == pytest.approx(1.0)
    assert np.abs(x - ref).max() <= TOL * s.ell


@pytest.mark.parametrize("S,mob", [(16, "oseen"), (100, "rpy"), (300, "rpy")])
def test_coop64_matches_grid_path(S, mob):
    s = _susp(S, mob, 7)
    nsteps = 300
    with _handle(s) as hg:
        hg.step(nsteps)
        xg = hg.positions()
        vg = hg.velocities()
    with _handle(s) as hc:
        hc.set_path("coop")
        hc.step(nsteps)
        xc = hc.positions()
        vc = hc.velocities()        # grid-path evaluation of the records the launch left
    assert np.abs(xc - xg).max() <= 1e-11 * s.ell
    assert np.abs(vc - vg).max() <= 1e-9 * np.abs(vg).max()


@pytest.mark.parametrize("chunks", [1, 2, 4])
def test_coop64_splits_agree(chunks):
    s = _susp(100, "rpy", 9)
    nsteps = 200
    with _handle(s) as h:
        h.step(nsteps)
        ref = h.positions()
    with _handle(s) as h:
        h.set_path("coop")
        h.set_chunks(chunks)
        assert h.get_launch()["bt"] == chunks
        h.step(nsteps)
        x = h.positions()
    assert np.abs(x - ref).max() <= 1e-11 * s.ell


def test_coop64_long_run_crosses_launches():
    s = inputs.make_suspension(24, seed=4, side=8.0)
    nsteps = 2500                     # three launches
    with _handle(s) as hg:
        hg.step(nsteps)
        xg = hg.positions()
        tg = hg.get_time()
    with _handle(s) as hc:
        hc.step(37)                   # start on the grid path
        hc.set_path("coop")
        hc.step(nsteps - 37)
        xc = hc.positions()
        tc = hc.get_time()
    assert tc[0] == tg[0] == nsteps
    assert tc[1] == pytest.approx(tg[1], rel=1e-15)
    assert np.abs(xc - xg).max() <= 1e-10 * s.ell


def test_coop64_period_averages_match_oracle():
    s = inputs.make_suspension(12, seed=6, side=8.0)
    m, periods = 100, 3
    s.dt = 1.0 / m
    _, ref = oracle.heun_period_avg(s.x0, 0, m, periods, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        h.enable_period_average(m, max_periods=periods)
        h.step(m * periods)
        assert h.period_count() == periods
        got = h.period_averages(0, periods)
    assert np.abs(got - ref).max() <= TOL * s.ell


def test_coop64_tag_wraparound():
    s = _susp(64, "rpy", 12)
    with _handle(s) as h:
        h.set_path("coop")
        h.step(1500)
        ref = h.positions()
    with _handle(s) as h:
        h.set_path("coop")
        h.set_flow_tag(0xFFFFFFFF - 300)
        h.step(1500)
        x = h.positions()
    assert np.array_equal(x, ref)


def test_coop64_reports_overlap():
    x0 = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.05, 0, 0], [2.05, 0, 0]])
    with dbs.Suspension(x0, a=0.05, mu=1.0, k0=1.0, ell=1.0, omega=2 * math.pi, dt=1e-3,
                        mobility="rpy", precision="fp64") as h:
        h.set_path("coop")
        h.step(1)
        with pytest.raises(dbs.DbsError) as ei:
            h.sync()
        assert ei.value.status == dbs.E_OVERLAP


def test_coop64_refuses_what_it_cannot_hold():
    s = _susp(593, "oseen", 2)        # more than 4 dumbbells per CTA on 148 SMs
    with _handle(s) as h:
        with pytest.raises(dbs.DbsError) as ei:
            h.set_path("coop")
        assert ei.value.status == dbs.E_ARG
        assert h.get_path()[0] == "grid"
        h.step(2)
        assert np.isfinite(h.positions()).all()
    s = _susp(32, "oseen", 2)
    with _handle(s) as h:             # noise, then the path
        h.set_noise(1e-3, seed=1)
        with pytest.raises(dbs.DbsError):
            h.set_path("coop")
        assert h.get_path()[0] == "grid"
        h.step(2)
        assert np.isfinite(h.positions()).all()
    with _handle(s) as h:             # the path, then noise
        h.set_path("coop")
        with pytest.raises(dbs.DbsError) as ei:
            h.set_noise(1e-3, seed=1)
        assert ei.value.status == dbs.E_STATE
        h.step(2)
        assert np.isfinite(h.positions()).all()


def test_coop64_kernel_refuses_a_launch_shape_it_was_not_built_for():
    lib = dbs.load()
    s = _susp(16, "oseen", 3)
    h = _handle(s)
    h.set_path("coop")
    assert lib.dbs_test_flow_misshape(h._h) == dbs.E_CUDA
    assert "shape" in lib.dbs_last_error(h._h).decode()
    h.close()
    with _handle(s) as h:
        h.set_path("coop")
        h.step(4)
        assert np.isfinite(h.positions()).all()
