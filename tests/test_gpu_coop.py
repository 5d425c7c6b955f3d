"""GPU parity of the cooperative path (one launch advances up to 1024 steps).

* A suspension stepped on the cooperative path follows the FP64 oracle within
  the trajectory tolerance (1e-4 ell after 1000 Heun steps).
* It ends where the grid path ends, to well inside the oracle tolerance (its
  spring force and Heun average are FP32, the grid path's FP64; both keep FP64
  positions).
* Every split request (dumbbells per CTA, 1 .. 16; raised where the grid
  would not fit the SMs) gives the same trajectory.
* Runs longer than one launch (1024 steps) and than the clock ring (4096 steps)
  continue the clock and the step counter; stroke averages accumulated on the
  cooperative path match the oracle's.
* The bounded wait reports DBS_E_TIMEOUT when the word it polls never arrives,
  and the device stays usable afterwards.
* Sizes the path cannot hold are refused with DBS_E_ARG and leave the handle
  usable on the grid path (the FP64 form of the path: test_gpu_coop64.py).
* The kernel refuses a launch in a shape other than the one it was told
  (DBS_E_CUDA), before touching state or exchange buffers; the device and the
  path stay usable.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}


def _handle(s, precision="fp32c"):
    return dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                          mobility=s.mobility, precision=precision, lam=s.lam, phi=s.phi)


@pytest.mark.parametrize("S,mob", [(1, "rpy"), (2, "oseen"), (16, "oseen"), (16, "rpy"), (31, "rpy"),
                                   (33, "oseen"), (300, "rpy"), (513, "oseen")])
def test_coop_path_follows_oracle(S, mob):
    s = inputs.make_suspension(S, seed=S + 11, density=0.002, mobility=mob) if S > 40 \
        else inputs.make_suspension(S, seed=1, side=8.0, mobility=mob)
    nsteps = 1000
    ref = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[mob], **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        assert h.get_path()[0] == "coop"
        h.step(nsteps)
        x = h.positions()
        assert h.get_time()[0] == nsteps
    assert np.abs(x - ref).max() <= 1e-4 * s.ell


@pytest.mark.parametrize("S", [64, 256, 512, 1024, 2048, 2300, 4096])   # 1 .. 32 dumbbells per CTA
def test_coop_path_matches_grid_path(S):
    s = inputs.paper_scale(S, seed=5)
    nsteps = 300
    with _handle(s) as hg:
        hg.step(nsteps)
        xg = hg.positions()
    with _handle(s) as hc:
        hc.set_path("coop")
        hc.step(nsteps)
        xc = hc.positions()
    assert np.abs(xc - xg).max() <= 1e-6 * s.ell


def test_coop_long_run_crosses_launches_and_clock_ring():
    s = inputs.make_suspension(24, seed=4, side=8.0)
    nsteps = 5000                     # > 4 launches of 1024 steps and > the 4096-entry ring
    with _handle(s) as hg:
        hg.step(nsteps)
        xg = hg.positions()
        tg = hg.get_time()
    with _handle(s) as hc:
        hc.step(37)                   # start on the grid path mid-launch
        hc.set_path("coop")
        hc.step(nsteps - 37)
        xc = hc.positions()
        tc = hc.get_time()
    assert tc[0] == tg[0] == nsteps
    assert tc[1] == pytest.approx(tg[1], rel=1e-15)
    assert np.abs(xc - xg).max() <= 1e-5 * s.ell


@pytest.mark.parametrize("S,chunks", [(100, 1), (100, 2), (100, 4), (100, 16), (700, 3), (700, 8),
                                      (700, 16), (2048, 5)])
def test_coop_chunk_counts_agree(S, chunks):
    s = inputs.paper_scale(S, seed=9)
    nsteps = 200
    with _handle(s) as h:
        h.set_path("coop")
        h.step(nsteps)
        ref = h.positions()
    with _handle(s) as h:
        h.set_path("coop")
        h.set_chunks(chunks)
        h.step(nsteps)
        x = h.positions()
    assert np.abs(x - ref).max() <= 1e-6 * s.ell


def test_coop_handles_of_one_split_coexist():
    # two suspensions on the same kernel instantiation (16 dumbbells per CTA) with
    # different record arrays: setting up the smaller one second must not stop the
    # larger one from launching
    big = inputs.paper_scale(2000, seed=31)
    small = inputs.paper_scale(1500, seed=32)
    with _handle(big) as hb, _handle(small) as hs:
        hb.set_path("coop")
        hs.set_path("coop")
        assert hb.get_launch()["bt"] == hs.get_launch()["bt"] == 16
        hb.step(20)
        hs.step(20)
        assert np.isfinite(hb.positions()).all() and np.isfinite(hs.positions()).all()


def test_coop_period_averages_match_oracle():
    s = inputs.make_suspension(12, seed=6, side=8.0)
    m, periods = 100, 3
    s.dt = 1.0 / m                    # one stroke period (omega = 2 pi) in m steps
    _, ref = oracle.heun_period_avg(s.x0, 0, m, periods, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        h.enable_period_average(m, max_periods=periods)
        h.step(m * periods)
        assert h.period_count() == periods
        got = h.period_averages(0, periods)
    assert np.abs(got - ref).max() <= 1e-4 * s.ell


def test_coop_period_averages_across_launches_match_grid_path():
    # averaging enabled mid-run and launches that end mid-period: the cooperative
    # kernel carries the period sums between launches in the grid path's FP64 form
    s = inputs.make_suspension(40, seed=14, side=12.0, mobility="rpy")
    m, periods = 700, 3
    out = []
    for path in ("grid", "coop"):
        with _handle(s) as h:
            h.set_path(path)
            h.step(50)
            h.enable_period_average(m, max_periods=periods)
            for n in (37, 1500, 563):
                h.step(n)
            assert h.period_count() == periods
            out.append((h.period_averages(0, periods), h.positions()))
    (ag, xg), (ac, xc) = out
    assert np.abs(xc - xg).max() <= 1e-6 * s.ell
    assert np.abs(ac - ag).max() <= 1e-6 * s.ell


@pytest.mark.parametrize("tag", [0xFFFFFFFF - 300, 0xFFFFFFFF - 3000])
def test_coop_tag_wraparound(tag):
    # the first launch (first case) or the second (second case) would run past
    # 2^32 tags: the buffers are cleared and the tags restart, results unchanged
    s = inputs.paper_scale(64, seed=12)
    with _handle(s) as h:
        h.set_path("coop")
        h.step(2000)
        ref = h.positions()
    with _handle(s) as h:
        h.set_path("coop")
        h.set_flow_tag(tag)
        h.step(2000)
        x = h.positions()
    assert np.array_equal(x, ref)


def test_coop_refuses_what_it_cannot_hold():
    s = inputs.make_suspension(4097, seed=2, density=0.002)
    with _handle(s) as h:
        with pytest.raises(dbs.DbsError) as ei:
            h.set_path("coop")
        assert ei.value.status == dbs.E_ARG
        assert h.get_path()[0] == "grid"
        h.step(2)
        assert np.isfinite(h.positions()).all()


def test_bounded_wait_times_out_and_device_stays_usable():
    assert dbs.check_wait_timeout(50) == dbs.E_TIMEOUT
    s = inputs.make_suspension(16, seed=0, side=8.0)
    ref = oracle.heun(s.x0, 0, 20, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    with _handle(s) as h:
        h.set_path("coop")
        h.step(20)
        assert np.abs(h.positions() - ref).max() <= 1e-4 * s.ell


def test_cooperative_kernel_refuses_a_launch_shape_it_was_not_built_for():
    # the kernel is told it has one CTA more than it was launched with: every CTA
    # must refuse before touching state or exchange buffers, the host reports it
    lib = dbs.load()
    for S in (16, 512):
        s = inputs.paper_scale(S, seed=3)
        h = dbs.Suspension.from_inputs(s, precision="fp32c")
        h.set_path("coop")
        assert lib.dbs_test_flow_misshape(h._h) == dbs.E_CUDA
        assert "shape" in lib.dbs_last_error(h._h).decode()
        h.close()
    # the device stays usable, and so does the cooperative path
    s = inputs.paper_scale(512, seed=3)
    with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
        h.set_path("coop")
        h.step(4)
        assert np.isfinite(h.positions()).all()
