"""GPU parity of the additive-noise dynamics (closing remarks of Sec. IV).

The device draws the same Philox4x32-10 / Box-Muller normals as the oracle
(counter = step and sphere, key = seed), so noisy trajectories are compared
element by element: every stepping path against oracle.heun(kT, seed) within
the trajectory tolerance (FP32C 1e-4 ell, FP64 1e-10 ell), kT = 0 against the
deterministic run, and free spheres against the Stokes-Einstein variance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}


def _handle(s, precision="fp32c", **kw):
    return dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                          mobility=s.mobility, precision=precision, lam=s.lam, phi=s.phi, **kw)


def _kT_for(s, frac=1.0):
    # noise displacement per step ~ frac x the deterministic one (dt x stroke speed)
    v = s.lam.mean() * s.ell * s.omega
    step = v * s.dt
    return (frac * step) ** 2 * 6 * math.pi * s.mu * s.a / (2 * s.dt)


@pytest.mark.parametrize("path,precision,tol", [("grid", "fp32c", 1e-4), ("grid", "fp64", 1e-10),
                                                ("cluster", "fp32c", 1e-4), ("coop", "fp32c", 1e-4)])
def test_noisy_trajectory_matches_oracle(path, precision, tol):
    s = inputs.make_suspension(24, seed=5, side=9.0, mobility="rpy")
    kT, seed, nsteps = _kT_for(s), 0x1234_5678_9ABC, 600
    ref = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[s.mobility], kT=kT, seed=seed, **s.phys())
    det = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    assert np.abs(ref - det).max() > 100 * tol * s.ell   # the noise is visible at this tolerance
    with _handle(s, precision) as h:
        if path != "grid":
            h.set_path(path)
        h.set_noise(kT, seed)
        h.step(nsteps)
        x = h.positions()
    assert np.abs(x - ref).max() <= tol * s.ell


@pytest.mark.parametrize("S", [12, 300, 1000])
def test_cooperative_noise_every_split_matches_grid_path(S):
    # the noise instantiation of the cooperative kernel at 16, 4 and 8 dumbbells
    # per CTA: the same increments as the grid path, trajectories within 1e-6 ell
    s = inputs.make_suspension(S, seed=40 + S, density=0.002, mobility="rpy") if S > 40 \
        else inputs.make_suspension(S, seed=40, side=8.0, mobility="rpy")
    kT, seed, nsteps = _kT_for(s), 777, 200
    with _handle(s, "fp32c") as hg:
        hg.set_noise(kT, seed)
        hg.step(nsteps)
        xg = hg.positions()
    with _handle(s, "fp32c") as hc:
        hc.set_path("coop")
        hc.set_noise(kT, seed)
        hc.step(nsteps)
        xc = hc.positions()
        T = hc.get_launch()["bt"]
    assert T == {12: 16, 300: 4, 1000: 8}[S]
    assert np.abs(xc - xg).max() <= 1e-6 * s.ell


def test_zero_temperature_is_the_deterministic_path():
    s = inputs.make_suspension(24, seed=6, side=9.0)
    with _handle(s) as h:
        h.step(50)
        a = h.positions()
    with _handle(s) as h:
        h.set_noise(0.0, 99)
        h.step(50)
        b = h.positions()
    assert np.array_equal(a, b)


def test_noise_continues_across_launches_and_paths():
    s = inputs.make_suspension(24, seed=7, side=9.0)
    kT, seed = _kT_for(s), 42
    ref = oracle.heun(s.x0, 0, 1300, dt=s.dt, mobility=MOB[s.mobility], kT=kT, seed=seed, **s.phys())
    with _handle(s) as h:
        h.set_noise(kT, seed)
        h.step(100)                  # grid
        h.set_path("coop")
        h.step(1100)                 # cooperative: one full launch and a partial one
        h.set_path("cluster")
        h.step(100)
        x = h.positions()
    assert np.abs(x - ref).max() <= 1e-4 * s.ell


def test_noisy_period_averages_agree_across_paths():
    # the stroke averages of a noisy run: grid path (FP64 sums in the epilogue,
    # its noisy trajectory checked against the oracle above) against the
    # cooperative one (double-single sums of the noisy positions within a
    # launch), with a period that straddles two launches
    s = inputs.make_suspension(24, seed=9, side=9.0, mobility="rpy")
    kT, seed, m, periods = _kT_for(s), 77, 500, 3
    s.dt = 1.0 / m
    out = []
    for path in ("grid", "coop"):
        with _handle(s) as h:
            h.set_path(path)
            h.set_noise(kT, seed)
            h.enable_period_average(m, max_periods=periods)
            h.step(700)
            h.step(800)
            out.append(h.period_averages(0, periods))
    assert np.abs(out[1] - out[0]).max() <= 1e-6 * s.ell


def test_free_spheres_diffuse_with_stokes_einstein_variance():
    s, F = inputs.colloids(2000, mobility="oseen")
    kT, nsteps = 1e-3, 200
    with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
        h.set_noise(kT, 3)
        h.step(nsteps)
        x = h.positions()
    d2 = (x - s.x0) ** 2
    D0 = kT / (6 * math.pi * s.mu * s.a)
    expected = 2 * D0 * nsteps * s.dt
    assert abs(d2.mean() / expected - 1.0) < 5 * math.sqrt(2.0 / d2.size)


def test_noise_arguments_validated():
    s = inputs.make_suspension(4, seed=1, side=8.0)
    with _handle(s) as h:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(dbs.DbsError) as ei:
                h.set_noise(bad, 0)
            assert ei.value.status == dbs.E_ARG
