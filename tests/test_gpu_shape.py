"""GPU parity of the shape-driven dynamics (Appendix A.2).

* Trajectories of dbs_set_dynamics(SHAPE, n) follow oracle.sd_heun with the
  same number n of constraint iterations (FP64 1e-10 ell, FP32C 1e-4 ell),
  Oseen and RPY, n = 1, 2, 3.
* Lengths stay on L(t); an isolated dumbbell neither moves nor turns.
* dbs_velocities in this mode reports H F for the constraint forces.
* Stroke averages accumulate as in the spring model (trapezoid rule).
* The mode refuses the cluster path, noise and external forces (DBS_E_STATE),
  and switching back to the spring continues the run (the cooperative path:
  test_gpu_shape_coop.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}


def _kw(s):
    kw = s.phys()
    kw.pop("k0")
    return kw


def _handle(s, precision="fp32c"):
    return dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                          mobility=s.mobility, precision=precision, lam=s.lam, phi=s.phi)


@pytest.mark.parametrize("mob,iters,precision,tol", [("oseen", 1, "fp64", 1e-10), ("oseen", 2, "fp64", 1e-10),
                                                     ("rpy", 3, "fp64", 1e-10), ("rpy", 2, "fp32c", 1e-4),
                                                     ("oseen", 3, "fp32c", 1e-4)])
def test_shape_trajectory_matches_oracle(mob, iters, precision, tol):
    s = inputs.make_suspension(12, seed=8, side=7.0, mobility=mob)
    nsteps = 300
    ref = oracle.sd_heun(s.x0, 0, nsteps, iters, dt=s.dt, mobility=MOB[mob], **_kw(s))
    with _handle(s, precision) as h:
        h.set_dynamics("shape", iters)
        h.step(nsteps)
        x = h.positions()
        assert h.get_time()[0] == nsteps
    assert np.abs(x - ref).max() <= tol * s.ell
    t = nsteps * s.dt
    L = s.ell + s.lam * np.sin(s.omega * t + s.phi)
    np.testing.assert_allclose(np.linalg.norm(x[1::2] - x[0::2], axis=1), L, rtol=1e-12)


def test_isolated_shape_dumbbell_stays_put():
    s = inputs.make_suspension(1, seed=3, side=8.0, mobility="oseen")
    with _handle(s, "fp64") as h:
        h.set_dynamics("shape", 1)
        h.step(500)
        x = h.positions()
    np.testing.assert_allclose(0.5 * (x[0] + x[1]), 0.5 * (s.x0[0] + s.x0[1]), atol=1e-12 * s.ell)
    e0 = (s.x0[1] - s.x0[0]) / np.linalg.norm(s.x0[1] - s.x0[0])
    e1 = (x[1] - x[0]) / np.linalg.norm(x[1] - x[0])
    np.testing.assert_allclose(e1, e0, atol=1e-12)


def test_shape_velocities_are_the_constraint_mobility_product():
    s = inputs.make_suspension(10, seed=9, side=7.0, mobility="rpy")
    with _handle(s, "fp64") as h:
        h.set_dynamics("shape", 2)
        h.step(20)
        x = h.positions()
        v = h.velocities()
    t = 20 * s.dt
    _, _, f = oracle.sd_rates(x, t, 2, mobility=oracle.RPY, **_kw(s))
    e = x[1::2] - x[0::2]
    n = e / np.linalg.norm(e, axis=1)[:, None]
    F = np.empty_like(x)
    F[0::2] = f[:, None] * n
    F[1::2] = -f[:, None] * n
    ref = oracle.mobility_apply(x, F, s.a, s.mu, oracle.RPY)
    assert np.abs(v - ref).max() <= 1e-12 * np.abs(ref).max()


def test_shape_stroke_averages():
    s = inputs.make_suspension(6, seed=10, side=7.0, mobility="oseen")
    m, periods = 40, 2
    s.dt = 1.0 / m
    x = s.x0.copy()
    Rbar = np.zeros((periods, 6, 3))
    for k in range(periods):
        acc = 0.5 * 0.5 * (x[0::2] + x[1::2])
        for j in range(1, m + 1):
            x = oracle.sd_heun(x, k * m + j - 1, 1, 2, dt=s.dt, mobility=oracle.OSEEN, **_kw(s))
            w = 0.5 if j == m else 1.0
            acc = acc + w * 0.5 * (x[0::2] + x[1::2])
        Rbar[k] = acc / m
    with _handle(s, "fp64") as h:
        h.set_dynamics("shape", 2)
        h.enable_period_average(m, max_periods=periods)
        h.step(m * periods)
        got = h.period_averages(0, periods)
    assert np.abs(got - Rbar).max() <= 1e-10 * s.ell


def test_shape_mode_restrictions_and_return_to_spring():
    s = inputs.make_suspension(16, seed=11, side=8.0)
    with _handle(s) as h:
        h.set_dynamics("shape", 2)
        for call in (lambda: h.set_path("cluster"),
                     lambda: h.set_noise(1e-3, 1), lambda: h.set_external_force(np.ones((32, 3)))):
            with pytest.raises(dbs.DbsError) as ei:
                call()
            assert ei.value.status == dbs.E_STATE
    with _handle(s) as h:
        h.set_dynamics("shape", 2)
        with pytest.raises(dbs.DbsError):
            dbs.Ensemble([h])            # ensembles run the spring model only
    with _handle(s) as h:
        with pytest.raises(dbs.DbsError):
            h.set_dynamics("shape", 0)
        h.set_dynamics("shape", 2)
        h.step(50)
        x_mid, n_mid = h.get_state()
        h.set_dynamics("spring")
        h.step(50)
        x = h.positions()
    ref = oracle.heun(x_mid, n_mid, 50, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    assert np.abs(x - ref).max() <= 1e-4 * s.ell
