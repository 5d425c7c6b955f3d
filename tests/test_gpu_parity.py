"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerances (stated by the method's accuracy target):
  * velocities, FP32 pair math with compensated accumulation:
        max_i |v_i - v_i^ref| / max_i |v_i^ref| <= 1e-5
  * velocities, all-FP64 path: <= 1e-12
  * trajectories after 1000 Heun steps: max_i |x_i - x_i^ref| <= 1e-4 ell
  * stroke-averaged rates: 1e-5 (FP32C) / 1e-12 (FP64) relative to max |rate|
Inputs are the seeded generators of ``paper_1004_1932_b300.inputs``; expected
values come from ``oracle`` only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu

TOL_V = {"fp32c": 1e-5, "fp64": 1e-12}
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}


def _ref_velocities(s, x, t, mobility, Fext=None):
    return oracle.velocities(x, t, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, lam=s.lam,
                             phi=s.phi, mobility=MOB[mobility], Fext=Fext)


def _relerr(v, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    return np.abs(v - ref).max() / scale


def _jittered(s, seed, scale=0.05):
    """Initial positions pushed off the spring minima so that every force is non-zero."""
    return s.x0 + np.random.default_rng(1000 + seed).normal(scale=scale, size=s.x0.shape)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("mob", ["oseen", "rpy"])
@pytest.mark.parametrize("S", [1, 2, 16, 37, 129, 300, 1000, 3001])
def test_velocities_ragged_sizes(prec, mob, S):
    s = inputs.make_suspension(S, seed=S, density=0.002, mobility=mob)
    x = _jittered(s, S)
    with dbs.Suspension(x, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                        mobility=mob, precision=prec, lam=s.lam, phi=s.phi) as h:
        v = h.velocities()
        u = h.interaction()
    ref = _ref_velocities(s, x, 0.0, mob)
    assert _relerr(v, ref) <= TOL_V[prec]
    F = oracle.spring_forces(x, s.ell, s.lam, s.omega, s.phi, s.k0, 0.0)
    uref = oracle.interaction(x, F, s.a, s.mu, MOB[mob])
    if S > 1:
        # the interaction part alone, relative to its own scale (diagnostic)
        assert _relerr(u, uref) <= (1e-4 if prec == "fp32c" else 1e-11)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_mobility_apply_random_forces(prec):
    s = inputs.make_suspension(200, seed=5, density=0.002, mobility="rpy")
    F = np.random.default_rng(6).normal(size=(400, 3))
    with dbs.Suspension.from_inputs(s, precision=prec) as h:
        v = h.mobility_apply(F)
        x = h.positions()
    np.testing.assert_array_equal(x, s.x0)      # apply does not touch the state
    ref = oracle.mobility_apply(s.x0, F, s.a, s.mu, oracle.RPY)
    assert _relerr(v, ref) <= TOL_V[prec]


def test_external_force_two_sphere_drift():
    # one passive dumbbell at rest length, equal external force on both spheres
    x0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    F = np.array([[0.0, 0.3, 0.0], [0.0, 0.3, 0.0]])
    for prec in ("fp32c", "fp64"):
        with dbs.Suspension(x0, a=0.05, mu=1.0, k0=1.0, ell=1.0, omega=2 * math.pi, dt=1e-3,
                            mobility="oseen", precision=prec) as h:
            h.set_external_force(F)
            v = h.velocities()
        expect = 0.3 * (1 / (6 * math.pi * 0.05) + 1 / (8 * math.pi * 1.0))
        np.testing.assert_allclose(v[:, 1], expect, rtol=TOL_V[prec])
        np.testing.assert_allclose(v[:, [0, 2]], 0.0, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_trajectory_small_fp64_oseen_1000_steps(prec):
    """S=16 (N=32), side 8, Oseen, dt=1e-3, 1000 steps from seed 0."""
    s = inputs.small_fp64_oseen(seed=0)
    ref = oracle.heun(s.x0, 0, 1000, dt=s.dt, mobility=oracle.OSEEN, **s.phys())
    with dbs.Suspension.from_inputs(s, precision=prec) as h:
        h.step(1000)
        x = h.positions()
        n, t = h.get_time()
    assert n == 1000 and t == pytest.approx(1.0)
    err = np.abs(x - ref).max()
    assert err <= 1e-4 * s.ell
    if prec == "fp64":
        assert err <= 1e-10 * s.ell


@pytest.mark.slow
def test_trajectory_paper_scale_1000_steps():
    """S=512 (N=1024) at density 0.002, lambda=0.2, FP32C RPY: first 1000 steps."""
    s = inputs.paper_scale(512, seed=0, mobility="rpy")
    ref = oracle.heun(s.x0, 0, 1000, dt=s.dt, mobility=oracle.RPY, **s.phys())
    with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
        h.step(1000)
        x = h.positions()
    assert np.abs(x - ref).max() <= 1e-4 * s.ell


@pytest.mark.parametrize("S", [2048, 32768])
def test_large_system_sampled_rows(S):
    """Full-size single systems (N = 4096 .. 65536) in the launch configuration
    the benchmark uses: velocities of sampled targets against the oracle."""
    s = inputs.paper_scale(S, seed=1, mobility="rpy")
    x = _jittered(s, S)
    with dbs.Suspension(x, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                        mobility="rpy", precision="fp32c", lam=s.lam, phi=s.phi) as h:
        v = h.velocities()
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([[0, 1, 2 * S - 1], rng.integers(0, 2 * S, 61)]))
    F = oracle.spring_forces(x, s.ell, s.lam, s.omega, s.phi, s.k0, 0.0)
    ref = oracle.mobility_rows(x, F, rows, s.a, s.mu, oracle.RPY)
    assert np.abs(v[rows] - ref).max() / np.abs(ref).max() <= TOL_V["fp32c"]
    # momentum balance of internal forces: total force zero; no sphere velocity is lost
    assert np.isfinite(v).all()


def test_isolated_dumbbell_does_not_swim():
    x0 = inputs.spheres_at_rest(np.array([[0.5, -1.0, 2.0]]), np.array([[0.6, 0.0, 0.8]]), 1.0,
                                np.array([0.2]), np.array([0.3]))
    for prec in ("fp32c", "fp64"):
        with dbs.Suspension(x0, a=0.05, mu=1.0, k0=1.0, ell=1.0, omega=2 * math.pi, dt=1e-3,
                            mobility="rpy", precision=prec, lam=[0.2], phi=[0.3]) as h:
            v = h.velocities()
            np.testing.assert_array_equal(v[0], -v[1])   # centroid velocity exactly 0
            h.step(1000)
            x = h.positions()
        np.testing.assert_allclose(0.5 * (x[0] + x[1]), 0.5 * (x0[0] + x0[1]), atol=1e-12)


def test_period_average_matches_oracle():
    s = inputs.make_suspension(24, seed=4, side=10.0, mobility="rpy")
    m, nper = 100, 3
    dt = 1.0 / m
    _, Rbar_ref = oracle.heun_period_avg(s.x0, 0, m, nper, dt=dt, mobility=oracle.RPY, **s.phys())
    with dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=dt,
                        mobility="rpy", precision="fp32c", lam=s.lam, phi=s.phi) as h:
        h.enable_period_average(m, max_periods=8)
        h.step(m * nper + 7)
        assert h.period_count() == nper
        Rbar = h.period_averages()
    assert np.abs(Rbar - Rbar_ref).max() <= 1e-4 * s.ell


def test_checkpoint_restart_is_bit_exact():
    s = inputs.make_suspension(300, seed=9, density=0.002)
    with dbs.Suspension.from_inputs(s) as h:
        h.step(70)
        x70, n70 = h.get_state()
        h.step(45)
        x_a = h.positions()
        h.set_state(x70, n70)
        h.step(45)
        x_b = h.positions()
        assert h.get_time()[0] == 115
    np.testing.assert_array_equal(x_a, x_b)


def test_runs_are_deterministic():
    s = inputs.make_suspension(700, seed=2, density=0.002)
    xs = []
    for _ in range(2):
        with dbs.Suspension.from_inputs(s) as h:
            h.step(40)
            xs.append(h.positions())
    np.testing.assert_array_equal(xs[0], xs[1])


def test_overlap_is_reported():
    # two dumbbells whose spheres 1 and 2 are 0.05 apart (< 2a = 0.1) under RPY
    x0 = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.05, 0, 0], [2.05, 0, 0]])
    with dbs.Suspension(x0, a=0.05, mu=1.0, k0=1.0, ell=1.0, omega=2 * math.pi, dt=1e-3,
                        mobility="rpy") as h:
        h.step(1)
        with pytest.raises(dbs.DbsError) as ei:
            h.sync()
        assert ei.value.status == dbs.E_OVERLAP
        with pytest.raises(dbs.DbsError):      # sticky
            h.step(1)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_stroke_averaged_rates_and_steps(prec):
    s = inputs.paper_scale(512, seed=0)
    kw = dict(a=s.a, ell=s.ell, omega=s.omega)
    Rd_ref, Nd_ref = oracle.sa_rates(s.R0, s.N0, s.phi, s.lam, **kw)
    h = dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, dt=0.1, precision=prec, **kw)
    Rd, Nd = h.rates()
    tol = 1e-5 if prec == "fp32c" else 1e-12
    assert _relerr(Rd, Rd_ref) <= tol
    assert _relerr(Nd, Nd_ref) <= tol
    R_ref, N_ref = oracle.sa_heun(s.R0, s.N0, s.phi, s.lam, dt=0.1, nsteps=200, **kw)
    h.step(200)
    R, N = h.state()
    h.close()
    # the state moves by dR; its error is the rates' error times the motion, plus rounding of R
    dR = np.abs(R_ref - s.R0).max()
    assert np.abs(R - R_ref).max() <= 10 * tol * dR + 1e-13 * np.abs(R_ref).max()
    np.testing.assert_allclose(np.linalg.norm(N, axis=1), 1.0, rtol=1e-14)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("S", [2, 33, 129, 300, 1000, 2500, 5000])
def test_stroke_averaged_rates_sizes(S, prec):
    # every split of the averaged-model kernel (1 .. 32 targets per CTA), ragged
    # last CTAs and tiles, against the oracle's rates; S = 5000 has more CTAs
    # than SMs (the plain-launch branch, state loaded in the epilogue)
    s = inputs.paper_scale(S, seed=21 + S)
    kw = dict(a=s.a, ell=s.ell, omega=s.omega)
    Rd_ref, Nd_ref = oracle.sa_rates(s.R0, s.N0, s.phi, s.lam, **kw)
    h = dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, dt=0.1, precision=prec, **kw)
    Rd, Nd = h.rates()
    h.close()
    tol = 1e-5 if prec == "fp32c" else 1e-12
    assert _relerr(Rd, Rd_ref) <= tol
    assert _relerr(Nd, Nd_ref) <= tol


@pytest.mark.parametrize("S", [2, 33, 300, 1000])
def test_pair_distance_error_matches_oracle(S):
    import torch
    rng = np.random.default_rng(12 + S)
    A0 = rng.uniform(-20, 20, (S, 3))
    A1 = A0 + rng.normal(scale=0.01, size=(S, 3))
    B0 = A0.copy()
    B1 = A0 + rng.normal(scale=0.01, size=(S, 3))
    t = [torch.from_numpy(a).cuda() for a in (A0, A1, B0, B1)]
    got = dbs.pair_distance_error(S, *t)
    ref = oracle.pair_distance_error(oracle.pair_distance_change(A0, A1),
                                     oracle.pair_distance_change(B0, B1))
    assert got["max"] == pytest.approx(ref["max"], rel=1e-12)
    assert got["rms"] == pytest.approx(ref["rms"], rel=1e-10)
    assert got["ref_rms"] == pytest.approx(ref["ref_rms"], rel=1e-10)
    # the enqueued form: the same kernel, its values left on the device (two calls
    # in a row on one stream, into two rows)
    out = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    dbs.pair_distance_error_async(S, *t, out[0], stream=s)
    dbs.pair_distance_error_async(S, t[0], t[2], t[0], t[2], out[1], stream=s)
    s.synchronize()
    o = out.cpu().numpy()
    assert list(o[0]) == [got["max"], got["rms"], got["ref_rms"], got["pairs"]]
    assert o[1, 0] == 0.0 and o[1, 1] == 0.0 and o[1, 3] == S * (S - 1) / 2
