"""The paper's other workloads on the GPU path.

* Colloids under a constant force (Sec. IV speed-up workload, Oseen): GPU
  trajectory against the oracle.
* Lattice ensembles (Sec. III.C, Figs. 3-4): each ensemble member's stroke
  averages against the oracle; then the physics the paper reports for them:
  the mean square displacement per period scales as rho^(8/3) (= spacing^-8,
  the D^-4 far-field law squared) at large spacing, and the checkerboard phase
  pattern moves the lattice more than random phases.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, experiments, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", ["grid", "coop"])
def test_colloids_follow_oracle(path):
    s, F = inputs.colloids(200, seed=2)
    ref = oracle.heun(s.x0, 0, 300, dt=s.dt, mobility=oracle.OSEEN, Fext=F, **s.phys())
    with dbs.Suspension.from_inputs(s) as h:
        h.set_external_force(F)
        h.set_path(path)
        h.step(300)
        x = h.positions()
    assert np.abs(x - ref).max() <= 1e-4
    # every colloid sinks (force along -z), faster than an isolated sphere (hydrodynamic drag reduction)
    dz = x[:, 2] - s.x0[:, 2]
    assert np.all(dz < 0)
    assert np.mean(-dz) > 300 * s.dt / (6 * math.pi * s.mu * s.a)


def test_lattice_members_follow_oracle():
    r = experiments.lattice_msd(x=3, spacing_over_ell=10.0, W=2, phases="random", periods=2,
                                dt_over_T=1e-3 * 0.5)
    for w in range(2):
        s = inputs.lattice(3, 10.0 * 5e-6, seed=w, phases="random", dt_over_T=1e-3 * 0.5)
        m = int(round(2 * math.pi / s.omega / s.dt))
        _, Rbar_ref = oracle.heun_period_avg(s.x0, 0, m, 2, dt=s.dt, mobility=oracle.RPY, **s.phys())
        assert np.abs(r["Rbar"][w] - Rbar_ref).max() <= 1e-4 * s.ell


@pytest.mark.slow
def test_lattice_msd_scaling_and_phase_pattern():
    kw = dict(x=3, W=6, periods=3, dt_over_T=1e-4)
    near = experiments.lattice_msd(spacing_over_ell=8.0, phases="checkerboard", **kw)["msd_m2"]
    far = experiments.lattice_msd(spacing_over_ell=16.0, phases="checkerboard", **kw)["msd_m2"]
    ratio = near / far
    assert 100 < ratio < 700, ratio          # ideal 2^8 = 256 for MSD ~ spacing^-8
    rnd = experiments.lattice_msd(spacing_over_ell=8.0, phases="random", **kw)["msd_m2"]
    assert near > rnd                         # checkerboard beats random phases (Figs. 3, 4)


def test_lattice_x5_members_follow_oracle():
    # a larger lattice (x = 5, S = 125: the paper's Fig. 3 size) on the batched
    # ensemble path against the oracle's stroke averages
    r = experiments.lattice_msd(x=5, spacing_over_ell=10.0, W=2, phases="checkerboard", periods=2,
                                dt_over_T=5e-4)
    assert r["S"] == 125
    for w in range(2):
        s = inputs.lattice(5, 10.0 * 5e-6, seed=w, phases="checkerboard", dt_over_T=5e-4)
        m = int(round(2 * math.pi / s.omega / s.dt))
        _, Rbar_ref = oracle.heun_period_avg(s.x0, 0, m, 2, dt=s.dt, mobility=oracle.RPY, **s.phys())
        assert np.abs(r["Rbar"][w] - Rbar_ref).max() <= 1e-4 * s.ell


def test_effective_amplitude_follows_linear_response():
    # the k0 = 1, a = 0.05 springs lag the rest length: each dumbbell's length
    # oscillates with ~0.30 of the nominal amplitude, lagging ~73 degrees, as the
    # linearised isolated-dumbbell length equation predicts (Eqs. (3), (4))
    s = inputs.paper_scale(256, seed=8)
    r = experiments.effective_amplitude(s)
    ratio, lag = experiments.linear_response_ratio(s)
    assert abs(r["ratio_mean"] - ratio) <= 0.02 * ratio
    assert abs(r["lag_mean"] - lag) <= math.radians(2.0)
    assert np.all(np.abs(r["lam_eff"] / s.lam - ratio) <= 0.1 * ratio)


def test_effective_amplitude_matches_oracle_trajectory():
    # the same measurement on an oracle trajectory of a small dense suspension
    s = inputs.make_suspension(16, seed=2, side=8.0)
    r = experiments.effective_amplitude(s, samples=50, settle_periods=1, path="coop")
    m = int(round(2 * math.pi / s.omega / s.dt))
    stride = m // 50
    x = oracle.heun(s.x0, 0, m, dt=s.dt, mobility=oracle.RPY, **s.phys())
    d, tk = [], []
    for k in range(50):
        d.append(np.linalg.norm(x[1::2] - x[0::2], axis=1))
        tk.append((m + k * stride) * s.dt)
        x = oracle.heun(x, m + k * stride, stride, dt=s.dt, mobility=oracle.RPY, **s.phys())
    d, tk = np.array(d), np.array(tk)
    ph = s.omega * tk[:, None] + s.phi[None, :]
    dev = d - d.mean(axis=0)
    lam_ref = np.hypot(2 / 50 * np.sum(dev * np.sin(ph), axis=0), 2 / 50 * np.sum(dev * np.cos(ph), axis=0))
    assert np.abs(r["lam_eff"] - lam_ref).max() <= 1e-6


def test_averaged_model_at_the_measured_amplitude_tracks_the_full_model():
    # the stroke-averaged model with the nominal amplitude overpredicts the soft
    # springs' motion ~10x; with each dumbbell's measured amplitude its
    # pair-distance error drops well below the microscopic model's own change
    s = inputs.paper_scale(128, seed=4)
    eff = experiments.effective_amplitude(s)
    nominal = experiments.sa_comparison(s, periods=8)
    measured = experiments.sa_comparison(s, periods=8, lam=eff["lam_eff"])
    assert nominal["full_rms"] == pytest.approx(measured["full_rms"], rel=1e-12)
    assert nominal["sa_rms"] > 5 * nominal["full_rms"]
    assert measured["rms"] < 0.25 * nominal["rms"]
    assert measured["rms"] < 0.6 * measured["full_rms"]
