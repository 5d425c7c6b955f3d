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


def test_colloids_follow_oracle():
    s, F = inputs.colloids(200, seed=2)
    ref = oracle.heun(s.x0, 0, 300, dt=s.dt, mobility=oracle.OSEEN, Fext=F, **s.phys())
    with dbs.Suspension.from_inputs(s) as h:
        h.set_external_force(F)
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
