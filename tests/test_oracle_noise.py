"""Pins of the oracle's additive-noise path (closing remarks of Sec. IV).

* Philox4x32-10 reproduces the published known-answer vectors
  (tests/golden/philox4x32_10_kat.txt).
* The Box-Muller normals have mean 0, unit variance, the normal 1-sigma mass
  and uncorrelated components (statistical tolerances of 5 standard errors).
* kT = 0 gives exactly the deterministic Heun trajectory.
* Free spheres (k0 = 0: no force, so no drift) diffuse with the variance
  2 kT dt / (6 pi mu a) per component and step: the Stokes-Einstein
  coefficient of the self part of Eq. (3).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(oracle.philox4x32_10(ctr, key)) == out


def test_normals_statistics():
    z = np.array([oracle.sphere_normals(7, n, i) for n in range(20) for i in range(2500)])
    x = z.ravel()
    m = x.size
    assert abs(x.mean()) < 5 / math.sqrt(m)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / m)
    p1 = np.mean(np.abs(x) < 1.0)
    assert abs(p1 - math.erf(1 / math.sqrt(2))) < 5 * math.sqrt(0.68 * 0.32 / m)
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 5 / math.sqrt(z.shape[0])


def test_zero_temperature_is_deterministic_heun():
    s = inputs.make_suspension(8, seed=2, side=8.0)
    a = oracle.heun(s.x0, 3, 40, dt=s.dt, mobility=oracle.RPY, **s.phys())
    b = oracle.heun(s.x0, 3, 40, dt=s.dt, mobility=oracle.RPY, kT=0.0, seed=5, **s.phys())
    assert np.array_equal(a, b)


def test_free_diffusion_matches_stokes_einstein():
    s = inputs.make_suspension(1000, seed=3, density=0.002)
    kw = s.phys()
    kw["k0"] = 0.0
    kT, nsteps = 0.02, 50
    x = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=oracle.OSEEN, kT=kT, seed=11, **kw)
    d2 = (x - s.x0) ** 2
    D0 = kT / (6 * math.pi * s.mu * s.a)
    expected = 2 * D0 * nsteps * s.dt
    m = d2.size
    assert abs(d2.mean() / expected - 1.0) < 5 * math.sqrt(2.0 / m)
