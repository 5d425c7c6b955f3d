"""Pins of the oracle's shape-driven model (Appendix A.2).

* Isolated dumbbell: the constraint force is dL/dt / b^{ss} with the printed
  b^{ss} = (4 kappa / L)(1 - 2L/(3a)), kappa = 1/(8 pi mu) (Oseen); it neither
  translates nor rotates, and Heun keeps its length on L(t) exactly.
* The iteration f_(n) converges to the exact solution of the constraint
  equations, computed independently as one dense linear solve in 40-digit
  arithmetic (oracle.shape_driven.rates).
* Stiff-spring limit: the spring model of Eq. (4) approaches the shape-driven
  model as k0 grows (the statement that motivates the shape-driven model),
  with an error falling like 1/k0.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
from oracle import shape_driven
from paper_1004_1932_b300 import inputs


def _kw(s):
    kw = s.phys()
    kw.pop("k0")
    return kw


def test_isolated_dumbbell():
    s = inputs.make_suspension(1, seed=0, side=8.0, mobility="oseen")
    Rd, Nd, f = oracle.sd_rates(s.x0, 0.0, 1, mobility=oracle.OSEEN, **_kw(s))
    L = s.ell + s.lam[0] * math.sin(s.phi[0])
    Ld = s.lam[0] * s.omega * math.cos(s.phi[0])
    kappa = 1 / (8 * math.pi * s.mu)
    bss = 4 * kappa / L * (1 - 2 * L / (3 * s.a))
    assert f[0] == pytest.approx(Ld / bss, rel=1e-13)
    v_scale = abs(Ld)
    assert np.abs(Rd).max() <= 1e-14 * v_scale
    assert np.abs(Nd).max() <= 1e-14 * v_scale
    nsteps = 300
    x = oracle.sd_heun(s.x0, 0, nsteps, 1, dt=s.dt, mobility=oracle.OSEEN, **_kw(s))
    t = nsteps * s.dt
    assert np.linalg.norm(x[1] - x[0]) == pytest.approx(s.ell + s.lam[0] * math.sin(s.omega * t + s.phi[0]), rel=1e-13)
    np.testing.assert_allclose(0.5 * (x[0] + x[1]), 0.5 * (s.x0[0] + s.x0[1]), atol=1e-13)
    n0 = (s.x0[1] - s.x0[0]) / np.linalg.norm(s.x0[1] - s.x0[0])
    n1 = (x[1] - x[0]) / np.linalg.norm(x[1] - x[0])
    np.testing.assert_allclose(n1, n0, atol=1e-13)


def test_iteration_converges_to_the_exact_constraint_solution():
    s = inputs.make_suspension(3, seed=4, side=6.0, mobility="oseen")
    Rd, Nd, f = oracle.sd_rates(s.x0, 0.0, 80, mobility=oracle.OSEEN, **_kw(s))
    R = [list(map(mp.mpf, 0.5 * (s.x0[2 * i] + s.x0[2 * i + 1]))) for i in range(3)]
    Nv = []
    for i in range(3):
        e = s.x0[2 * i + 1] - s.x0[2 * i]
        Nv.append(list(map(mp.mpf, e / np.linalg.norm(e))))
    L = [mp.mpf(s.ell) + mp.mpf(s.lam[i]) * mp.sin(mp.mpf(s.phi[i])) for i in range(3)]
    Ld = [mp.mpf(s.lam[i]) * mp.mpf(s.omega) * mp.cos(mp.mpf(s.phi[i])) for i in range(3)]
    exact = shape_driven.rates(R, Nv, L, Ld, mp.mpf(s.a), mp.mpf(s.mu))
    Re = np.array([[float(c) for c in r] for r, _ in exact])
    Ne = np.array([[float(c) for c in n] for _, n in exact])
    assert np.abs(Rd - Re).max() <= 1e-10 * np.abs(Re).max()
    assert np.abs(Nd - Ne).max() <= 1e-10 * np.abs(Ne).max()


def test_stiff_spring_limit():
    s = inputs.make_suspension(2, seed=1, side=5.0, mobility="oseen")
    dt, nsteps = 2e-5, 2000
    kw = _kw(s)
    kw.pop("dt", None)
    shape = oracle.sd_heun(s.x0, 0, nsteps, 30, dt=dt, mobility=oracle.OSEEN, **kw)
    errs = []
    for k0 in (1e2, 1e3, 1e4):
        spring = oracle.heun(s.x0, 0, nsteps, dt=dt, mobility=oracle.OSEEN, k0=k0, **kw)
        errs.append(np.abs(spring - shape).max())
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1]
