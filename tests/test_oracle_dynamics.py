"""Pins of the oracle's spring force (Eq. (4)), Heun integrator (Sec. IV) and
stroke-period averages (Eqs. (6b), (7b)) against closed forms and reductions.

* An isolated dumbbell cannot swim (Purcell's scallop theorem, Sec. I and the
  single-dumbbell check of Sec. IV): its centroid never moves and its axis
  never turns, while its length obeys the scalar ODE
      dd/dt = -2 k0 (d - L(t)) (1/(6 pi mu a) - h(d)),
  h = 1/(4 pi mu d) (Oseen) or 1/(4 pi mu d) - a^2/(6 pi mu d^3) (RPY),
  which a library ODE solver integrates to 1e-12.
* Heun is second order: the error against the ODE solution drops 4x when dt halves.
* A dumbbell at rest length with lambda = 0 under a uniform external force
  drifts at the constant two-sphere speed, so its stroke average over
  [kT, (k+1)T] is the centre at (k + 1/2) T.
* Aligned pairs (Sec. III.A, Fig. 1): with phase difference pi/2 both
  dumbbells move the same way at equal speed and keep their separation; with
  zero phase difference the pair does not translate; the displacement per
  period falls off as D^-4.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_1004_1932_b300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _single(mob, lam=0.2, phi=0.7, a=0.05, mu=1.0, k0=1.0, ell=1.0):
    Nv = np.array([[0.36, -0.48, 0.8]])
    R = np.array([[1.5, -0.25, 2.0]])
    x0 = inputs.spheres_at_rest(R, Nv, ell, np.array([lam]), np.array([phi]))
    # start off the minimum so the relaxation term is exercised too
    x0[1] += 0.05 * Nv[0]
    return x0, dict(a=a, mu=mu, k0=k0, ell=ell, omega=2 * math.pi, lam=np.array([lam]),
                    phi=np.array([phi]))


def _scalar_ode(x0, p, mob, t_end):
    a, mu, k0, ell, om = p["a"], p["mu"], p["k0"], p["ell"], p["omega"]
    lam, phi = p["lam"][0], p["phi"][0]

    def h(d):
        out = 1.0 / (4 * math.pi * mu * d)
        if mob == oracle.RPY:
            out -= a * a / (6 * math.pi * mu * d ** 3)
        return out

    def rhs(t, y):
        d = y[0]
        L = ell + lam * math.sin(om * t + phi)
        return [-2 * k0 * (d - L) * (1 / (6 * math.pi * mu * a) - h(d))]

    d0 = np.linalg.norm(x0[1] - x0[0])
    sol = solve_ivp(rhs, (0, t_end), [d0], method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[0, -1]


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_isolated_dumbbell_scallop_and_length_ode(mob):
    x0, p = _single(mob)
    dt, n = 1e-3, 1500
    x = oracle.heun(x0, 0, n, dt=dt, mobility=mob, **p)
    c0 = 0.5 * (x0[0] + x0[1])
    c1 = 0.5 * (x[0] + x[1])
    np.testing.assert_allclose(c1, c0, rtol=0, atol=1e-14)            # no net swimming
    N0 = (x0[1] - x0[0]) / np.linalg.norm(x0[1] - x0[0])
    N1 = (x[1] - x[0]) / np.linalg.norm(x[1] - x[0])
    np.testing.assert_allclose(N1, N0, rtol=0, atol=1e-14)            # no rotation
    d_ref = _scalar_ode(x0, p, mob, n * dt)
    assert abs(np.linalg.norm(x[1] - x[0]) - d_ref) < 1e-6   # Heun O(dt^2) global error


def test_heun_second_order():
    x0, p = _single(oracle.RPY)
    t_end = 1.0
    d_ref = _scalar_ode(x0, p, oracle.RPY, t_end)
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        x = oracle.heun(x0, 0, int(round(t_end / dt)), dt=dt, mobility=oracle.RPY, **p)
        errs.append(abs(np.linalg.norm(x[1] - x[0]) - d_ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


def test_stroke_average_of_uniform_drift():
    a, mu, ell = 0.05, 1.0, 1.0
    Nv = np.array([[0.0, 0.6, 0.8]])
    R = np.array([[0.3, 0.1, -0.2]])
    x0 = inputs.spheres_at_rest(R, Nv, ell, np.array([0.0]), np.array([0.0]))
    Fe = np.array([[0.2, -0.1, 0.05], [0.2, -0.1, 0.05]])
    # two-sphere drift speed at separation ell (Oseen), force components along/across N
    Fpar = np.dot(Fe[0], Nv[0]) * Nv[0]
    Fperp = Fe[0] - Fpar
    V = Fe[0] / (6 * math.pi * mu * a) + Fpar / (4 * math.pi * mu * ell) + Fperp / (8 * math.pi * mu * ell)
    m, nper, dt = 200, 3, 5e-3
    T = m * dt
    p = dict(a=a, mu=mu, k0=1.0, ell=ell, omega=2 * math.pi / T, lam=np.array([0.0]), phi=np.array([0.0]))
    _, Rbar = oracle.heun_period_avg(x0, 0, m, nper, dt=dt, mobility=oracle.OSEEN, Fext=Fe, **p)
    for k in range(nper):
        np.testing.assert_allclose(Rbar[k, 0], R[0] + V * (k + 0.5) * T, rtol=1e-12, atol=1e-13)


def _aligned_pair(D_over_ell, dphi, periods=3):
    g = GOLDEN["fig1_parameters"]
    ell = g["ell_m"]
    a, lam = g["a_over_ell"] * ell, g["lambda_over_ell"] * ell
    omega = g["omega_per_s"]
    T = 2 * math.pi / omega
    m = int(round(1 / g["dt_over_T"]))
    dt = T / m
    Nv = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    R = np.array([[0.0, 0.0, 0.0], [D_over_ell * ell, 0.0, 0.0]])
    phi = np.array([0.0, dphi])
    lam_a = np.array([lam, lam])
    x0 = inputs.spheres_at_rest(R, Nv, ell, lam_a, phi)
    p = dict(a=a, mu=g["mu_pa_s"], k0=g["k0_kg_per_s2"], ell=ell, omega=omega, lam=lam_a, phi=phi)
    _, Rbar = oracle.heun_period_avg(x0, 0, m, periods, dt=dt, mobility=oracle.RPY, **p)
    return Rbar, ell, a, lam, omega


@pytest.mark.slow
def test_aligned_pair_comoves_and_decays_as_D4():
    disp = {}
    for D in (5.0, 10.0):
        Rbar, ell, a, lam, omega = _aligned_pair(D, GOLDEN["fig1_parameters"]["dphi"])
        # discard the first period (Sec. IV settling transient); per-period displacement after it
        d1 = Rbar[2, :, 0] - Rbar[1, :, 0]
        # both dumbbells move the same way at equal speed, separation kept
        assert d1[0] * d1[1] > 0
        assert abs(d1[0] - d1[1]) < 0.05 * abs(d1[0])
        assert np.abs(Rbar[2, :, 1:]).max() < 1e-12 * ell
        disp[D] = 0.5 * (d1[0] + d1[1])
    # D^-4 law (Sec. III.A, Fig. 1b): 16x between D=5 and D=10, up to near-field corrections
    ratio = disp[5.0] / disp[10.0]
    assert 12.0 < ratio < 20.0, ratio


@pytest.mark.slow
def test_aligned_pair_in_phase_does_not_swim():
    Rbar_in, ell, *_ = _aligned_pair(10.0, 0.0)
    Rbar_q, *_ = _aligned_pair(10.0, GOLDEN["fig1_parameters"]["dphi"])
    move_in = np.abs(Rbar_in[2, :, 0] - Rbar_in[1, :, 0]).max()
    move_q = np.abs(Rbar_q[2, :, 0] - Rbar_q[1, :, 0]).max()
    # a reciprocal (in-phase) stroke gives at most a residue far below the pi/2 drift
    assert move_in < 0.05 * move_q


def test_spring_force_is_minus_gradient_of_potential():
    """Eq. (4): F = -dU/dX, checked by central differences of U."""
    rng = np.random.default_rng(7)
    S = 3
    x = rng.normal(size=(2 * S, 3))
    lam = rng.uniform(0.1, 0.3, S)
    phi = rng.uniform(0, 2 * math.pi, S)
    ell, om, k0, t = 1.0, 2 * math.pi, 1.7, 0.37

    def U(xx):
        tot = 0.0
        for s in range(S):
            d = np.linalg.norm(xx[2 * s + 1] - xx[2 * s])
            L = ell + lam[s] * math.sin(om * t + phi[s])
            tot += 0.5 * k0 * (d - L) ** 2
        return tot

    F = oracle.spring_forces(x, ell, lam, om, phi, k0, t)
    h = 1e-6
    for i in range(2 * S):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            assert abs(F[i, k] + (U(xp) - U(xm)) / (2 * h)) < 1e-8
    # force-free per dumbbell (internal force, Sec. II)
    np.testing.assert_allclose(F[0::2] + F[1::2], 0.0, atol=0)
