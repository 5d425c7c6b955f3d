"""Pins of the oracle's stroke-averaged far-field model, Eqs. (9a)-(9e), Sec. III.

* The exact (unexpanded) stroke average of two shape-driven Oseen dumbbells
  (Appendix A.2 construction, ``oracle.shape_driven``) converges to the
  oracle's J and K at generic geometries as a/ell, lambda/ell, ell/D -> 0.
  This fixes the prefactors (printed 9/64 and 15/64), the signs and every
  polynomial coefficient; the appendix contraction's 15/32 is ruled out.
* Aligned dumbbells reduce to the 1d law of Eq. (10) with its printed 9/16.
* J and K vanish when the phases differ by a multiple of pi (Sec. III.B (iii)).
* Aligned pairs do not rotate (Sec. III.A).
* |J| ~ D^-4 and |K| ~ D^-5 (Sec. III.B (i), (ii)).
* Heun on (R, N) is second order and keeps |N| = 1.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import shape_driven

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


GEOMS = [
    # (Dhat, N^s, N^r, phi^s, phi^r)
    (_unit([0.5, -0.3, 0.8]), _unit([0.3, 0.8, -0.5]), _unit([-0.6, 0.2, 0.7]), 0.4, 1.9),
    (_unit([1.0, 0.2, -0.1]), _unit([0.1, 0.1, 1.0]), _unit([0.7, -0.7, 0.1]), 2.5, 0.3),
    (_unit([-0.2, 0.9, 0.3]), _unit([0.9, 0.3, 0.1]), _unit([0.5, 0.5, -0.7]), 5.0, 1.2),
]


def _rel_err(Dmag, small, geom):
    Dh, Ns, Nr, ps, pr = geom
    ell, omega, mu = 1.0, 2 * math.pi, 1.0
    a = lam = small
    R = np.stack([Dmag * Dh, np.zeros(3)])
    Nv = np.stack([Ns, Nr])
    exact = shape_driven.stroke_averaged_rates(R, Nv, [ps, pr], ell=ell, lam=lam, omega=omega,
                                               a=a, mu=mu, M=8)
    Rd, Nd = oracle.sa_rates(R, Nv, np.array([ps, pr]), np.array([lam, lam]), a=a, ell=ell,
                             omega=omega)
    ej = np.linalg.norm(np.array(exact[0][0]) - Rd[0]) / np.linalg.norm(Rd[0])
    en = np.linalg.norm(np.array(exact[0][1]) - Nd[0]) / np.linalg.norm(Nd[0])
    return ej, en


@pytest.mark.parametrize("g", range(len(GEOMS)))
def test_far_field_law_is_limit_of_exact_stroke_average(g):
    coarse = _rel_err(20.0, 0.01, GEOMS[g])
    fine = _rel_err(80.0, 0.0025, GEOMS[g])
    # first-order convergence in the small parameters: ~4x smaller error, and small
    for c, f in zip(coarse, fine):
        assert f < 0.012, (coarse, fine)
        assert f < 0.45 * c, (coarse, fine)


def test_appendix_contraction_prefactor_is_ruled_out():
    """With K prefactor 15/32 the rotation rate would be off by a factor of 2."""
    Dh, Ns, Nr, ps, pr = GEOMS[0]
    R = np.stack([80.0 * Dh, np.zeros(3)])
    Nv = np.stack([Ns, Nr])
    exact = shape_driven.stroke_averaged_rates(R, Nv, [ps, pr], ell=1.0, lam=0.0025,
                                               omega=2 * math.pi, a=0.0025, mu=1.0, M=8)
    _, Nd = oracle.sa_rates(R, Nv, np.array([ps, pr]), np.array([0.0025] * 2), a=0.0025, ell=1.0,
                            omega=2 * math.pi, kpref=15.0 / 32.0)
    assert np.linalg.norm(np.array(exact[0][1]) - Nd[0]) / np.linalg.norm(Nd[0]) > 0.4


def test_aligned_pair_reduces_to_1d_law():
    c916 = GOLDEN["sa_1d_coefficient"]["value"]
    a, ell, lam, omega = 0.2, 1.0, 0.1, 500.0
    for D, dphi in ((10.0, math.pi / 2), (4.0, 0.7), (25.0, -2.0)):
        ax = _unit([0.2, -0.4, 0.9])
        R = np.stack([np.zeros(3), D * ax])
        Nv = np.stack([ax, ax])
        phi = np.array([0.0, dphi])
        Rd, Nd = oracle.sa_rates(R, Nv, phi, np.array([lam, lam]), a=a, ell=ell, omega=omega)
        for s, r in ((0, 1), (1, 0)):
            Dh = _unit(R[s] - R[r])
            expect = c916 * a * omega * math.sin(phi[s] - phi[r]) * (lam / ell) ** 2 * (ell / D) ** 4 * Dh
            np.testing.assert_allclose(Rd[s], expect, rtol=1e-13, atol=1e-30)
        np.testing.assert_allclose(Nd, 0.0, atol=1e-14 * np.abs(Rd).max())   # aligned: no rotation
        # both dumbbells move the same way at equal speed (Fig. 1a)
        np.testing.assert_allclose(Rd[0], Rd[1], rtol=1e-13)


def test_phase_locked_pairs_do_not_interact():
    rng = np.random.default_rng(3)
    S = 6
    R = rng.uniform(-10, 10, size=(S, 3))
    Nv = np.array([_unit(v) for v in rng.normal(size=(S, 3))])
    phi = 0.37 + math.pi * rng.integers(-3, 4, size=S)
    Rd, Nd = oracle.sa_rates(R, Nv, phi, np.full(S, 0.2), a=0.05, ell=1.0, omega=2 * math.pi)
    assert np.abs(Rd).max() < 1e-17 and np.abs(Nd).max() < 1e-17


def test_distance_scaling():
    Dh, Ns, Nr, ps, pr = GEOMS[1]
    vals = []
    for D in (10.0, 20.0, 40.0):
        Rd, Nd = oracle.sa_rates(np.stack([D * Dh, np.zeros(3)]), np.stack([Ns, Nr]),
                                 np.array([ps, pr]), np.array([0.2, 0.2]), a=0.05, ell=1.0,
                                 omega=2 * math.pi)
        vals.append((np.linalg.norm(Rd[0]), np.linalg.norm(Nd[0])))
    for k in range(2):
        np.testing.assert_allclose(vals[k][0] / vals[k + 1][0], 16.0, rtol=1e-12)
        np.testing.assert_allclose(vals[k][1] / vals[k + 1][1], 32.0, rtol=1e-12)


def test_rates_orthogonal_and_antisymmetric_in_pair():
    rng = np.random.default_rng(8)
    S = 12
    R = rng.uniform(-12, 12, size=(S, 3))
    Nv = np.array([_unit(v) for v in rng.normal(size=(S, 3))])
    phi = rng.uniform(0, 2 * math.pi, S)
    Rd, Nd = oracle.sa_rates(R, Nv, phi, rng.uniform(0.1, 0.3, S), a=0.05, ell=1.0,
                             omega=2 * math.pi)
    # dN/dt is tangent to the unit sphere
    np.testing.assert_allclose(np.sum(Nd * Nv, axis=1), 0.0, atol=1e-20)
    # a pair's J is odd under exchanging the dumbbells when N^s = N^r (Eq. (9c):
    # s <-> -r, sin(dphi) flips): the pair centre-of-mass moves, relative motion cancels
    R2 = np.stack([R[0], R[1]])
    N2 = np.stack([Nv[0], Nv[0]])
    Rd2, _ = oracle.sa_rates(R2, N2, phi[:2], np.array([0.2, 0.2]), a=0.05, ell=1.0,
                             omega=2 * math.pi)
    np.testing.assert_allclose(Rd2[0], Rd2[1], rtol=1e-12)


def test_sa_heun_second_order_and_unit_norm():
    rng = np.random.default_rng(9)
    S = 8
    R = rng.uniform(-3, 3, size=(S, 3)) * 1.5
    Nv = np.array([_unit(v) for v in rng.normal(size=(S, 3))])
    phi = rng.uniform(0, 2 * math.pi, S)
    lam = np.full(S, 0.3)
    kw = dict(a=0.2, ell=1.0, omega=2 * math.pi * 50)
    t_end = 1.0
    ref_R, ref_N = oracle.sa_heun(R, Nv, phi, lam, dt=t_end / 512, nsteps=512, **kw)
    errs = []
    for n in (16, 32, 64):
        R1, N1 = oracle.sa_heun(R, Nv, phi, lam, dt=t_end / n, nsteps=n, **kw)
        np.testing.assert_allclose(np.linalg.norm(N1, axis=1), 1.0, rtol=1e-14)
        errs.append(np.abs(R1 - ref_R).max())
    assert errs[0] > 0
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


def test_pair_distance_change():
    R0 = np.array([[0.0, 0, 0], [3.0, 0, 0], [0, 4.0, 0]])
    R1 = np.array([[0.0, 0, 0], [3.5, 0, 0], [0, 4.0, 1.0]])
    dD = oracle.pair_distance_change(R0, R1)
    np.testing.assert_allclose(dD, dD.T)
    assert dD[0, 1] == pytest.approx(0.5)
    assert dD[0, 2] == pytest.approx(math.sqrt(17.0) - 4.0)
    assert dD[1, 2] == pytest.approx(math.sqrt(3.5 ** 2 + 17.0) - 5.0)
    e = oracle.pair_distance_error(dD, np.zeros_like(dD))
    assert e["max"] == pytest.approx(max(0.5, math.sqrt(17) - 4, math.sqrt(3.5 ** 2 + 17) - 5))
