"""Pins of the oracle's mobility (Eq. (3), Sec. II) against facts other than itself.

* The tensor is rebuilt symbolically from the Stokes Green's function:
  Oseen = (delta lap - grad grad) r / (8 pi mu) (the Stokeslet written as the
  biharmonic potential r), and for equal spheres the RPY pair term is
  (1 + a^2/3 lap) applied to it (lap^2 of the Stokeslet vanishes for r > 0).
  None of this retypes the printed closed form.
* Two-sphere drift (Stokes drag plus the Oseen/RPY correction) for forces
  parallel and perpendicular to the line of centres.
* Reciprocity, symmetry and positive definiteness (Sec. II: H is positive
  definite for r > 2a), translation/rotation invariance, and the paper's own
  full-tensor method against the pair loop.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle

MU = 1.3
A = 0.07


def _symbolic_tensor(a_val, mu_val, rpy):
    X = sp.symbols("x0:3", real=True)
    r = sp.sqrt(sum(c * c for c in X))
    lap = lambda f: sum(sp.diff(f, c, 2) for c in X)
    O = [[(sp.KroneckerDelta(i, j) * lap(r) - sp.diff(r, X[i], X[j])) / (8 * sp.pi * mu_val)
          for j in range(3)] for i in range(3)]
    if rpy:
        O = [[O[i][j] + sp.Rational(1, 3) * a_val ** 2 * lap(O[i][j]) for j in range(3)]
             for i in range(3)]
    return sp.lambdify(X, sp.Matrix(O), "numpy")


@pytest.fixture(scope="module")
def sym_tensors():
    return {rpy: _symbolic_tensor(sp.Float(A), sp.Float(MU), rpy) for rpy in (False, True)}


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_tensor_matches_greens_function(sym_tensors, mob):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 3)) * 2.0
    H = oracle.mobility_matrix(x, A, MU, mob)
    f = sym_tensors[mob == oracle.RPY]
    for al in range(5):
        for be in range(5):
            blk = H[3 * al:3 * al + 3, 3 * be:3 * be + 3]
            if al == be:
                # Stokes drag of one sphere: v = F / (6 pi mu a)
                np.testing.assert_allclose(blk, np.eye(3) / (6 * math.pi * MU * A), rtol=1e-14)
            else:
                ref = np.array(f(*(x[al] - x[be])), dtype=float)
                np.testing.assert_allclose(blk, ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_two_sphere_drift(mob):
    r = 3.7
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    stokes = 1.0 / (6 * math.pi * MU * A)
    par = stokes + 1.0 / (4 * math.pi * MU * r)
    perp = stokes + 1.0 / (8 * math.pi * MU * r)
    if mob == oracle.RPY:
        par += -A * A / (6 * math.pi * MU * r ** 3)
        perp += A * A / (12 * math.pi * MU * r ** 3)
    for F, speed in (([2.0, 0.0, 0.0], par), ([0.0, -1.5, 0.0], perp), ([0.0, 0.0, 0.5], perp)):
        Fs = np.array([F, F])
        v = oracle.mobility_apply(x, Fs, A, MU, mob)
        np.testing.assert_allclose(v, Fs * speed, rtol=1e-14, atol=1e-16)
        # the pair drifts rigidly: separation unchanged
        np.testing.assert_allclose(v[0], v[1], rtol=1e-15, atol=0)


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_reciprocity_and_symmetry(mob):
    rng = np.random.default_rng(2)
    x = rng.uniform(-4, 4, size=(24, 3))
    F1 = rng.normal(size=(24, 3))
    F2 = rng.normal(size=(24, 3))
    v1 = oracle.mobility_apply(x, F1, A, MU, mob)
    v2 = oracle.mobility_apply(x, F2, A, MU, mob)
    assert abs(np.sum(F2 * v1) - np.sum(F1 * v2)) <= 1e-12 * np.sum(np.abs(F2 * v1))
    H = oracle.mobility_matrix(x, A, MU, mob)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-15)


def test_rpy_positive_definite_outside_contact():
    from paper_1004_1932_b300 import inputs
    s = inputs.make_suspension(40, seed=3, side=12.0, a=0.2)
    d = np.linalg.norm(s.x0[:, None, :] - s.x0[None, :, :], axis=-1)
    assert d[~np.eye(80, dtype=bool)].min() > 2 * 0.2
    H = oracle.mobility_matrix(s.x0, 0.2, 1.0, oracle.RPY)
    np.linalg.cholesky(H)  # raises if not positive definite
    assert np.linalg.eigvalsh(H).min() > 0


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_full_tensor_method_equals_pair_loop(mob):
    rng = np.random.default_rng(4)
    x = rng.uniform(-5, 5, size=(30, 3))
    F = rng.normal(size=(30, 3))
    H = oracle.mobility_matrix(x, A, MU, mob)
    v_dense = (H @ F.reshape(-1)).reshape(-1, 3)
    v_loop = oracle.mobility_apply(x, F, A, MU, mob)
    np.testing.assert_allclose(v_loop, v_dense, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mob", [oracle.OSEEN, oracle.RPY])
def test_translation_rotation_invariance(mob):
    rng = np.random.default_rng(5)
    x = rng.uniform(-5, 5, size=(20, 3))
    F = rng.normal(size=(20, 3))
    v = oracle.mobility_apply(x, F, A, MU, mob)
    vt = oracle.mobility_apply(x + np.array([3.25, -1.5, 0.75]), F, A, MU, mob)
    np.testing.assert_allclose(vt, v, rtol=1e-12, atol=1e-13)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    vr = oracle.mobility_apply(x @ q.T, F @ q.T, A, MU, mob)
    np.testing.assert_allclose(vr, v @ q.T, rtol=1e-12, atol=1e-13)


def test_rpy_extra_term_scales_as_a_squared():
    """RPY - Oseen is the a^2 line of Eq. (3b): doubling a multiplies it by 4."""
    rng = np.random.default_rng(6)
    x = rng.uniform(-5, 5, size=(10, 3))
    F = rng.normal(size=(10, 3))
    d1 = oracle.mobility_apply(x, F, A, MU, oracle.RPY) - oracle.mobility_apply(x, F, A, MU, oracle.OSEEN)
    d2 = (oracle.mobility_apply(x, F, 2 * A, MU, oracle.RPY)
          - oracle.mobility_apply(x, F, 2 * A, MU, oracle.OSEEN))
    assert np.abs(d1).max() > 1e-5
    np.testing.assert_allclose(d2, 4 * d1, rtol=1e-9, atol=1e-14)


def test_interaction_is_velocity_minus_stokes_drag():
    rng = np.random.default_rng(10)
    x = rng.uniform(-5, 5, size=(12, 3))
    F = rng.normal(size=(12, 3))
    for mob in (oracle.OSEEN, oracle.RPY):
        u = oracle.interaction(x, F, A, MU, mob)
        v = oracle.mobility_apply(x, F, A, MU, mob)
        np.testing.assert_allclose(u + F / (6 * math.pi * MU * A), v, rtol=1e-13, atol=1e-14)


def test_rows_match_full_apply():
    rng = np.random.default_rng(11)
    x = rng.uniform(-5, 5, size=(40, 3))
    F = rng.normal(size=(40, 3))
    rows = np.array([0, 7, 39, 13])
    for mob in (oracle.OSEEN, oracle.RPY):
        full = oracle.mobility_apply(x, F, A, MU, mob)
        np.testing.assert_array_equal(oracle.mobility_rows(x, F, rows, A, MU, mob), full[rows])
