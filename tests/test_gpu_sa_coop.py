"""GPU parity of the cooperative path of the stroke-averaged model (Sec. III.B).

* FP32C systems with S <= 4096 take the cooperative path by default; FP64 ones
  and larger ones keep one launch per evaluation, and asking for the
  cooperative path there is refused with DBS_E_ARG, leaving the handle usable.
* Stepped on the cooperative path, every split (2 .. 32 dumbbells per CTA,
  one CTA holding a whole system, ragged last CTAs) follows the FP64 oracle's
  Heun steps of Eqs. (9a)-(9e) within the FP32C tolerance of the
  one-launch-per-evaluation path, and ends where that path ends; N stays a
  unit vector to FP64 rounding.
* Runs longer than one launch (1024 averaged steps) continue where the last
  launch ended, the rates read after cooperative steps are those of the
  current state, and two runs from one state are bit-identical.
* The kernel refuses a launch in a shape other than the one it was told
  (DBS_E_CUDA), before touching state or exchange words; the device and the
  path stay usable.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5   # FP32 pair sums, relative to the largest rate


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _sa(s, precision="fp32c", dt=0.1):
    return dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega, dt=dt,
                              precision=precision)


def _motion_bound(R, R_ref, R0, tol):
    # the state moves by dR; its error is the rates' error times the motion, plus rounding of R
    dR = np.abs(R_ref - R0).max()
    return np.abs(R - R_ref).max() <= 10 * tol * dR + 1e-13 * np.abs(R_ref).max()


def test_path_choice_and_refusals():
    s = inputs.paper_scale(512, seed=3)
    with _sa(s) as h:
        assert h.get_path() == ("coop", 4)
    with _sa(s, precision="fp64") as h:
        assert h.get_path() == ("grid", 0)
        with pytest.raises(dbs.DbsError) as ei:
            h.set_path("coop")
        assert ei.value.status == dbs.E_ARG
        h.step(2)                       # still usable
        assert np.isfinite(h.state()[0]).all()
    big = inputs.paper_scale(4097, seed=4)
    with _sa(big) as h:
        assert h.get_path()[0] == "grid"
        with pytest.raises(dbs.DbsError):
            h.set_path("coop")
        h.step(1)
        assert np.isfinite(h.state()[0]).all()


@pytest.mark.parametrize("S", [2, 17, 148, 297, 300, 512, 1000, 2369, 4096])   # 2 .. 32 per CTA
def test_coop_follows_oracle_and_grid_path(S):
    s = inputs.paper_scale(S, seed=40 + S)
    kw = dict(a=s.a, ell=s.ell, omega=s.omega)
    nsteps = 60
    R_ref, N_ref = oracle.sa_heun(s.R0, s.N0, s.phi, s.lam, dt=0.1, nsteps=nsteps, **kw)
    with _sa(s) as hc:
        assert hc.get_path()[0] == "coop"
        hc.step(nsteps)
        Rc, Nc = hc.state()
    with _sa(s) as hg:
        hg.set_path("grid")
        hg.step(nsteps)
        Rg, Ng = hg.state()
    assert _motion_bound(Rc, R_ref, s.R0, TOL)
    assert np.abs(Nc - N_ref).max() <= 1e-4 * max(np.abs(N_ref - s.N0).max(), 1e-12) + 1e-12
    np.testing.assert_allclose(np.linalg.norm(Nc, axis=1), 1.0, rtol=1e-14)
    assert np.abs(Rc - Rg).max() <= 10 * TOL * np.abs(Rg - s.R0).max() + 1e-13 * np.abs(Rg).max()


def test_coop_long_run_rates_and_determinism():
    s = inputs.paper_scale(96, seed=7)
    kw = dict(a=s.a, ell=s.ell, omega=s.omega)
    nsteps = 2100                       # three launches of at most 1024 steps
    R_ref, N_ref = oracle.sa_heun(s.R0, s.N0, s.phi, s.lam, dt=0.1, nsteps=nsteps, **kw)
    runs = []
    for _ in range(2):
        with _sa(s) as h:
            h.step(1000)
            h.step(nsteps - 1000)
            R, N = h.state()
            Rd, Nd = h.rates()          # at the current state (records repacked)
            runs.append((R, N))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    R, N = runs[0]
    assert _motion_bound(R, R_ref, s.R0, TOL)
    Rd_ref, Nd_ref = oracle.sa_rates(R, N, s.phi, s.lam, **kw)
    assert _relerr(Rd, Rd_ref) <= TOL
    assert _relerr(Nd, Nd_ref) <= TOL


def test_switching_paths_mid_run():
    s = inputs.paper_scale(300, seed=8)
    kw = dict(a=s.a, ell=s.ell, omega=s.omega)
    R_ref, _ = oracle.sa_heun(s.R0, s.N0, s.phi, s.lam, dt=0.1, nsteps=90, **kw)
    with _sa(s) as h:
        h.step(30)
        h.set_path("grid")
        h.step(30)
        h.set_path("coop")
        h.step(30)
        R, N = h.state()
    assert _motion_bound(R, R_ref, s.R0, TOL)
    np.testing.assert_allclose(np.linalg.norm(N, axis=1), 1.0, rtol=1e-14)


def test_cooperative_kernel_refuses_a_launch_shape_it_was_not_built_for():
    # told one CTA more than it was launched with, every CTA refuses before
    # touching state or exchange words; the host reports it, the state is kept
    lib = dbs.load()
    s = inputs.paper_scale(512, seed=5)
    h = _sa(s)
    h.step(3)
    R0, N0 = h.state()
    assert lib.dbs_test_sa_flow_misshape(h._h) == dbs.E_CUDA
    assert "shape" in lib.dbs_sa_last_error(h._h).decode()
    with pytest.raises(dbs.DbsError):          # sticky
        h.step(1)
    h.close()
    # the device and the cooperative path stay usable, from the same state
    with dbs.StrokeAveraged(R0, N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega, dt=0.1) as h2:
        assert h2.get_path()[0] == "coop"
        h2.step(4)
        R, N = h2.state()
    assert np.isfinite(R).all() and np.isfinite(N).all()
    with _sa(s, precision="fp64") as hf:       # not on the cooperative path
        assert lib.dbs_test_sa_flow_misshape(hf._h) == dbs.E_STATE
