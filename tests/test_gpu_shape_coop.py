"""GPU parity of the shape-driven dynamics (Appendix A.2) on the cooperative path.

* FP32C trajectories with n = 1, 2, 3 constraint iterations, Oseen and RPY,
  follow oracle.sd_heun within the FP32C tolerance (1e-4 ell after 300 steps),
  with every length on L(t) to FP64 rounding.
* At paper scale (splits of 2 to 16 dumbbells per CTA, ragged last CTAs) the
  cooperative path ends where the grid path ends; runs longer than one launch
  (1024 steps) continue where the last launch ended; stroke averages match the
  grid path's; dbs_velocities afterwards reports H F for the constraint forces;
  the kernel refuses a launch shape other than the one it was told (DBS_E_CUDA).
* FP64 stays on the grid path (DBS_E_STATE), and switching back to the spring
  model on the cooperative path continues the run.
"""
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


def _lengths_on_L(x, s, nsteps):
    t = nsteps * s.dt
    L = s.ell + s.lam * np.sin(s.omega * t + s.phi)
    np.testing.assert_allclose(np.linalg.norm(x[1::2] - x[0::2], axis=1), L, rtol=1e-12)


@pytest.mark.parametrize("mob,iters", [("oseen", 1), ("rpy", 2), ("oseen", 3), ("rpy", 3)])
def test_coop_shape_trajectory_matches_oracle(mob, iters):
    s = inputs.make_suspension(12, seed=8, side=7.0, mobility=mob)
    nsteps = 300
    ref = oracle.sd_heun(s.x0, 0, nsteps, iters, dt=s.dt, mobility=MOB[mob], **_kw(s))
    with _handle(s) as h:
        h.set_path("coop")
        h.set_dynamics("shape", iters)
        assert h.get_path()[0] == "coop"
        h.step(nsteps)
        x = h.positions()
        assert h.get_time()[0] == nsteps
    assert np.abs(x - ref).max() <= 1e-4 * s.ell
    _lengths_on_L(x, s, nsteps)


@pytest.mark.parametrize("S,iters", [(100, 2), (300, 1), (512, 2), (1000, 2), (2048, 3)])
def test_coop_shape_matches_grid_path(S, iters):
    s = inputs.paper_scale(S, seed=S + 3)
    nsteps = 200
    with _handle(s) as hg:
        hg.set_dynamics("shape", iters)
        hg.step(nsteps)
        xg = hg.positions()
    with _handle(s) as hc:
        hc.set_dynamics("shape", iters)   # dynamics first, then the path: either order works
        hc.set_path("coop")
        hc.step(nsteps)
        xc = hc.positions()
    assert np.abs(xc - xg).max() <= 1e-6 * s.ell
    _lengths_on_L(xc, s, nsteps)


def test_coop_shape_long_run_averages_and_velocities():
    s = inputs.make_suspension(40, seed=12, side=12.0, mobility="rpy")
    m, periods = 1000, 2                # period averages over 1000 steps: 2 launches each
    nsteps = m * periods + 100
    out = []
    for path in ("grid", "coop"):
        with _handle(s) as h:
            h.set_path(path)
            h.set_dynamics("shape", 2)
            h.enable_period_average(m, max_periods=periods)
            h.step(37)
            h.step(nsteps - 37)
            x = h.positions()
            Rbar = h.period_averages(0, periods)
            v = h.velocities()
            out.append((x, Rbar, v))
    (xg, Rg, vg), (xc, Rc, vc) = out
    assert np.abs(xc - xg).max() <= 1e-6 * s.ell
    assert np.abs(Rc - Rg).max() <= 1e-6 * s.ell
    assert np.abs(vc - vg).max() <= 1e-5 * np.abs(vg).max()
    _lengths_on_L(xc, s, nsteps)


def test_coop_shape_restrictions_and_return_to_spring():
    s = inputs.make_suspension(16, seed=11, side=8.0)
    with _handle(s, "fp64") as h:
        h.set_dynamics("shape", 2)
        with pytest.raises(dbs.DbsError) as ei:
            h.set_path("coop")
        assert ei.value.status == dbs.E_STATE
    with _handle(s) as h:
        h.set_path("coop")
        h.set_dynamics("shape", 2)
        h.step(50)
        x_mid, n_mid = h.get_state()
        h.set_dynamics("spring")
        assert h.get_path()[0] == "coop"
        h.step(50)
        x = h.positions()
    ref = oracle.heun(x_mid, n_mid, 50, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
    assert np.abs(x - ref).max() <= 1e-4 * s.ell


def test_coop_shape_kernel_refuses_a_launch_shape_it_was_not_built_for():
    # told one CTA more than it was launched with, every CTA refuses before
    # touching state or exchange words; the device and the path stay usable
    lib = dbs.load()
    s = inputs.paper_scale(512, seed=13)
    h = _handle(s)
    h.set_path("coop")
    h.set_dynamics("shape", 2)
    assert lib.dbs_test_flow_misshape(h._h) == dbs.E_CUDA
    assert "shape" in lib.dbs_last_error(h._h).decode()
    h.close()
    with _handle(s) as h2:
        h2.set_path("coop")
        h2.set_dynamics("shape", 2)
        h2.step(4)
        assert np.isfinite(h2.positions()).all()
