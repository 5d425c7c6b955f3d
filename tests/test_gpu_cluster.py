"""GPU parity of the cluster-resident path and of ensembles.

* A suspension stepped on the cluster path follows the FP64 oracle within the
  trajectory tolerance (1e-4 ell after 1000 Heun steps), and the grid path
  within the same tolerance.
* Members of an ensemble (different sizes, amplitudes, mobilities and cluster
  sizes) end where the same systems end when stepped alone on the grid path;
  stroke averages accumulated inside the resident kernel match the oracle's.
* Chunks of steps larger than one resident launch (1024 steps) continue the
  clock and the step counter exactly.
* The benchmark's 256-system ensemble: sampled members (smallest, median,
  largest) follow the oracle over 20 steps, every member stays finite.
* The resident kernel refuses a launch in a shape other than the one it was
  built for (told to expect twice its cluster size) with DBS_E_CUDA, before
  touching member state, and the device stays usable.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
MOB = {"oseen": oracle.OSEEN, "rpy": oracle.RPY}


def _handle(s, **kw):
    return dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                          mobility=s.mobility, precision="fp32c", lam=s.lam, phi=s.phi, **kw)


@pytest.mark.parametrize("S,mob,G", [(16, "oseen", 0), (16, "rpy", 2), (300, "rpy", 0), (300, "oseen", 4)])
def test_cluster_path_follows_oracle(S, mob, G):
    s = inputs.make_suspension(S, seed=S + 7, density=0.002, mobility=mob) if S > 16 \
        else inputs.make_suspension(S, seed=0, side=8.0, mobility=mob)
    nsteps = 1000
    ref = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[mob], **s.phys())
    with _handle(s) as h:
        h.set_path("cluster", G)
        path, g = h.get_path()
        assert path == "cluster" and g >= 1
        h.step(nsteps)
        x = h.positions()
        assert h.get_time()[0] == nsteps
    assert np.abs(x - ref).max() <= 1e-4 * s.ell


def test_cluster_path_continues_grid_path_and_counts_steps():
    s = inputs.make_suspension(200, seed=3, density=0.002)
    with _handle(s) as hg:
        hg.step(1500)
        xg = hg.positions()
    with _handle(s) as hc:
        hc.step(100)                 # grid
        hc.set_path("cluster")
        hc.step(1300)                # cluster: one full resident launch + a partial one
        hc.set_path("grid")
        hc.step(100)                 # grid again
        xc = hc.positions()
        assert hc.get_time()[0] == 1500
        v = hc.velocities()
    assert np.isfinite(v).all()
    assert np.abs(xc - xg).max() <= 1e-4 * s.ell


def test_ensemble_members_match_alone():
    specs = [(8, 0.1, "rpy"), (37, 0.3, "oseen"), (130, 0.2, "rpy"), (600, 0.15, "rpy"), (9, 0.25, "oseen")]
    systems = [inputs.make_suspension(S, seed=i, density=0.002, lam=lam, mobility=mob)
               for i, (S, lam, mob) in enumerate(specs)]
    nsteps = 600
    alone = []
    for s in systems:
        with _handle(s) as h:
            h.step(nsteps)
            alone.append(h.positions())
    hs = [_handle(s) for s in systems]
    with dbs.Ensemble(hs) as e:
        G = e.get_clusters()
        assert len(G) == len(hs) and all(g in (1, 2, 4, 8, 16) for g in G)
        e.step(nsteps)
        e.sync()
        for s, h, ref in zip(systems, hs, alone):
            x = h.positions()
            assert h.get_time()[0] == nsteps
            assert np.abs(x - ref).max() <= 1e-4 * s.ell
        # explicit cluster sizes (the autotuner's hook) give the same trajectories
        e.set_clusters([1, 1, 2, 4, 1])
        e.step(50)
        e.sync()
    for h in hs:
        h.close()


def test_full_ensemble_sampled_members_follow_oracle():
    # the batched-ensemble workload the benchmark times: 256 systems, S log-uniform
    # in [8, 2048], amplitudes in [0.1, 0.3], built-in cluster sizes; the smallest,
    # median-sized and largest members against the oracle, every member finite
    systems = inputs.ensemble(256)
    nsteps = 20
    hs = [_handle(s) for s in systems]
    with dbs.Ensemble(hs) as e:
        e.step(nsteps)
        e.sync()
    order = sorted(range(len(systems)), key=lambda i: systems[i].S)
    for i in order[:2] + order[127:129] + order[-1:]:
        s = systems[i]
        ref = oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=MOB[s.mobility], **s.phys())
        x = hs[i].positions()
        assert hs[i].get_time()[0] == nsteps
        assert np.abs(x - ref).max() <= 1e-6 * s.ell
    for h in hs:
        assert np.isfinite(h.positions()).all()
        h.close()


def test_ensemble_period_average_matches_oracle():
    s = inputs.make_suspension(24, seed=4, side=10.0, mobility="rpy")
    m, nper = 100, 3
    dt = 1.0 / m
    _, Rbar_ref = oracle.heun_period_avg(s.x0, 0, m, nper, dt=dt, mobility=oracle.RPY, **s.phys())
    h = dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=dt,
                       mobility="rpy", precision="fp32c", lam=s.lam, phi=s.phi)
    h.enable_period_average(m, max_periods=8)
    h.set_path("cluster")
    h.step(m * nper + 7)
    assert h.period_count() == nper
    Rbar = h.period_averages()
    h.close()
    assert np.abs(Rbar - Rbar_ref).max() <= 1e-4 * s.ell


def test_ensemble_rejects_fp64_members():
    s = inputs.make_suspension(10, seed=1, side=8.0)
    h = dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                       precision="fp64")
    with pytest.raises(dbs.DbsError) as ei:
        dbs.Ensemble([h])
    assert ei.value.status == dbs.E_ARG
    h.close()


def test_cluster_path_refusal_leaves_handle_usable():
    s = inputs.make_suspension(5000, seed=2, density=0.002)   # beyond both the cluster and cooperative paths
    h = dbs.Suspension(s.x0, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                       precision="fp32c", lam=s.lam, phi=s.phi)
    with pytest.raises(dbs.DbsError) as ei:
        h.set_path("cluster")
    assert ei.value.status == dbs.E_ARG
    with pytest.raises(dbs.DbsError):
        h.set_path("coop")
    assert h.get_path()[0] == "grid"
    h.step(2)
    assert np.isfinite(h.positions()).all()
    h.close()


def test_resident_kernel_refuses_a_launch_shape_it_was_not_built_for():
    # two launch classes (a small and a large member); both kernels are told to
    # expect twice their cluster size and must refuse
    members = [_handle(inputs.paper_scale(S, seed=S)) for S in (40, 300)]
    ens = dbs.Ensemble(members)
    lib = dbs.load()
    rc = lib.dbs_test_ensemble_misshape(ens._h)
    assert rc == dbs.E_CUDA
    assert "shape" in lib.dbs_ensemble_last_error(ens._h).decode()
    ens.close()
    for m in members:
        m.close()
    # the device stays usable
    h = _handle(inputs.paper_scale(40, seed=40))
    h.step(2)
    assert np.isfinite(h.positions()).all()
    h.close()
