"""The paper's experiments run on the library (every step on the GPU).

lattice_msd      Figs. 3-4 (Sec. III.C): dumbbells on an x^3 cubic lattice,
                 W seeded orientation sets, checkerboard or random phases; the
                 mean square displacement of the stroke-averaged centres over
                 one stroke period after the first (settling) period is
                 discarded, <<R(T)^2>> = mean_w mean_s |Rbar_2 - Rbar_1|^2.
                 All W systems advance together as one ensemble.
lattice_msd_sa   the same quantity from the stroke-averaged model of
                 Eqs. (9a)-(9e) started from the same initial condition.
colloids_rate    Sec. IV speed-up workload: N colloids under a constant force
                 (Oseen); GPU Heun steps per second.

    python -m paper_1004_1932_b300.experiments lattice --x 5 --W 100 --spacing 10 [--phases random]
    python -m paper_1004_1932_b300.experiments colloids --N 2000 --steps 2000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import dbs, inputs


def lattice_systems(x, spacing_over_ell, W, phases, seed0=0, **kw):
    ell = kw.get("ell", 5e-6)
    return [inputs.lattice(x, spacing_over_ell * ell, seed=seed0 + w, phases=phases, **kw)
            for w in range(W)]


def lattice_msd(x=5, spacing_over_ell=10.0, W=100, phases="checkerboard", periods=3, seed0=0,
                precision="fp32c", **kw):
    """<<R(T)^2>> of the microscopic model, the W systems batched as one ensemble."""
    systems = lattice_systems(x, spacing_over_ell, W, phases, seed0, **kw)
    s0 = systems[0]
    T = 2 * math.pi / s0.omega
    m = int(round(T / s0.dt))
    hs = [dbs.Suspension.from_inputs(s, precision=precision) for s in systems]
    for h in hs:
        h.enable_period_average(m, max_periods=periods)
    t0 = time.perf_counter()
    if precision == "fp32c":
        with dbs.Ensemble(hs) as e:
            e.step(m * periods)
            e.sync()
    else:
        for h in hs:
            h.step(m * periods)
        for h in hs:
            h.sync()
    el = time.perf_counter() - t0
    Rbar = np.stack([h.period_averages(0, periods) for h in hs])   # [W, periods, S, 3]
    for h in hs:
        h.close()
    d = Rbar[:, 2, :, :] - Rbar[:, 1, :, :] if periods >= 3 else Rbar[:, -1] - Rbar[:, 0]
    msd = float(np.mean(np.sum(d * d, axis=-1)))
    return {"x": x, "S": s0.S, "W": W, "spacing_over_ell": spacing_over_ell, "phases": phases,
            "density_per_m3": 1.0 / (spacing_over_ell * s0.ell) ** 3, "msd_m2": msd,
            "msd_over_ell2": msd / s0.ell ** 2, "steps": m * periods, "seconds": el,
            "system_steps_per_s": W * m * periods / el, "Rbar": Rbar}


def lattice_msd_sa(x=5, spacing_over_ell=10.0, W=100, phases="checkerboard", seed0=0,
                   sa_steps=100, precision="fp64", **kw):
    """<<R(T)^2>> of the stroke-averaged model over one period from the same initial
    condition (the averaged model has no settling transient)."""
    systems = lattice_systems(x, spacing_over_ell, W, phases, seed0, **kw)
    s0 = systems[0]
    T = 2 * math.pi / s0.omega
    out = []
    for s in systems:
        sa = dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega,
                                dt=T / sa_steps, precision=precision)
        sa.step(sa_steps)
        R, _ = sa.state()
        sa.close()
        out.append(np.sum((R - s.R0) ** 2, axis=-1))
    msd = float(np.mean(out))
    return {"x": x, "W": W, "spacing_over_ell": spacing_over_ell, "phases": phases, "msd_m2": msd,
            "msd_over_ell2": msd / s0.ell ** 2}


def colloids_rate(N=2000, steps=2000, mobility="oseen", precision="fp32c"):
    s, F = inputs.colloids(N, mobility=mobility)
    with dbs.Suspension.from_inputs(s, precision=precision) as h:
        h.set_external_force(F)
        h.step(64)
        h.sync()
        t0 = time.perf_counter()
        h.step(steps)
        h.sync()
        el = time.perf_counter() - t0
    return {"N": N, "steps": steps, "seconds": el, "heun_steps_per_s": steps / el,
            "pairs_per_s": 2 * N * (N - 1) * steps / el}


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    la = sub.add_parser("lattice")
    la.add_argument("--x", type=int, default=5)
    la.add_argument("--W", type=int, default=100)
    la.add_argument("--spacing", type=float, nargs="+", default=[10.0])
    la.add_argument("--phases", default="checkerboard", choices=["checkerboard", "random"])
    la.add_argument("--dt-over-T", type=float, default=1e-4)
    la.add_argument("--sa", action="store_true", help="also the stroke-averaged model")
    co = sub.add_parser("colloids")
    co.add_argument("--N", type=int, default=2000)
    co.add_argument("--steps", type=int, default=2000)
    a = ap.parse_args(argv)
    if a.cmd == "lattice":
        for sp in a.spacing:
            r = lattice_msd(a.x, sp, a.W, a.phases, dt_over_T=a.dt_over_T)
            r.pop("Rbar")
            if a.sa:
                r["sa_msd_over_ell2"] = lattice_msd_sa(a.x, sp, a.W, a.phases,
                                                       dt_over_T=a.dt_over_T)["msd_over_ell2"]
            print(json.dumps(r), flush=True)
    else:
        print(json.dumps(colloids_rate(a.N, a.steps)), flush=True)


if __name__ == "__main__":
    main()
