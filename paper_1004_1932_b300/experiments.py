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
effective_amplitude
                 the stroke amplitude the dumbbells actually perform: the
                 lengths d_s(t) of the microscopic model over one period
                 (after settling periods) projected on sin and cos of
                 (omega t + phi_s).  The spring model is shape-driven (Sec. II)
                 only when the spring relaxes much faster than one stroke; at
                 k0 = 1, a = 0.05 it lags, so its amplitude is smaller than the
                 rest length's.
sa_comparison    the pair-distance error of the stroke-averaged model of
                 Eqs. (9a)-(9e) against the period-averaged centres of the
                 microscopic model, at given stroke amplitudes.
serving_trace    a Poisson stream of simulation requests through the serving
                 engine (admission by a device-memory budget, continuous
                 batching): makespan, request latencies, and the engine's host
                 accounting (ticks, ensemble rebuilds); the same requests one
                 at a time in arrival order, from measured per-step times.

    python -m paper_1004_1932_b300.experiments lattice --x 5 --W 100 --spacing 10 [--phases random]
    python -m paper_1004_1932_b300.experiments colloids --N 2000 --steps 2000
    python -m paper_1004_1932_b300.experiments serving [--requests 200 --steps-hi 1e5 --rate 200]
    python -m paper_1004_1932_b300.experiments serving --full
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


def effective_amplitude(s, samples=50, settle_periods=4, precision="fp32c", path="coop"):
    """Measured stroke amplitude of the microscopic model (every step on the GPU).

    After ``settle_periods`` periods (the lengths relax from the initial condition
    with a time of about half a period at k0 = 1, a = 0.05: four periods leave
    e^-8 of the transient), the dumbbell lengths d_s(t_k) are read at
    ``samples`` equally spaced times of the next period; their first Fourier
    coefficients against sin(omega t + phi_s) and cos(omega t + phi_s) give
    d_s ~ mean_s + lam_eff_s sin(omega t + phi_s - lag_s).  Returns the
    per-dumbbell lam_eff_s and lag_s and their means."""
    T = 2 * math.pi / s.omega
    m = int(round(T / s.dt))
    if m % samples:
        raise ValueError("samples must divide the steps of one period")
    stride = m // samples
    d = np.empty((samples, s.S))
    tk = np.empty(samples)
    with dbs.Suspension.from_inputs(s, precision=precision) as h:
        if precision == "fp32c" and path:
            h.set_path(path)
        h.step(m * settle_periods)
        for k in range(samples):
            x = h.positions()
            tk[k] = h.get_time()[1]
            d[k] = np.linalg.norm(x[1::2] - x[0::2], axis=1)
            h.step(stride)
    ph = s.omega * tk[:, None] + s.phi[None, :]
    dev = d - d.mean(axis=0)
    A = 2.0 / samples * np.sum(dev * np.sin(ph), axis=0)
    B = 2.0 / samples * np.sum(dev * np.cos(ph), axis=0)
    lam_eff = np.hypot(A, B)
    lag = np.arctan2(-B, A)
    return {"lam_eff": lam_eff, "lag": lag, "lam_eff_mean": float(lam_eff.mean()),
            "ratio_mean": float(np.mean(lam_eff / s.lam)), "lag_mean": float(lag.mean())}


def linear_response_ratio(s):
    """Amplitude ratio and lag of an isolated dumbbell's length in the linearised
    spring model: d' = -kappa (d - L(t)) with kappa = 2 k0 (1/(6 pi mu a) - h(ell)),
    h the pair mobility along the axis (Oseen 1/(4 pi mu r), RPY minus
    a^2/(6 pi mu r^3), Eq. (3b)); ratio = 1/sqrt(1 + (omega/kappa)^2)."""
    r = s.ell
    h = 1.0 / (4 * math.pi * s.mu * r)
    if s.mobility == "rpy":
        h -= s.a ** 2 / (6 * math.pi * s.mu * r ** 3)
    kappa = 2 * s.k0 * (1.0 / (6 * math.pi * s.mu * s.a) - h)
    w = s.omega / kappa
    return 1.0 / math.sqrt(1.0 + w * w), math.atan(w)


def sa_comparison(s, periods=4, lam=None, sa_steps=10, precision="fp32c", path="coop"):
    """Pair-distance error of the stroke-averaged model against the microscopic
    one: period-averaged centres of periods 1 and ``periods - 1`` (the first
    period is discarded) against the averaged model at the middle of those
    periods, both started from the same initial condition.  ``lam``: the
    averaged model's stroke amplitudes (default: the nominal ones)."""
    import torch
    T = 2 * math.pi / s.omega
    m = int(round(T / s.dt))
    lam = s.lam if lam is None else np.broadcast_to(np.asarray(lam, float), s.lam.shape).copy()
    with dbs.Suspension.from_inputs(s, precision=precision) as h, \
            dbs.StrokeAveraged(s.R0, s.N0, s.phi, lam, a=s.a, ell=s.ell, omega=s.omega,
                               dt=T / sa_steps, precision=precision) as sa:
        if precision == "fp32c" and path:
            h.set_path(path)
        h.enable_period_average(m, max_periods=periods)
        h.step(m * periods)
        sa.step(sa_steps + sa_steps // 2)                     # middle of period 1
        ref = torch.empty((s.S, 3), dtype=torch.float64, device="cuda")
        sa.copy_centres(ref)
        sa.step(sa_steps * (periods - 2))                     # middle of period periods - 1
        torch.cuda.synchronize()
        A0, A1 = h.period_average_device(1), h.period_average_device(periods - 1)
        out = dbs.pair_distance_error(s.S, A0, A1, ref.data_ptr(), sa.centres_device())
        # the same call with the models swapped gives the RMS of the microscopic model's change
        full = dbs.pair_distance_error(s.S, ref.data_ptr(), sa.centres_device(), A0, A1)
        return {"max": out["max"], "rms": out["rms"], "sa_rms": out["ref_rms"],
                "full_rms": full["ref_rms"], "pairs": out["pairs"]}


def _quantile(v, p):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(p * (len(v) - 1))))] if v else None


def serving_trace(n_req=200, rate=200.0, steps_lo=1e3, steps_hi=1e5, budget=64 << 30, block=256,
                  sizes=(16, 64, 256, 1024, 4096), seed=0, per_step_s=None):
    """The serving engine on a Poisson trace (every step on the GPU).  Latency =
    completion on the host clock minus the request's arrival time.  The one-at-a-
    time comparison serves the same requests in arrival order, each for steps x
    its size's measured time per Heun step on its fastest single-system path
    (``per_step_s``: {S: seconds}; measured here if not given)."""
    trace = inputs.request_trace(n_req, rate, sizes=sizes, steps_lo=steps_lo, steps_hi=steps_hi,
                                 seed=seed)
    if per_step_s is None:
        per_step_s = step_times(sizes)
    susp = {rid: inputs.make_suspension(S, seed=1000 + rid, density=0.002) for _, S, _, rid in trace}
    eng = dbs.Engine(hbm_budget_bytes=budget, block_steps=block)
    t0 = time.perf_counter()
    ids, arr_of, done = {}, {}, {}
    k = 0
    while len(done) < len(trace):
        now = time.perf_counter() - t0
        while k < len(trace) and trace[k][0] <= now:
            arr, S, n, rid = trace[k]
            ids[rid] = eng.submit_inputs(susp[rid], n)
            arr_of[rid] = (arr, time.perf_counter() - t0)
            k += 1
        a, q = eng.tick()
        for rid, eid in ids.items():
            if rid in done:
                continue
            st, _, lat = eng.poll(eid)
            if st in (dbs.REQ_DONE, dbs.REQ_FAILED, dbs.REQ_CANCELLED):
                arr, sub = arr_of[rid]
                done[rid] = (st, (sub - arr) + lat)
        if a == 0 and q == 0 and k < len(trace):
            time.sleep(max(0.0, trace[k][0] - (time.perf_counter() - t0)))
    makespan = time.perf_counter() - t0
    stats = eng.stats()
    eng.close()
    lat = [v[1] for v in done.values() if v[0] == dbs.REQ_DONE]
    steps_total = sum(n for _, _, n, _ in trace)
    t_free, lat_seq = 0.0, []
    for arr, S, n, _ in trace:
        t_free = max(arr, t_free) + n * per_step_s[S]
        lat_seq.append(t_free - arr)
    return {"requests": n_req, "rate_per_s": rate, "steps": [steps_lo, steps_hi],
            "budget_bytes": budget, "block_steps": block, "completed": len(lat),
            "engine": {"makespan_s": makespan, "system_steps_per_s": steps_total / makespan,
                       "requests_per_s": len(lat) / makespan,
                       "p50_latency_s": _quantile(lat, 0.5), "p99_latency_s": _quantile(lat, 0.99)},
            "engine_host": stats,
            "one_at_a_time_modelled": {"makespan_s": t_free, "system_steps_per_s": steps_total / t_free,
                                       "p50_latency_s": _quantile(lat_seq, 0.5),
                                       "p99_latency_s": _quantile(lat_seq, 0.99),
                                       "per_step_s": {str(k_): v for k_, v in per_step_s.items()}}}


def step_times(sizes=(16, 64, 256, 1024, 4096), steps=400):
    """Seconds per Heun step of one suspension of each size on its fastest
    single-system path (the cooperative path up to 4096 dumbbells)."""
    out = {}
    for S in sizes:
        s = inputs.make_suspension(S, seed=5, density=0.002)
        with dbs.Suspension.from_inputs(s, precision="fp32c") as h:
            if S <= 4096:
                h.set_path("coop")
            h.step(32)
            h.sync()
            t0 = time.perf_counter()
            h.step(steps)
            h.sync()
            out[S] = (time.perf_counter() - t0) / steps
    return out


def serving_full():
    """The serving configuration: a 200-request Poisson trace (200 requests/s,
    steps log-uniform in [1e3, 1e5], 64 GB budget); the same request mix at half
    the engine's measured capacity (100 requests); and a small budget (room for
    three of the largest requests) that makes admission queue."""
    per_step = step_times()
    full = serving_trace(200, 200.0, 1e3, 1e5, per_step_s=per_step)
    cap = full["engine"]["requests_per_s"]
    half = serving_trace(100, 0.5 * cap, 1e3, 1e5, seed=1, per_step_s=per_step)
    small = serving_trace(48, 200.0, 1e3, 1e4, budget=3 * dbs.request_bytes(4096), seed=2,
                          per_step_s=per_step)
    return {"offered_200_per_s": full, "half_capacity": {"rate_per_s": 0.5 * cap, **half},
            "small_budget": small}


def colloids_rate(N=2000, steps=2000, mobility="oseen", precision="fp32c", path="auto"):
    """Heun steps per second of N colloids under a constant force; `path` "auto"
    times the stepping paths first (autotune.choose_path) and keeps the fastest."""
    from . import autotune
    s, F = inputs.colloids(N, mobility=mobility)
    with dbs.Suspension.from_inputs(s, precision=precision) as h:
        h.set_external_force(F)
        if path == "auto":
            path = autotune.choose_path(h)["path"]
        else:
            h.set_path(path)
        h.step(64)
        h.sync()
        t0 = time.perf_counter()
        h.step(steps)
        h.sync()
        el = time.perf_counter() - t0
    return {"N": N, "steps": steps, "path": path, "seconds": el, "heun_steps_per_s": steps / el,
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
    co.add_argument("--path", default="auto", choices=["auto", "grid", "cluster", "coop"])
    sv = sub.add_parser("serving")
    sv.add_argument("--full", action="store_true", help="the three runs of serving_full()")
    sv.add_argument("--requests", type=int, default=48)
    sv.add_argument("--rate", type=float, default=200.0)
    sv.add_argument("--steps-hi", type=float, default=1e4)
    a = ap.parse_args(argv)
    if a.cmd == "serving":
        r = serving_full() if a.full else serving_trace(a.requests, a.rate, 1e3, a.steps_hi)
        print(json.dumps(r), flush=True)
        return
    if a.cmd == "lattice":
        for sp in a.spacing:
            r = lattice_msd(a.x, sp, a.W, a.phases, dt_over_T=a.dt_over_T)
            r.pop("Rbar")
            if a.sa:
                r["sa_msd_over_ell2"] = lattice_msd_sa(a.x, sp, a.W, a.phases,
                                                       dt_over_T=a.dt_over_T)["msd_over_ell2"]
            print(json.dumps(r), flush=True)
    else:
        print(json.dumps(colloids_rate(a.N, a.steps, path=a.path)), flush=True)


if __name__ == "__main__":
    main()
