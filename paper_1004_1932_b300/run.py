"""Run one seeded suspension on the GPU and report its timings.

    python -m paper_1004_1932_b300.run --S 512 --mobility rpy --steps 20 [--precision fp32c]
    python -m paper_1004_1932_b300.run --S 512 --path coop --steps 2048
    python -m paper_1004_1932_b300.run --S 512 --path coop --breakdown 5
    python -m paper_1004_1932_b300.run --S 8192 --sa --steps 20

Creates the paper-scale workload (density 0.002, lambda 0.2, seeded).  On the
grid path it advances ``--steps`` Heun steps one launch at a time
(``dbs_step_timed``) and prints the mean device time of one pair-sum launch
with the algorithmic FP32 rate; on the cluster and cooperative paths it prints
the wall time per Heun step.  ``--breakdown P`` runs P stroke periods of the
benchmark's hot path (1000 Heun steps, 10 stroke-averaged steps, the
pair-distance comparison) and prints the CUDA-event time of each part on the
stream.  ``--sa`` advances the stroke-averaged model alone (dt = T/10) and
prints the CUDA-event time of one of its Heun steps.
"""
import argparse
import json

from . import dbs, inputs

FLOPS_PER_PAIR = {"oseen": 27, "rpy": 34}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--S", type=int, default=512)
    ap.add_argument("--mobility", default="rpy", choices=["rpy", "oseen"])
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--path", default="grid", choices=["grid", "cluster", "coop"])
    ap.add_argument("--breakdown", type=int, default=0, help="stroke periods of the hot path to time by part")
    ap.add_argument("--kT", type=float, default=0.0, help="additive Brownian noise (dbs_set_noise), 0 = off")
    ap.add_argument("--shape", type=int, default=0,
                    help="shape-driven dynamics with this many constraint iterations (0 = spring)")
    ap.add_argument("--cluster", type=int, default=0, help="cluster size of the cluster path (0 = auto)")
    ap.add_argument("--sa", action="store_true", help="the stroke-averaged model alone")
    a = ap.parse_args(argv)
    s = inputs.paper_scale(a.S, seed=a.seed, mobility=a.mobility)
    N = 2 * a.S
    if a.sa:
        print(json.dumps(stroke_averaged(s, a)))
        return
    if a.breakdown:
        print(json.dumps(breakdown(s, a)))
        return
    with dbs.Suspension.from_inputs(s, precision=a.precision, device=0) as h:
        if a.kT > 0:
            h.set_noise(a.kT, a.seed)
        if a.shape > 0:
            import time
            if a.path == "coop":          # shape-driven: grid (default) or cooperative path
                h.set_path("coop")
            h.set_dynamics("shape", a.shape)
            h.step(8)
            h.sync()
            t0 = time.perf_counter()
            h.step(a.steps)
            h.sync()
            el = time.perf_counter() - t0
            print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "precision": a.precision,
                              "dynamics": "shape", "iterations": a.shape, "path": h.get_path()[0],
                              "ms_per_step": 1e3 * el / a.steps,
                              "pair_sums_per_step": 2 * a.shape}))
            return
        if a.path == "grid":
            ms = h.step_timed(a.steps)
            print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "precision": a.precision,
                              "path": "grid", "ms_per_launch": ms,
                              "tflops": N * (N - 1) * FLOPS_PER_PAIR[a.mobility] / (ms * 1e-3) / 1e12}))
        else:
            import time
            h.set_path(a.path, a.cluster)
            h.step(64)
            h.sync()
            t0 = time.perf_counter()
            h.step(a.steps)
            h.sync()
            el = time.perf_counter() - t0
            print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "path": a.path, "kT": a.kT,
                              "cluster": h.get_path()[1], "ms_per_step": 1e3 * el / a.steps}))


def stroke_averaged(s, a):
    """CUDA-event time of one Heun step of the stroke-averaged model (dt = T/10)."""
    import math
    import torch
    stream = torch.cuda.Stream()
    with dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega,
                            dt=2 * math.pi / s.omega / 10, precision=a.precision, stream=stream) as h:
        h.step(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.step(a.steps)
        e1.record(stream)
        e1.synchronize()
    return {"S": a.S, "model": "stroke-averaged", "precision": a.precision, "steps": a.steps,
            "us_per_step": e0.elapsed_time(e1) * 1e3 / a.steps}


def breakdown(s, a):
    """CUDA-event time of each part of the benchmark's stroke period."""
    import math
    import torch
    T = 2 * math.pi / s.omega
    m = int(round(T / s.dt))
    stream = torch.cuda.Stream()
    parts = {"heun": 0.0, "stroke_averaged": 0.0, "comparison": 0.0}
    with dbs.Suspension.from_inputs(s, precision="fp32c", stream=stream) as h, \
            dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega, dt=T / 10,
                               precision="fp32c", stream=stream) as sa, torch.cuda.stream(stream):
        h.set_path(a.path, a.cluster)
        sa.set_path("grid")   # as in bench.py, where it overlaps the microscopic model
        h.enable_period_average(m, max_periods=a.breakdown + 2)
        ref = torch.empty((a.S, 3), dtype=torch.float64, device="cuda")
        for k in range(a.breakdown + 2):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            h.step(m)
            ev[1].record(stream)
            sa.step(10)
            ev[2].record(stream)
            if k == 1:
                sa.copy_centres(ref)
            if k >= 2:
                dbs.pair_distance_error(a.S, h.period_average_device(1), h.period_average_device(k),
                                        ref.data_ptr(), sa.centres_device(), stream=stream)
            ev[3].record(stream)
            ev[3].synchronize()
            if k >= 2:
                parts["heun"] += ev[0].elapsed_time(ev[1])
                parts["stroke_averaged"] += ev[1].elapsed_time(ev[2])
                parts["comparison"] += ev[2].elapsed_time(ev[3])
    tot = sum(parts.values())
    return {"S": a.S, "path": a.path, "periods": a.breakdown,
            "ms_per_period": {k: v / a.breakdown for k, v in parts.items()},
            "share": {k: v / tot for k, v in parts.items()}}


if __name__ == "__main__":
    main()
