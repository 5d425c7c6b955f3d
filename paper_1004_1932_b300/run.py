"""Run one seeded suspension on the GPU and report the pair-sum launch time.

    python -m paper_1004_1932_b300.run --S 512 --mobility rpy --steps 20 [--precision fp32c]

Creates the paper-scale workload (density 0.002, lambda 0.2, seeded), advances
it ``--steps`` Heun steps one launch at a time (``dbs_step_timed``) and prints
the mean device time of one pair-sum launch with the algorithmic FP32 rate.
This is the command the profiles in ``profiles/`` are taken with.
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
    ap.add_argument("--path", default="grid", choices=["grid", "cluster"])
    ap.add_argument("--cluster", type=int, default=0, help="cluster size of the cluster path (0 = auto)")
    a = ap.parse_args(argv)
    s = inputs.paper_scale(a.S, seed=a.seed, mobility=a.mobility)
    N = 2 * a.S
    with dbs.Suspension.from_inputs(s, precision=a.precision, device=0) as h:
        if a.path == "grid":
            ms = h.step_timed(a.steps)
            print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "precision": a.precision,
                              "path": "grid", "ms_per_launch": ms,
                              "tflops": N * (N - 1) * FLOPS_PER_PAIR[a.mobility] / (ms * 1e-3) / 1e12}))
        else:
            import time
            h.set_path("cluster", a.cluster)
            h.sync()
            t0 = time.perf_counter()
            h.step(a.steps)
            h.sync()
            el = time.perf_counter() - t0
            print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "path": "cluster",
                              "cluster": h.get_path()[1], "ms_per_step": 1e3 * el / a.steps}))


if __name__ == "__main__":
    main()
