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
    a = ap.parse_args(argv)
    s = inputs.paper_scale(a.S, seed=a.seed, mobility=a.mobility)
    with dbs.Suspension.from_inputs(s, precision=a.precision, device=0) as h:
        ms = h.step_timed(a.steps)
    N = 2 * a.S
    print(json.dumps({"S": a.S, "N": N, "mobility": a.mobility, "precision": a.precision,
                      "ms_per_launch": ms,
                      "tflops": N * (N - 1) * FLOPS_PER_PAIR[a.mobility] / (ms * 1e-3) / 1e12}))


if __name__ == "__main__":
    main()
