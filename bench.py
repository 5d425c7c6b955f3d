"""Benchmark of the active-dumbbell hot path on B300.

Workload (default): one suspension of S=512 dumbbells (N=1024 spheres) at
number density 0.002, stroke amplitude 0.2, k0=1, a=0.05, mu=1, T=1,
dt=1e-3, RPY mobility, FP32 pair math with compensated accumulation and FP64
state; plus the stroke-averaged model of the same initial condition and the
pair-distance comparison of the two.

One benchmark step = one stroke period of the whole hot path:
  * 1000 Heun steps of the microscopic model (two all-pairs evaluations each,
    spring forces, Heun update, stroke-average accumulation of the centres),
  * the stroke-averaged model advanced over the same period (dt_SA = T/10),
  * the pair-distance comparison of the period-averaged centres against the
    averaged model (read back to the host).
Metric: sphere-pair interactions per second = 2 N (N-1) Heun steps / s.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own independent suspension (seed = rank):
weak scaling, no data-path collective; the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEPS_PER_PERIOD = 1000
SA_STEPS_PER_PERIOD = 10
FLOPS_PER_PAIR = {"oseen": 27, "rpy": 34}   # algorithmic FP32 flops (FMA = 2), rsqrt not counted
# the stroke-averaged pair term (Eqs. (9b), (9c)) as the kernel evaluates it: the
# difference vector, its norm, three projections, the amplitude-phase product and the three
# polynomials, the J and K updates; FMA = 2, rsqrt not counted
SA_FLOPS_PER_PAIR = 96
# DRAM bytes (read + write) per launch of the dominant kernel, copied from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same launch:
# the cooperative kernel, 1024 Heun steps, S = 512, RPY (null for any other path
# or size); the line says where the number comes from.
NCU_TRAFFIC = {("coop", 512, "rpy"): 150528 + 6144}
TRAFFIC_SOURCE = ("copied from one ncu capture of the same launch (the benchmark cannot run "
                  "ncu itself); null when no capture of the kernel as it stands exists")
METRIC = "sphere-pair interactions/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200, help="timed stroke periods")
    p.add_argument("--warmup", type=int, default=3, help="untimed stroke periods")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--S", type=int, default=512)
    p.add_argument("--mobility", default="rpy", choices=["rpy", "oseen"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-large", action="store_true", help="skip the N=65536 kernel measurement")
    p.add_argument("--no-ensemble", action="store_true", help="skip the 256-system ensemble measurement")
    p.add_argument("--no-serving", action="store_true", help="skip the serving-trace measurement")
    p.add_argument("--path", default="auto", choices=["auto", "grid", "cluster", "coop"],
                   help="stepping path of the microscopic model (auto: the autotuner times all three)")
    p.add_argument("--cpu-sample-steps", type=int, default=400,
                   help="Heun steps of the oracle timed for the CPU baseline")
    p.add_argument("--no-cpu-sweep", action="store_true",
                   help="skip the oracle's timings on the other workloads (cpu_baseline.sweep)")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Each rank simulates its own independent suspension (weak scaling)."""
    return int(rank)


def _workload_config(S, mobility, flush):
    return {"workload": f"single suspension S={S} (N={2 * S}) density 0.002, lambda=0.2, "
                        f"{mobility.upper()}, FP32 pair math + FP64 state, dt=1e-3, one step = "
                        f"one stroke period ({STEPS_PER_PERIOD} Heun steps) + stroke-averaged "
                        f"model + pair-distance comparison",
            "S": S, "N": 2 * S, "heun_steps_per_step": STEPS_PER_PERIOD,
            "sa_steps_per_step": SA_STEPS_PER_PERIOD, "mobility": mobility,
            "l2": flush}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def _fp32_peak_tflops(sms, mhz):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def _cpu_baseline(S, mobility, nsteps):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the workload."""
    import oracle
    from paper_1004_1932_b300 import inputs
    s = inputs.paper_scale(S, seed=0, mobility=mobility)
    cores = os.cpu_count()
    oracle.set_threads(cores)
    mob = oracle.RPY if mobility == "rpy" else oracle.OSEEN
    oracle.heun(s.x0, 0, 2, dt=s.dt, mobility=mob, **s.phys())  # load / first touch
    t0 = time.perf_counter()
    oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=mob, **s.phys())
    el = time.perf_counter() - t0
    N = 2 * S
    return {"value": 2 * N * (N - 1) * nsteps / el, "unit": METRIC, "cores": cores,
            "kind": "oracle",
            "sample": f"{nsteps} Heun steps of the same S={S} suspension (FP64 C oracle, OpenMP over "
                      f"targets), {el:.2f} s"}


def _cpu_sweep(mobility):
    """The oracle on the other workloads, each on a bounded sample (about 10 s in all):
    the paper-scale suspension on one thread, the small FP64 Oseen suspension per Heun
    step, one velocity evaluation at N = 4096 and 16384 (N = 65536 scaled from 16384 by
    N^2, the pair loop being exactly N(N-1) terms), and the 256-system ensemble from 10
    Heun steps of every 8th member, scaled by its pair count."""
    import oracle
    from paper_1004_1932_b300 import inputs
    cores = os.cpu_count()
    mob = oracle.RPY if mobility == "rpy" else oracle.OSEEN

    def heun_rate(s, nsteps, threads, m=mob):
        oracle.set_threads(threads)
        oracle.heun(s.x0, 0, 1, dt=s.dt, mobility=m, **s.phys())
        t0 = time.perf_counter()
        oracle.heun(s.x0, 0, nsteps, dt=s.dt, mobility=m, **s.phys())
        return (time.perf_counter() - t0) / nsteps

    out = {"cores_all": cores}
    s = inputs.paper_scale(512, seed=0, mobility=mobility)
    el = heun_rate(s, 10, 1)
    out["paper_scale_s512_one_thread"] = {"pairs_per_s": 2 * 1024 * 1023 / el, "ms_per_heun_step": 1e3 * el,
                                          "sample": "10 Heun steps"}
    s1 = inputs.small_fp64_oseen(0)
    out["small_s16_oseen_fp64"] = {
        "us_per_heun_step_one_thread": 1e6 * heun_rate(s1, 1000, 1, oracle.OSEEN),
        "us_per_heun_step_all_cores": 1e6 * heun_rate(s1, 1000, cores, oracle.OSEEN),
        "sample": "1000 Heun steps"}
    oracle.set_threads(cores)
    ev = []
    for S in (2048, 8192):
        sl = inputs.paper_scale(S, seed=0, mobility=mobility)
        t0 = time.perf_counter()
        oracle.velocities(sl.x0, 0.0, mobility=mob, **sl.phys())
        el = time.perf_counter() - t0
        N = 2 * S
        ev.append({"N": N, "s_all_cores": el, "pairs_per_s": N * (N - 1) / el})
    N = 65536
    ev.append({"N": N, "s_all_cores": ev[-1]["s_all_cores"] * (N * (N - 1)) / (16384 * 16383),
               "scaled": "from N = 16384 by N(N-1)"})
    out["velocity_evaluation"] = ev
    systems = inputs.ensemble(256)
    pairs_all = sum(2 * (2 * m.S) * (2 * m.S - 1) for m in systems)
    sample = systems[::8]
    pairs_sample = sum(2 * (2 * m.S) * (2 * m.S - 1) for m in sample)
    t0 = time.perf_counter()
    for m in sample:
        oracle.heun(m.x0, 0, 10, dt=m.dt, mobility=mob, **m.phys())
    el = (time.perf_counter() - t0) / 10 * pairs_all / pairs_sample
    out["ensemble_256"] = {"s_per_step_all_cores": el, "system_steps_per_s": 256 / el,
                           "sample": "10 Heun steps of members 0, 8, ..., 248, scaled by pair count"}
    return out


def ensemble_measure(dbs, inputs, torch, stream, steps=1000, count=256, ws=1, rank=0, dev=None):
    """256 independent suspensions, S log-uniform in [8, 2048], lambda ~ U[0.1, 0.3],
    seeds 0..255: batched on thread-block clusters vs one system per launch.  Over
    several ranks each rank runs its LPT share (pair work S^2 x steps) and the times
    are the maxima over ranks (no collective on the data path)."""
    from paper_1004_1932_b300 import partition
    systems_all = inputs.ensemble(count)
    assign = partition.lpt([partition.pair_work(m.S, steps) for m in systems_all], ws)
    systems = [m for m, r in zip(systems_all, assign) if r == rank]
    hs = [dbs.Suspension.from_inputs(s, precision="fp32c", stream=stream) for s in systems]
    pairs = sum(2 * (2 * s.S) * (2 * s.S - 1) for s in systems_all)
    ens = dbs.Ensemble(hs, stream=stream)
    from paper_1004_1932_b300 import autotune
    tuned = autotune.tune_ensemble(ens, hs)
    ens.step(16)
    ens.sync()
    t0 = time.perf_counter()
    ens.step(steps)
    ens.sync()
    el_b = reduce_max(time.perf_counter() - t0, dev)
    G = ens.get_clusters()
    ens.close()
    seq_steps = max(32, steps // 5)
    for h in hs:
        h.step(32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in hs:
        h.step(seq_steps)
    for h in hs:
        h.sync()
    el_s = reduce_max(time.perf_counter() - t0, dev)
    # the same, each system on its fastest single-system path (cooperative launch)
    for h in hs:
        h.set_path("coop")
        h.step(8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in hs:
        h.step(seq_steps)
    for h in hs:
        h.sync()
    el_c = reduce_max(time.perf_counter() - t0, dev)
    for h in hs:
        h.close()
    b = count * steps / el_b
    sq = count * seq_steps / el_s
    sc = count * seq_steps / el_c
    return {"workload": f"{count} suspensions, S log-uniform in [8, 2048], lambda ~ U[0.1, 0.3], "
                        f"seeds 0..{count - 1}, RPY, FP32C",
            "ranks": ws, "split": "LPT on S^2 x steps, no collective" if ws > 1 else None,
            "batched": {"steps": steps, "seconds": el_b, "system_steps_per_s": b,
                        "pairs_per_s": pairs * steps / el_b,
                        "clusters": {str(g): G.count(g) for g in sorted(set(G))},
                        "autotune": {"choice": tuned["choice"],
                                     "s_per_step": tuned["s_per_step"]},
                        "launch": "one resident launch per class per 1024 steps, replayed from a "
                                  "captured CUDA graph"},
            "one_system_per_launch": {"path": "grid", "steps": seq_steps, "seconds": el_s,
                                      "system_steps_per_s": sq, "pairs_per_s": pairs * seq_steps / el_s},
            "one_system_at_a_time_cooperative": {"steps": seq_steps, "seconds": el_c,
                                                 "system_steps_per_s": sc,
                                                 "pairs_per_s": pairs * seq_steps / el_c},
            "speedup": b / sq, "speedup_vs_cooperative": b / sc}


def _gather_lists(values, ws):
    """Concatenate a per-rank list over all ranks (the metric only, not the data path)."""
    if ws == 1:
        return list(values)
    import torch.distributed as dist
    parts = [None] * ws
    dist.all_gather_object(parts, list(values))
    return [v for p in parts for v in p]


def serving_measure(dbs, inputs, n_req=48, rate=200.0, steps_lo=1e3, steps_hi=1e4, block=256,
                    budget=64 << 30, ws=1, rank=0, dev=None):
    """Poisson trace (mean `rate` req/s), S uniform over {16, 64, 256, 1024, 4096},
    steps log-uniform in [steps_lo, steps_hi]: the engine (continuous batching under an
    HBM budget) against serving the same requests one at a time in arrival order.
    Over several ranks, each request is routed on arrival to the rank with the least
    pair work assigned so far; every rank runs its own engine on its share."""
    from paper_1004_1932_b300 import partition
    full = inputs.request_trace(n_req, rate, steps_lo=steps_lo, steps_hi=steps_hi)
    route = partition.route_stream([partition.pair_work(S, n) for _, S, n, _ in full], ws)
    trace = [t for t, r in zip(full, route) if r == rank]
    susp = {rid: inputs.make_suspension(S, seed=1000 + rid, density=0.002) for _, S, _, rid in trace}
    eng = dbs.Engine(hbm_budget_bytes=budget, block_steps=block)
    t0 = time.perf_counter()
    ids, sub_t, done = {}, {}, {}
    k = 0
    while len(done) < len(trace):
        now = time.perf_counter() - t0
        while k < len(trace) and trace[k][0] <= now:
            arr, S, n, rid = trace[k]
            ids[rid] = eng.submit_inputs(susp[rid], n)
            sub_t[rid] = (arr, time.perf_counter() - t0)
            k += 1
        a, q = eng.tick()
        for rid, eid in ids.items():
            if rid in done:
                continue
            st, _, lat = eng.poll(eid)
            if st in (dbs.REQ_DONE, dbs.REQ_FAILED, dbs.REQ_CANCELLED):
                arr, sub = sub_t[rid]
                done[rid] = (st, (sub - arr) + lat)
        if a == 0 and q == 0 and k < len(trace):
            time.sleep(max(0.0, trace[k][0] - (time.perf_counter() - t0)))
    makespan = reduce_max(time.perf_counter() - t0, dev)
    eng_host = eng.stats()
    eng.close()
    lat = sorted(_gather_lists([v[1] for v in done.values() if v[0] == dbs.REQ_DONE], ws))
    total_steps = sum(n for _, _, n, _ in full)
    # one at a time in arrival order (grid path), measured run times, simulated queueing
    t_free, lat_seq, busy = 0.0, [], 0.0
    for arr, S, n, rid in trace:
        with dbs.Suspension.from_inputs(susp[rid], precision="fp32c") as h:
            h.sync()
            ts = time.perf_counter()
            h.step(n)
            h.positions()
            run = time.perf_counter() - ts
        start = max(arr, t_free)
        t_free = start + run
        busy += run
        lat_seq.append(t_free - arr)
    lat_seq = sorted(_gather_lists(lat_seq, ws))
    t_free, busy = reduce_max(t_free, dev), reduce_max(busy, dev)
    # the same, each request on its fastest single-system path (cooperative for S <= 4096)
    t_free_c, lat_c, busy_c = 0.0, [], 0.0
    for arr, S, n, rid in trace:
        with dbs.Suspension.from_inputs(susp[rid], precision="fp32c") as h:
            if S <= 4096:
                h.set_path("coop")
            h.sync()
            ts = time.perf_counter()
            h.step(n)
            h.positions()
            run = time.perf_counter() - ts
        start = max(arr, t_free_c)
        t_free_c = start + run
        busy_c += run
        lat_c.append(t_free_c - arr)
    lat_c = sorted(_gather_lists(lat_c, ws))
    t_free_c, busy_c = reduce_max(t_free_c, dev), reduce_max(busy_c, dev)
    q = lambda v, p: v[min(len(v) - 1, int(round(p * (len(v) - 1))))]
    return {"trace": f"{n_req} requests, Poisson {rate:g}/s (seed 0), S in {{16,64,256,1024,4096}}, "
                     f"steps log-uniform [{steps_lo:g}, {steps_hi:g}], HBM budget {budget >> 30} GB, "
                     f"block {block} steps",
            "ranks": ws, "routing": "least assigned pair work, on arrival" if ws > 1 else None,
            "completed": len(lat),
            "engine": {"makespan_s": makespan, "system_steps_per_s": total_steps / makespan,
                       "p50_latency_s": q(lat, 0.5), "p99_latency_s": q(lat, 0.99),
                       "host": eng_host},
            "one_at_a_time": {"path": "grid", "makespan_s": t_free, "system_steps_per_s": total_steps / busy,
                              "p50_latency_s": q(lat_seq, 0.5), "p99_latency_s": q(lat_seq, 0.99)},
            "one_at_a_time_fastest_path": {"path": "cooperative (S <= 4096), grid", "makespan_s": t_free_c,
                                           "system_steps_per_s": total_steps / busy_c,
                                           "p50_latency_s": q(lat_c, 0.5), "p99_latency_s": q(lat_c, 0.99)}}


def sharded_measure(dbs, inputs, torch, stream, ws, rank, dev, S=32768, steps=10):
    """One suspension of S dumbbells split by target rows over all ranks (NCCL
    all-gather of the packed records after every evaluation): strong scaling."""
    from paper_1004_1932_b300 import shard
    s = inputs.paper_scale(S, seed=0)
    sh = shard.Shard(s, ws, rank, precision="fp32c", stream=stream, device=dev.index)
    ex = shard.GroupExchange()
    shard.step([sh], 2, ex)
    torch.cuda.synchronize(dev)
    torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    shard.step([sh], steps, ex)
    e1.record(stream)
    e1.synchronize()
    el = reduce_max(e0.elapsed_time(e1) / 1e3, dev)
    rows = (sh.row0, sh.row1)
    sh.close()
    N = 2 * S
    return {"workload": f"one suspension S={S} (N={N}) density 0.002, RPY, FP32C, split by target rows "
                        f"over {ws} ranks (all-gather of the packed records after every evaluation)",
            "scaling": "strong", "heun_steps": steps, "ms_per_heun_step": 1e3 * el / steps,
            "pairs_per_s": 2 * N * (N - 1) * steps / el, "rank0_rows": rows}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1004_1932_b300 import inputs
    S, N = args.S, 2 * args.S
    cores = os.cpu_count()
    oracle.set_threads(cores)
    s = inputs.paper_scale(S, seed=0, mobility=args.mobility)
    mob = oracle.RPY if args.mobility == "rpy" else oracle.OSEEN
    per_step = 10   # Heun steps of the oracle per reference step (bounded sample of a period)
    x = s.x0
    n = 0
    for _ in range(args.warmup):
        x = oracle.heun(x, n, per_step, dt=s.dt, mobility=mob, **s.phys())
        n += per_step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = oracle.heun(x, n, per_step, dt=s.dt, mobility=mob, **s.phys())
        n += per_step
    el = time.perf_counter() - t0
    value = 2 * N * (N - 1) * per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(S, args.mobility, "n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step = {per_step} Heun steps of the S={S} "
                                       f"suspension on the FP64 C oracle"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1004_1932_b300 import dbs, inputs
    dbs.load()

    S, N = args.S, 2 * args.S
    s = inputs.paper_scale(S, seed=rank_seed(rank), mobility=args.mobility)
    stream = torch.cuda.Stream(device=dev)
    T = 2 * math.pi / s.omega
    m = STEPS_PER_PERIOD
    dt_sa = T / SA_STEPS_PER_PERIOD
    assert abs(m * s.dt - T) < 1e-12
    total_periods = args.warmup + args.steps + 2
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size
    flush_buf = torch.empty(int(2 * l2_bytes) // 4, dtype=torch.float32, device=dev)

    from paper_1004_1932_b300 import autotune
    if args.path == "auto":
        probe = dbs.Suspension.from_inputs(s, precision="fp32c", stream=stream, device=local)
        path_choice = autotune.choose_path(probe)
        probe.close()
    else:
        path_choice = {"path": args.path, "s_per_step": None}

    # the averaged model is independent of the microscopic one until the comparison:
    # it runs on a stream of its own, on the SMs the microscopic model leaves free
    sa_stream = torch.cuda.Stream(device=dev)

    def make():
        h = dbs.Suspension.from_inputs(s, precision="fp32c", stream=stream, device=local)
        h.set_path(path_choice["path"])
        sa = dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega,
                                dt=dt_sa, precision="fp32c", stream=sa_stream, device=local)
        # overlapped with the microscopic model on the SMs it leaves free: one launch
        # per evaluation (a cooperative launch needs all its CTAs resident at once)
        sa.set_path("grid")
        h.enable_period_average(m, max_periods=total_periods)
        return h, sa

    sa_ref = torch.empty((S, 3), dtype=torch.float64, device=dev)
    errs = []

    def period(h, sa, k, res=None):
        """One benchmark step: stroke period k of the full hot path (the microscopic
        model on `stream`, the averaged model forked onto `sa_stream` and joined back
        before the comparison).  With `res` (a device tensor, one row of 4 doubles
        per period) the comparison's values stay on the device and the host does
        not wait for them; without, they are read back to the host."""
        fork = torch.cuda.Event()
        fork.record(stream)
        h.step(m)
        sa_stream.wait_event(fork)
        sa.step(SA_STEPS_PER_PERIOD // 2 if k == 0 else SA_STEPS_PER_PERIOD)
        if k == 1:
            sa.copy_centres(sa_ref)
        join = torch.cuda.Event()
        join.record(sa_stream)
        stream.wait_event(join)
        if k >= 2:
            args_ = (S, h.period_average_device(1), h.period_average_device(k), sa_ref.data_ptr(),
                     sa.centres_device())
            if res is not None:
                dbs.pair_distance_error_async(*args_, res[k], stream=stream)
            else:
                errs.append(dbs.pair_distance_error(*args_, stream=stream))

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    # ---- device-resident run -------------------------------------------------
    h, sa = make()
    res_dev = torch.zeros((args.warmup + args.steps, 4), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            period(h, sa, k, res_dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = Clocks(cvd.split(",")[local] if cvd else str(local))
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush_buf.zero_()                       # L2 flush between timed iterations
            ev0[i].record(stream)
            period(h, sa, args.warmup + i, res_dev)
            ev1[i].record(stream)
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    h.sync()
    ms = reduce_max(ms, dev)
    pairs_per_step = 2 * N * (N - 1) * m
    value = ws * pairs_per_step * args.steps / (ms / 1e3)
    # our kernels per benchmark step: the microscopic model (grid: 2 per Heun step;
    # cluster and cooperative: one launch per <= 1024 steps), the clock-ring refills
    # (one per 2048 steps), the stroke-averaged model (2 per step) and the comparison
    model_launches = 2 * m if path_choice["path"] == "grid" else -(-m // 1024)
    launches_per_step = model_launches + 2 * SA_STEPS_PER_PERIOD + 1
    ring_fills = -(-(m * args.steps) // 2048)

    # ---- live per-launch duration of the dominant kernel (CUDA events, its stream) ----
    props = torch.cuda.get_device_properties(dev)
    mhz_max = clk.get("sm_max_mhz") or 2032.0
    peak = _fp32_peak_tflops(props.multi_processor_count, mhz_max)
    if path_choice["path"] in ("cluster", "coop"):
        # one launch advances 1024 Heun steps (2048 pair sums)
        kname = ("resident_kernel (cluster-resident pair sums + Heun, 1024 steps per launch)"
                 if path_choice["path"] == "cluster" else
                 "flow_kernel (cooperative dataflow: each CTA owns T dumbbells and sums them "
                 "over all records, fused Heun epilogue, tagged point-to-point exchange of "
                 "records, 1024 steps per launch)")
        kev0, kev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = []
        for _ in range(3):
            h.sync()
            kev0.record(stream)
            h.step(1024)
            kev1.record(stream)
            kev1.synchronize()
            launches.append(kev0.elapsed_time(kev1))
        mean_ms = sum(launches) / len(launches)
        flops_launch = 2 * 1024 * N * (N - 1) * FLOPS_PER_PAIR[args.mobility]
    else:
        kname = "eval_kernel (pair sum + fused Heun epilogue)"
        mean_ms = h.step_timed(200)
        flops_launch = N * (N - 1) * FLOPS_PER_PAIR[args.mobility]
    achieved = flops_launch / (mean_ms / 1e3) / 1e12
    rows = res_dev.cpu().numpy()
    last_err = ({"max": float(rows[-1, 0]), "rms": float(rows[-1, 1]), "ref_rms": float(rows[-1, 2]),
                 "pairs": int(rows[-1, 3])} if args.warmup + args.steps > 2 else None)
    h.close()
    sa.close()

    # ---- the same kernel on large single systems: FP32C vs all-FP64 ----------------
    # (S = 2048, 8192, 32768; one pair-sum launch of the grid path, CUDA events),
    # and 100 Heun steps of each size on its autotuned stepping path (FP32C)
    large = None
    if not args.no_large:
        from paper_1004_1932_b300 import autotune
        fp64_peak = props.multi_processor_count * 2 * 2 * mhz_max * 1e6 / 1e12   # 2 DFMA/clk/SM
        sweep = []
        for Sl in (2048, 8192, 32768):
            sl = inputs.paper_scale(Sl, seed=rank, mobility=args.mobility)
            Nl = 2 * Sl
            row = {"S": Sl, "N": Nl}
            for prec, reps in (("fp32c", 6), ("fp64", 2)):
                hl = dbs.Suspension.from_inputs(sl, precision=prec, stream=stream, device=local)
                hl.step_timed(1)
                ms_l = hl.step_timed(reps)
                hl.close()
                ach_l = Nl * (Nl - 1) * FLOPS_PER_PAIR[args.mobility] / (ms_l / 1e3) / 1e12
                row[prec] = {"launch_ms": ms_l, "pairs_per_s": Nl * (Nl - 1) / (ms_l / 1e3),
                             "achieved_tflops": ach_l,
                             "frac_of_fp32_peak": ach_l / peak,
                             **({"frac_of_fp64_peak": ach_l / fp64_peak} if prec == "fp64" else {})}
            hl = dbs.Suspension.from_inputs(sl, precision="fp32c", stream=stream, device=local)
            choice = autotune.choose_path(hl, steps=100)
            hl.step(8)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            hl.step(100)
            ev1.record(stream)
            ev1.synchronize()
            hl.close()
            el = ev0.elapsed_time(ev1) / 1e3 / 100
            ach_s = 2 * Nl * (Nl - 1) * FLOPS_PER_PAIR[args.mobility] / el / 1e12
            row["fp32c_stepping"] = {"path": choice["path"], "heun_steps": 100, "us_per_heun_step": el * 1e6,
                                     "pairs_per_s": 2 * Nl * (Nl - 1) / el, "achieved_tflops": ach_s,
                                     "frac_of_fp32_peak": ach_s / peak}
            sweep.append(row)
        top = sweep[-1]["fp32c"]
        large = {"workload": "single suspension S=32768 (N=65536), density 0.002, same kernel",
                 "launch_ms": top["launch_ms"], "achieved": top["achieved_tflops"], "peak": peak,
                 "unit": "TFLOP/s", "frac": top["frac_of_fp32_peak"], "pairs_per_s": top["pairs_per_s"],
                 "size_sweep": sweep,
                 "fp64_peak_tflops": fp64_peak,
                 "note": "one pair-sum launch (grid path); FP64 peak = SMs x 2 DFMA/clk x 2 x max clock; "
                         "fp32c_stepping: 100 Heun steps (two evaluations each, fused epilogues) on the "
                         "autotuned path, CUDA events"}

    # ---- end to end through the C-ABI with host buffers -----------------------
    # ---- the stroke-averaged kernel on its own (CUDA events on its stream) --------
    sa_kernel = None
    if not args.no_large:
        sa_kernel = {"kernel": "stroke-averaged pair sums with the Heun update: sa_flow_kernel "
                               "(cooperative, one launch per 1024 averaged steps; FP32C, S <= 4096) "
                               "or sa_eval_kernel (2 launches per averaged step)",
                     "flops_per_pair": SA_FLOPS_PER_PAIR, "peak": peak, "unit": "TFLOP/s", "sizes": []}

        def sa_time(ss, reps, path):
            sst = torch.cuda.Stream(device=dev)
            with dbs.StrokeAveraged(ss.R0, ss.N0, ss.phi, ss.lam, a=ss.a, ell=ss.ell, omega=ss.omega,
                                    dt=0.1, precision="fp32c", stream=sst) as sk:
                if path:
                    sk.set_path(path)
                used = sk.get_path()[0]
                sk.step(4)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(sst)
                sk.step(reps)
                e1.record(sst)
                e1.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps, used

        for Ss, reps in ((S, 1000), (8192, 20)):
            ss = inputs.paper_scale(Ss, seed=rank, mobility=args.mobility)
            el, used = sa_time(ss, reps, None)
            ach = 2 * Ss * (Ss - 1) * SA_FLOPS_PER_PAIR / el / 1e12
            row = {"S": Ss, "path": used, "us_per_step": el * 1e6, "achieved": ach, "frac": ach / peak}
            if used == "coop":
                row["grid_path_us_per_step"] = sa_time(ss, 200, "grid")[0] * 1e6
            sa_kernel["sizes"].append(row)

    e2e = None
    if not args.no_e2e:
        x_host = torch.from_numpy(s.x0.copy()).pin_memory()
        out_host = torch.empty((N, 3), dtype=torch.float64).pin_memory()
        h2d = x_host.numel() * 8
        d2h = out_host.numel() * 8 + 4 * 8
        h, sa = make()
        errs.clear()
        res_e2e = torch.zeros((args.warmup + args.steps, 4), dtype=torch.float64, device=dev)
        cmp_host = torch.zeros((args.warmup + args.steps, 4), dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            for k in range(args.warmup):
                period(h, sa, k, res_e2e)
        barrier()
        t0 = time.perf_counter()
        xs = x_host.numpy()
        for i in range(args.steps):
            k = args.warmup + i
            n_now = k * m
            h.set_state(xs, n_now)                 # host -> device: this step's input state
            with torch.cuda.stream(stream):
                period(h, sa, k, res_e2e)
                cmp_host[k].copy_(res_e2e[k], non_blocking=True)   # device -> host: the comparison
            out_host.numpy()[:] = h.positions()     # device -> host: the step's positions (synchronises)
            xs = out_host.numpy()
        barrier()
        el = reduce_max(time.perf_counter() - t0, dev)
        e2e = {"value": ws * pairs_per_step * args.steps / el, "unit": "pairs/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        h.close()
        sa.close()

    # ---- the stroke-averaged model at the nominal and at the measured amplitude ---
    # (outside the timed region): the k0 = 1 springs lag the rest length, so the
    # dumbbells stroke with a smaller amplitude lambda_eff than the nominal lambda
    sa_cmp = {"timed_loop": last_err}
    if not args.no_large:
        from paper_1004_1932_b300 import experiments
        periods = args.warmup + args.steps
        eff = experiments.effective_amplitude(s, path=path_choice["path"])
        lr_ratio, lr_lag = experiments.linear_response_ratio(s)
        sa_cmp.update({
            "periods": periods,
            "nominal": experiments.sa_comparison(s, periods=periods, path=path_choice["path"]),
            "lambda_eff": experiments.sa_comparison(s, periods=periods, lam=eff["lam_eff"],
                                                    path=path_choice["path"]),
            "lambda_eff_over_lambda": eff["ratio_mean"], "lag_deg": math.degrees(eff["lag_mean"]),
            "linear_response": {"ratio": lr_ratio, "lag_deg": math.degrees(lr_lag)},
            "note": "pair-distance error of the stroke-averaged model (Eqs. (9a)-(9e)) against the "
                    "period-averaged centres, with the nominal stroke amplitudes and with each "
                    "dumbbell's measured amplitude (first Fourier coefficient of its length over one "
                    "period after a settling period)"})

    # ---- the small FP64 suspension (S = 16, Oseen, all-FP64) on the GPU -----------
    small = None
    if not args.no_large:
        s1 = inputs.small_fp64_oseen(0)
        N1 = 2 * s1.S
        per_path = {}
        for p1 in ("grid", "coop"):
            with dbs.Suspension.from_inputs(s1, precision="fp64", stream=stream, device=local) as h1:
                h1.set_path(p1)
                h1.step(64)
                h1.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h1.step(1000)
                e1.record(stream)
                e1.synchronize()
                per_path[p1] = e0.elapsed_time(e1) / 1e3 / 1000
        el1 = per_path["coop"]
        small = {"workload": "S=16 (N=32), cube side 8, Oseen, all-FP64, dt=1e-3, 1000 Heun steps "
                             "(cooperative FP64 path: one launch, 16 CTAs of one dumbbell)",
                 "us_per_heun_step": el1 * 1e6, "heun_steps_per_s": 1.0 / el1,
                 "pairs_per_s": 2 * N1 * (N1 - 1) / el1,
                 "us_per_heun_step_by_path": {k: v * 1e6 for k, v in per_path.items()},
                 "bound": "FP64 latency (each FP64 instruction holds its SM sub-partition 64 cycles) "
                          "and the record exchange; the grid path: 2 pair-sum launches per Heun step"}

    ensemble = None if args.no_ensemble else ensemble_measure(dbs, inputs, torch, stream, ws=ws,
                                                              rank=rank, dev=dev)
    sharded = sharded_measure(dbs, inputs, torch, stream, ws, rank, dev) if ws > 1 else None
    serving = None if args.no_serving else serving_measure(dbs, inputs, ws=ws, rank=rank, dev=dev)

    if rank != 0:
        return
    cpu = _cpu_baseline(S, args.mobility, args.cpu_sample_steps) if ws == 1 else None
    if cpu is not None and not args.no_cpu_sweep:
        cpu["sweep"] = _cpu_sweep(args.mobility)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_note": "FP32 pair math with two-sum compensation; FP64 positions, clock and Heun update",
        "data": "synthetic (seeded random suspension, no dataset)",
        "config": _workload_config(S, args.mobility, "flushed between timed steps (2x L2 write)"),
        "heun_steps_per_s": ws * m * args.steps / (ms / 1e3),
        "path": path_choice,
        "roofline": {"bound": "alu", "kernel": kname,
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((path_choice["path"], S, args.mobility)),
                     "traffic_source": TRAFFIC_SOURCE,
                     "launch_ms": mean_ms, "flops_per_launch": flops_launch,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                   f"{mhz_max:.0f} MHz (max SM clock)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps + ring_fills,
        "clocks": clk,
        "sa_comparison": sa_cmp,
        "small_system": small,
        "sharded_large_system": sharded,
        "large_system_kernel": large,
        "ensemble": ensemble,
        "serving": serving,
        "sa_kernel": sa_kernel,
    }
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
