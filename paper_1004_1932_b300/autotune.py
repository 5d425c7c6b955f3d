"""Autotuners: the j-split (chunks) of the grid path's pair-sum launch, the
stepping path of a suspension (with the cooperative path's split), and the
cluster sizes of an ensemble, each chosen by timing candidates on the device.

The kernel's work units are (i-block of dumbbells) x (j-chunk); how many
chunks fill the 148 SMs best depends on S, precision, mobility and occupancy
in ways a closed-form rule only approximates (see ``choose_launch`` in the
library).  ``tune()`` times the library's own choice and a candidate set
around whole waves of the persistent grid with ``dbs_step_timed`` (CUDA events
around every launch) and keeps the fastest.  Results are cached per device
name, precision, mobility and S in a JSON file.
"""
from __future__ import annotations

import json
import os

from . import dbs

# the cache lives in the user's cache directory (never inside the package);
# DBS_TUNE_CACHE names another file
CACHE = os.environ.get("DBS_TUNE_CACHE",
                       os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")),
                                    "paper_1004_1932_b300", "tuned_chunks.json"))


def _key(h: "dbs.Suspension", device_name: str, precision: str, mobility: str) -> str:
    return f"{device_name}|{precision}|{mobility}|S={h.S}"


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def candidates(S: int, launch: dict, sms: int = 148) -> list[int]:
    """Chunk counts worth timing: the built-in choice, powers of two, and the
    splits that make the unit count a small multiple of the resident grid."""
    bt = launch["bt"]
    iblocks = (S + bt - 1) // bt
    cmax = max(1, S // 8)
    out = {launch["chunks"], 1}
    c = 2
    while c <= cmax:
        out.add(c)
        c *= 2
    grid = max(launch["grid"], 1)
    for waves in (1, 2, 3, 4, 6, 8):
        c = (waves * grid) // iblocks
        for d in (-1, 0, 1):
            if 1 <= c + d <= cmax:
                out.add(c + d)
    return sorted(x for x in out if 1 <= x <= cmax)


def tune(h: "dbs.Suspension", *, device_name: str = "cuda", precision: str = "fp32c",
         mobility: str = "rpy", reps: int | None = None, use_cache: bool = True,
         write_cache: bool = True) -> dict:
    """Choose and apply the fastest chunk count for handle ``h``.

    Advances the suspension by the timing steps (the caller restores its state
    if that matters, e.g. with get_state/set_state)."""
    key = _key(h, device_name, precision, mobility)
    cache = _load() if use_cache else {}
    if key in cache:
        h.set_chunks(int(cache[key]["chunks"]))
        return {"chunks": int(cache[key]["chunks"]), "cached": True}
    base = h.get_launch()
    if reps is None:
        reps = max(4, min(200, int(2e9 / max(1, h.N) ** 2)))
    results = {}
    for c in candidates(h.S, base):
        h.set_chunks(c)
        h.step_timed(2)
        results[c] = h.step_timed(reps)
    best = min(results, key=results.get)
    h.set_chunks(best)
    entry = {"chunks": best, "ms_per_launch": results[best],
             "builtin": {"chunks": base["chunks"], "ms_per_launch": results.get(base["chunks"])}}
    if write_cache:
        cache = _load()
        cache[key] = entry
        try:
            os.makedirs(os.path.dirname(CACHE) or ".", exist_ok=True)
            with open(CACHE + ".tmp", "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(CACHE + ".tmp", CACHE)
        except OSError:
            pass
    return {**entry, "cached": False, "timed": results}


def choose_path(h: "dbs.Suspension", steps: int = 1024) -> dict:
    """Time ``steps`` Heun steps on the grid, cluster and cooperative paths (where the
    suspension fits it), the cooperative one at its built-in split and at 4, 8 and 16
    dumbbells per CTA, and keep the fastest.  The suspension's state is restored to
    where it started, so the choice does not change the trajectory."""
    import time
    x0, n0 = h.get_state()
    timings = {}
    coop_split = {}

    def _time():
        h.step(64)
        h.sync()
        t = time.perf_counter()
        h.step(steps)
        h.sync()
        el = (time.perf_counter() - t) / steps
        h.set_state(x0, n0)
        return el

    for path in ("grid", "cluster", "coop"):
        try:
            h.set_path(path)
        except dbs.DbsError:
            continue
        if path != "coop":
            timings[path] = _time()
            continue
        # cooperative path: also the split (dumbbells per CTA) around the built-in one
        for req in (0, 4, 8, 16):
            h.set_chunks(req)
            T = h.get_launch()["bt"]
            if T not in coop_split:
                coop_split[T] = _time()
        timings[path] = min(coop_split.values())
    best = min(timings, key=timings.get)
    h.set_path(best)
    out = {"path": best, "s_per_step": timings}
    if best == "coop":
        T = min(coop_split, key=coop_split.get)
        h.set_chunks(T)
        out["coop_dumbbells_per_cta"] = T
        out["coop_split_s_per_step"] = coop_split
    h.set_state(x0, n0)
    return out


def _pow2_at_least(v: int) -> int:
    g = 1
    while g < v:
        g *= 2
    return g


def tune_ensemble(ens: "dbs.Ensemble", members, steps: int = 128) -> dict:
    """Cluster sizes (the tile shape of the resident kernel: CTAs per member)
    for an ensemble, chosen by timing.  Candidates: the built-in balance rule
    (G proportional to each member's S^2), the rule scaled by 1/2 and by 2, and
    the smallest clusters that fit.  Members' states are restored after every
    trial, so the choice does not change the trajectories."""
    import time
    states = [h.get_state() for h in members]
    ens.set_clusters(None)
    base = ens.get_clusters()
    gmin = [_pow2_at_least(max(1, -(-h.S // 512))) for h in members]
    cands = {"balance": None,
             "half": [max(m, g // 2) for g, m in zip(base, gmin)],
             "double": [min(16, 2 * g) for g in base],
             "smallest": gmin}
    timings = {}
    for name, G in cands.items():
        try:
            ens.set_clusters(G)
            ens.step(8)
            ens.sync()
            t = time.perf_counter()
            ens.step(steps)
            ens.sync()
            timings[name] = (time.perf_counter() - t) / steps
        except dbs.DbsError:
            pass
        for h, (x, n) in zip(members, states):
            h.set_state(x, n)
    best = min(timings, key=timings.get)
    ens.set_clusters(cands[best])
    return {"choice": best, "s_per_step": timings,
            "clusters": {str(g): c for g, c in sorted(_count(ens.get_clusters()).items())}}


def _count(G):
    out = {}
    for g in G:
        out[g] = out.get(g, 0) + 1
    return out
