"""Autotuner for the solver launch shapes (``ccd_tuning``).

Only speed depends on the tuning: the solvers reproduce Algorithm 2's
sequential order exactly for every valid launch shape, and the GPU tests
check that outputs are identical across tunings.  The tuner times a batch
under each candidate and keeps the fastest, caching the choice per GPU name
and workload tag in a JSON file (``$CCD_TUNING_CACHE`` or
``~/.cache/ccd_gb300/tuning.json``).

Tunables (see include/ccd.h):
  deep_threads         block size of the deep solver (128, 256 or 512)
  deep_slots           deep-solver blocks, i.e. queries with large frontiers
                       solved at once (0 = as many as fit: six per SM of 128
                       threads, three of 256, one of 512)
  small_blocks_per_sm  one-warp solver blocks per SM (its queue width)
  small_cap            frontier depth of a one-warp solver slot in boxes
  pool_cap             boxes per level a query may reach in the pooled solver
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Iterable

FIELDS = ("deep_threads", "deep_slots", "small_blocks_per_sm", "small_cap", "pool_cap")


def candidates(sms: int) -> list[dict]:
    out = []
    for dt, slots in ((128, 6 * sms), (256, 3 * sms), (256, 2 * sms), (512, sms)):
        for sb in (8, 16):
            for cap in (256, 1024):
                for pc in (64, 256):
                    out.append({"deep_threads": dt, "deep_slots": slots,
                                "small_blocks_per_sm": sb, "small_cap": cap, "pool_cap": pc})
    return out


def validate(t: dict) -> dict:
    t = {k: int(t.get(k, 0)) for k in FIELDS}
    if t["deep_threads"] not in (0, 128, 256, 512):
        raise ValueError("deep_threads must be 128, 256 or 512")
    if t["deep_slots"] < 0 or not 0 <= t["small_blocks_per_sm"] <= 32:
        raise ValueError("bad slot or block count")
    if t["small_cap"] and t["small_cap"] < 64:
        raise ValueError("small_cap must be >= 64")
    if t["pool_cap"] and not 32 <= t["pool_cap"] <= 4096:
        raise ValueError("pool_cap must be in 32..4096")
    return t


def cache_path() -> str:
    p = os.environ.get("CCD_TUNING_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "ccd_gb300", "tuning.json")


def _key(gpu: str, tag: str) -> str:
    return f"{gpu}|{tag}"


def load(gpu: str, tag: str, path: str | None = None) -> dict | None:
    path = path or cache_path()
    try:
        with open(path) as f:
            entry = json.load(f).get(_key(gpu, tag))
    except (OSError, ValueError):
        return None
    return validate(entry["tuning"]) if entry else None


def save(gpu: str, tag: str, tuning: dict, timings: list, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[_key(gpu, tag)] = {"tuning": validate(tuning), "timings": timings,
                            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(measure: Callable[[dict], float], cands: Iterable[dict], reps: int = 2):
    """Runs measure(tuning) -> seconds ``reps`` times per candidate and
    returns (best tuning, [(tuning, best seconds), ...])."""
    timings = []
    for c in cands:
        c = validate(c)
        t = min(measure(c) for _ in range(max(1, reps)))
        timings.append((c, t))
    best = min(timings, key=lambda x: x[1])[0]
    return best, timings


def get_or_tune(gpu: str, tag: str, measure: Callable[[dict], float], cands, reps: int = 2,
                path: str | None = None, retune: bool = False):
    """Cached tuning for (gpu, tag), tuning and caching it on a miss."""
    if not retune:
        hit = load(gpu, tag, path)
        if hit is not None:
            return hit, None
    best, timings = tune(measure, cands, reps)
    save(gpu, tag, best, [(t, s) for t, s in timings], path)
    return best, timings
