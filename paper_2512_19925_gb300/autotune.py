"""Autotuner for the batched engine: tile size and event budget.

A batch's results do not depend on its tuning (the tile size and the event
budget only reorder integer tally additions and requeue tracks), so the
trial steps are ordinary steps of the run: each candidate runs one or more
real steps, is scored by particle-segments per second, and the best one is
kept and cached as JSON under a signature of the workload (number of
problems, total particles and cells, precision, GPU name).
"""
from __future__ import annotations

import json
import os
import time

DEFAULT_CANDIDATES = ((2048, 64), (4096, 64), (8192, 64), (16384, 64), (4096, 16), (4096, 256))


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "hww_gb300", "autotune.json")


def signature(batch, gpu_name: str = "") -> str:
    wls = batch.workloads
    n_part = sum(int(w["particles_per_step"]) for w in wls)
    n_cells = sum(len(w["edges"]) - 1 for w in wls)
    prec = wls[0].get("precision", "fp64") if wls else "fp64"
    return "P%d_N%d_I%d_%s_%s" % (len(wls), n_part, n_cells, prec, gpu_name.replace(" ", "_"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def cached(batch, gpu_name: str = "", path: str | None = None):
    """The cached (tile, emax) for this workload, or None."""
    entry = _load(path or default_cache_path()).get(signature(batch, gpu_name))
    return (int(entry["tile"]), int(entry["emax"])) if entry else None


def autotune_batch(batch, candidates=DEFAULT_CANDIDATES, steps_per_trial=1, gpu_name: str = "",
                   path: str | None = None, sync=None, settle: int = 0):
    """Try each (tile, emax) on real steps, keep the fastest, cache it.

    `sync` is a callable that waits for the GPU (for example
    torch.cuda.synchronize); the trial steps are part of the run.  `settle`
    ordinary steps run first (on a cache miss): in a run's first steps the
    members' census banks and record queues are still growing to the run's
    demand, and a step in which any member overflows tracks the whole batch
    again with larger buffers, which would count against whichever
    candidate ran it."""
    path = path or default_cache_path()
    hit = cached(batch, gpu_name, path)
    if hit:
        batch.set_tuning(*hit)
        return hit, {}
    for _ in range(int(settle)):
        batch.run_step()
    rates = {}
    for tile, emax in candidates:
        batch.set_tuning(tile, emax)
        if sync:
            sync()
        t0 = time.perf_counter()
        segs = 0
        for _ in range(steps_per_trial):
            segs += batch.run_step()["segments"]
        if sync:
            sync()
        rates[(tile, emax)] = segs / max(time.perf_counter() - t0, 1e-9)
    best = max(rates, key=rates.get)
    batch.set_tuning(*best)
    data = _load(path)
    data[signature(batch, gpu_name)] = {"tile": best[0], "emax": best[1],
                                       "rates": {"%d/%d" % k: v for k, v in rates.items()}}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return best, rates
