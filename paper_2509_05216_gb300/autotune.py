"""Project-written autotuner for the rasterizer's launch options.

For a workload key (Gaussian count, resolution mix, views per batch, GPU name)
it times the real training step under every candidate value of each option
(CUDA events on the current stream, after a warm-up step) and keeps the
fastest.  Results are cached as JSON so a later run with the same key skips
the search.
"""
from __future__ import annotations

import json
import os

import torch

from . import gs

CANDIDATES = {gs.GS_OPT_RASTER_FWD: [2, 8, 4, 1], gs.GS_OPT_RASTER_BWD: [2, 4, 8, 1],
              gs.GS_OPT_BWD_DIRECT: [2, 0, 4, 8], gs.GS_OPT_SORT_ITEMS: [16, 12, 20, 24],
              gs.GS_OPT_TILE_ORDER: [0, 1]}


def workload_key(n, cams, batch):
    res = sorted({(c["width"], c["height"]) for c in cams})
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "n%d|res%s|b%d|%s" % (n, ",".join("%dx%d" % r for r in res), batch, name)


def _cache_path():
    return os.environ.get("GS_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                             "gs_gb300_autotune.json"))


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(db):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_step(step, reps=3):
    """Shortest of `reps` single-step times (ms) after one warm-up step: the
    minimum is the least disturbed by clock or power-state drift."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        ev0.record()
        step()
        ev1.record()
        torch.cuda.synchronize()
        best = min(best, ev0.elapsed_time(ev1))
    return best


def report(key):
    """The timings (ms per step, "option=value") of the cached search for
    `key`, or None."""
    entry = _load().get(key)
    return entry.get("ms") if entry else None


def tune(ctxs, step, key, candidates=None, reps=3, rounds=2, use_cache=True):
    """Pick option values for `ctxs` (contexts the step uses) by timing `step`,
    one option at a time (the others at their current values).  Each
    candidate is timed in `rounds` interleaved rounds and keeps its best time.

    Returns {option: value} and leaves the chosen values set."""
    candidates = candidates or CANDIDATES
    db = _load() if use_cache else {}
    if key in db:
        chosen = {int(k): v for k, v in db[key]["options"].items()}
    else:
        chosen, report = {}, {}
        for opt, values in candidates.items():
            times = {v: float("inf") for v in values}
            for _ in range(rounds):
                for v in values:
                    for c in ctxs:
                        c.gs_set_option(opt, v)
                    times[v] = min(times[v], time_step(step, reps))
            best = min(values, key=lambda v: times[v])
            for v in values:
                report["%d=%d" % (opt, v)] = round(times[v], 3)
            for c in ctxs:
                c.gs_set_option(opt, best)
            chosen[opt] = best
        db[key] = {"options": {str(k): v for k, v in chosen.items()}, "ms": report}
        if use_cache:
            _save(db)
    for opt, v in chosen.items():
        for c in ctxs:
            c.gs_set_option(opt, v)
    return chosen
