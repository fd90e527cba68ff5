"""Autotuner for the BF16 tensor-core 7L sampler.

Times the caller's workload for every candidate number of 128-path tiles in
flight per CTA (sl_tc_set_slots) with CUDA events, keeps the fastest, and
caches the choice in a JSON file keyed by device name and workload shape.
"""
from __future__ import annotations

import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


CANDIDATES = ((4, 1), (3, 1), (2, 1), (4, 2), (2, 2))   # (slots, tiles per warpgroup)


def tune_slots(run, key, candidates=CANDIDATES, reps=3, use_cache=True):
    """run(): one call of the workload on the current stream.  Tries each
    (slots, tiles per warpgroup); returns (best, timings_ms)."""
    import torch
    import paper_2302_05170_b300 as sl

    full_key = "%s|%s" % (torch.cuda.get_device_name(), key)
    cache = _load()
    def apply(c):
        sl.tc_set_pipeline(1)          # every slot count is valid with one tile per warpgroup
        sl.tc_set_slots(c[0])
        sl.tc_set_pipeline(c[1])
    if use_cache and full_key in cache:
        apply(tuple(cache[full_key]["best"]))
        return tuple(cache[full_key]["best"]), cache[full_key]["ms"]
    times = {}
    for c in candidates:
        apply(c)
        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run()
        b.record()
        b.synchronize()
        times["%d/%d" % c] = a.elapsed_time(b) / reps
    best = min(candidates, key=lambda c: times["%d/%d" % c])
    apply(best)
    cache[full_key] = {"best": list(best), "ms": times}
    try:
        with open(CACHE + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(CACHE + ".tmp", CACHE)
    except OSError:
        pass
    return best, times
