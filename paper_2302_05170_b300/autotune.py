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


def tune_slots(run, key, candidates=(2, 3, 4, 5), reps=3, use_cache=True):
    """run(): one call of the workload on the current stream.  Returns (best_slots, timings_ms)."""
    import torch
    import paper_2302_05170_b300 as sl

    full_key = "%s|%s" % (torch.cuda.get_device_name(), key)
    cache = _load()
    if use_cache and full_key in cache:
        sl.tc_set_slots(cache[full_key]["slots"])
        return cache[full_key]["slots"], cache[full_key]["ms"]
    times = {}
    for s in candidates:
        sl.tc_set_slots(s)
        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run()
        b.record()
        b.synchronize()
        times[str(s)] = a.elapsed_time(b) / reps
    best = int(min(times, key=times.get))
    sl.tc_set_slots(best)
    cache[full_key] = {"slots": best, "ms": times}
    try:
        with open(CACHE + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(CACHE + ".tmp", CACHE)
    except OSError:
        pass
    return best, times
