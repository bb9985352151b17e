"""Autotuner of the Voigt kernel's launch configuration.

The knobs are those of rox_set_launch_config (include/rox.h): warps per CTA (4 or 8), CTAs per
SM of the persistent grid, and how many rounds of warps' worth of work items are split into
parts at the end of a launch. None of them changes a result (the summation order of every span
is fixed), so the tuner only times: for each candidate it runs the caller's step once untimed,
then `reps` times between CUDA events, and keeps the fastest median. Results are cached in a
JSON file keyed by (GPU name, SM count, workload class); `apply` sets the cached configuration
for a workload class, or the library's default where the cache has no entry.
"""
import json
import os
import statistics

import torch

from . import _binding as rb

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")

# (warps per CTA, CTAs per SM (0: as many as fit), split rounds)
CANDIDATES = [(8, 0, 1), (8, 0, 2), (8, 2, 1), (8, 1, 1), (4, 0, 1), (4, 0, 2), (4, 4, 1), (4, 3, 1)]


def key(workload_class, device=None):
    p = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
    return "%s|%d SMs|%s" % (p.name, p.multi_processor_count, workload_class)


def _as_dict(c):
    return {"warps_per_cta": c[0], "ctas_per_sm": c[1], "split_rounds": c[2]}


def sweep(step, candidates=CANDIDATES, reps=2):
    """Times `step()` (one launch sequence on the current stream) under every candidate; returns
    [(candidate dict, median ms)] in candidate order and leaves the default configuration set."""
    out = []
    try:
        for c in candidates:
            rb.rox_set_launch_config(*c)
            step()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                step()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            out.append((_as_dict(c), statistics.median(ms)))
    finally:
        rb.rox_reset_launch_config()
    return out


def load(path=CACHE):
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save(workload_class, results, path=CACHE, note=""):
    """Records a sweep's results and its best configuration under key(workload_class)."""
    cache = load(path)
    best, best_ms = min(results, key=lambda r: r[1])
    default_ms = next((ms for c, ms in results if c == _as_dict(CANDIDATES[0])), None)
    cache[key(workload_class)] = {"best": best, "best_ms": best_ms, "default_ms": default_ms, "note": note,
                                  "results": [{"config": c, "ms": ms} for c, ms in results]}
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return best


def apply(workload_class, path=CACHE):
    """Sets the cached best configuration of workload_class on this GPU (the default if there is
    none); returns (configuration dict, whether it came from the cache)."""
    entry = load(path).get(key(workload_class))
    if entry is None:
        rb.rox_reset_launch_config()
        return rb.rox_get_launch_config(), False
    b = entry["best"]
    rb.rox_set_launch_config(b["warps_per_cta"], b["ctas_per_sm"], b["split_rounds"])
    return rb.rox_get_launch_config(), True
