"""Launch-shape autotuner for the batched walk.

Times trevr_compute_flux_batched for every candidate (work-item size in sinks,
block size, walk variant) on the caller's own batch, keeps the fastest, and caches the choice
in a JSON file keyed by GPU name and a size class of the batch (log2 of its
total sink count and of its tree count), so later batches of the same shape
skip the search. The traversal stacks need no tuning: they hold 64 entries,
more than the deepest possible cell (63 cuts of the 63-bit key).
"""
from __future__ import annotations

import json
import math
import os

import torch

ITEM_SIZES = (32, 64, 128, 256)
BLOCK_SIZES = (64, 128, 256)
VARIANTS = (1, 2, 3)  # per-lane walk, warp-shared walk, warp-shared with merged rays
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "trevr_gb300", "autotune.json")


def size_class(batch) -> str:
    return f"sinks2^{int(math.log2(max(1, batch.n_sinks)))}_trees2^{int(math.log2(len(batch.trees)))}"


def _key(batch) -> str:
    return f"{torch.cuda.get_device_name()}|{size_class(batch)}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(batch, theta, tau_ref, cache_path=DEFAULT_CACHE, repeats=2, use_cache=True):
    """Return {'sinks_per_warp', 'block_size', 'walk_variant', 'ms', 'table'} for the batch."""
    key = _key(batch)
    cache = _load(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True)
    table = {}
    best = None
    stream = torch.cuda.current_stream()
    for var in VARIANTS:
        for item in ITEM_SIZES:
            for bs in BLOCK_SIZES:
                shape = dict(sinks_per_warp=item, block_size=bs, walk_variant=var)
                batch.run(theta, tau_ref, **shape)  # warm up, build the work items
                ts = []
                for _ in range(repeats):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    batch.run(theta, tau_ref, **shape)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                t = min(ts)
                table[f"v{var}_{item}x{bs}"] = t
                if best is None or t < best[3]:
                    best = (item, bs, var, t)
    res = {"sinks_per_warp": best[0], "block_size": best[1], "walk_variant": best[2],
           "ms": best[3], "table": table}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache = _load(cache_path)
            cache[key] = res
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(res, cached=False)
