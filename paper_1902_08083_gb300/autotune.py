"""Launch-shape autotuners for the batched walk and the single-tree walk.

tune() times trevr_compute_flux_batched for every candidate (work-item size in
sinks, block size, walk variant) on the caller's own batch; tune_walk() times
trevr_compute_flux for every walk shape (walk variant, and sinks per warp for the
per-lane walk) on the caller's own tree. Each keeps the fastest and caches the
choice in a JSON file keyed by GPU name and a size class of the problem (log2 of
its sink count and of its tree or source count), so later problems of the same
shape skip the search. The traversal stacks need no tuning: they hold 64 entries,
more than the deepest possible cell (63 cuts of the 63-bit key), so a smaller
limit could only overflow.
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


# single-tree walk shapes: (walk variant, sinks per warp); the warp-shared walks
# (2, 3) take one sink per lane, the per-lane walk (1) a chunk of sinks per warp
WALK_SHAPES = ((3, 0), (2, 0), (1, 32), (1, 64), (1, 128))


def size_class(batch) -> str:
    return f"sinks2^{int(math.log2(max(1, batch.n_sinks)))}_trees2^{int(math.log2(len(batch.trees)))}"


def walk_size_class(n_sinks, n_src) -> str:
    return f"walk_sinks2^{int(math.log2(max(1, n_sinks)))}_src2^{int(math.log2(max(1, n_src)))}"


def _device_name() -> str:
    return torch.cuda.get_device_name()


def _key(batch) -> str:
    return f"{_device_name()}|{size_class(batch)}"


def _store(cache_path, key, res):
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache = _load(cache_path)
        cache[key] = res
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass


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
        _store(cache_path, key, res)
    return dict(res, cached=False)


def _time_walk(tree, theta, tau_ref, sink_idx, shape, repeats):
    """Device time (ms) of one trevr_compute_flux call in the given shape: the
    fastest of `repeats` calls after one warm-up, CUDA events on the current stream."""
    from . import trevr
    var, spw = shape
    stream = torch.cuda.current_stream()
    out = trevr.compute_flux(tree, theta, tau_ref, sink_idx=sink_idx, walk_variant=var,
                             sinks_per_warp=spw)
    ts = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        trevr.compute_flux(tree, theta, tau_ref, sink_idx=sink_idx, out=out, walk_variant=var,
                           sinks_per_warp=spw)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def tune_walk(tree, theta, tau_ref, sink_idx=None, cache_path=DEFAULT_CACHE, repeats=2,
              use_cache=True, shapes=WALK_SHAPES, timer=None):
    """Return {'walk_variant', 'sinks_per_warp', 'ms', 'table', 'cached'} for the flux
    walk on this tree (all its sinks, or the sinks in sink_idx). Pass the chosen
    fields to trevr.compute_flux as walk_variant= and sinks_per_warp=. `timer`
    replaces the timing call (tree, theta, tau_ref, sink_idx, shape, repeats) -> ms."""
    n = tree.n_gas if sink_idx is None else int(sink_idx.shape[0])
    key = f"{_device_name()}|{walk_size_class(n, tree.n_src)}"
    if use_cache:
        cache = _load(cache_path)
        if key in cache:
            return dict(cache[key], cached=True)
    timer = timer or _time_walk
    table = {}
    best = None
    for shape in shapes:
        t = float(timer(tree, theta, tau_ref, sink_idx, shape, repeats))
        table[f"v{shape[0]}_{shape[1]}"] = t
        if best is None or t < best[1]:
            best = (shape, t)
    res = {"walk_variant": best[0][0], "sinks_per_warp": best[0][1], "ms": best[1],
           "table": table}
    if use_cache:
        _store(cache_path, key, res)
    return dict(res, cached=False)
