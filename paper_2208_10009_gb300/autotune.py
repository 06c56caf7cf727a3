"""Autotuner for the batched refinement kernel's launch shape.

The batched kernel's speed depends on the block size, on how many lanes cooperate on one
path (1, 8, 16 or 32) and on how many blocks stay resident per SM; the best choice depends on
the number of paths, their orders and iteration counts.  `tune_batch_refine` times every
combination on the caller's own paths (refinement rewrites the paths in place, so the
caller supplies `relaunch`, which must regenerate the rough paths before each trial) and
returns the fastest.  Results are kept per process, keyed by device, K, iteration cap and
the path count rounded up to a power of two; set SBR_AUTOTUNE_CACHE to a JSON file path to
persist them.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

import torch

_CACHE: dict[str, dict] = {}


def _key(ctx, K, max_iters, target, npaths):
    bucket = 1 << max(0, int(npaths - 1).bit_length())
    return f"{torch.cuda.get_device_name(ctx.device)}|K{K}|it{max_iters}|tg{target:.3g}|p{bucket}"


def _load_file():
    path = os.environ.get("SBR_AUTOTUNE_CACHE")
    if path and os.path.exists(path):
        try:
            _CACHE.update(json.load(open(path)))
        except Exception:
            pass


def _save_file():
    path = os.environ.get("SBR_AUTOTUNE_CACHE")
    if path:
        with open(path, "w") as f:
            json.dump(_CACHE, f, indent=1)


def tune_batch_refine(ctx, scene, paths, relaunch, max_iters: int, K: int, target: float = 0.0, trials: int = 3,
                      blocks=(64, 128, 256), lanes=(1, 8, 16, 32), per_sm=(0, 4, 2), force: bool = False) -> dict:
    """Return {"block_threads", "lanes_per_path", "blocks_per_sm", "ms", "table"} for the
    fastest batched-refinement launch shape on these paths."""
    _load_file()
    relaunch()
    n = ctx.paths_count(paths)
    key = _key(ctx, K, max_iters, target, n)
    if key in _CACHE and not force:
        return _CACHE[key]
    stream = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    table = []
    for b, l, s in itertools.product(blocks, lanes, per_sm):
        times = []
        for _ in range(trials):
            relaunch()
            e0.record(stream)
            ctx.batch_refine(scene, paths, max_iters, K, target=target, block_threads=b, lanes_per_path=l,
                             blocks_per_sm=s)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        table.append({"block_threads": b, "lanes_per_path": l, "blocks_per_sm": s, "ms": statistics.median(times)})
    best = min(table, key=lambda r: r["ms"])
    out = dict(best, paths=n, table=table)
    _CACHE[key] = out
    _save_file()
    return out
