"""Ray-range sharding of one launch over several processes (one GPU each).

Rays are traced independently (§III.A, Fig. 4), so the ray ids of every transmitter are
split into contiguous ranges, one per rank, with the scene and receivers replicated.  The
one exchange step is double-count removal (§III.A, first path test): it needs every
record of a (Tx, Rx, face sequence) key, so the ranks all-gather their reception records
(position-independent 64-byte records naming lattice ray ids), and each rank then removes
double counts over the gathered set for the (Tx, Rx) pairs it owns.  Refinement, the
validity test and the outputs are per path, so each rank refines its own pairs' paths with
no further exchange.  The result is the single-launch result, split by pair owner.

This module only partitions and moves bytes; every step of the path runs in the CUDA
library (``records_dedup`` filters by owner on the device).
"""
from __future__ import annotations

import numpy as np
import torch

RECORD_BYTES = 64


def ray_range(n_rays: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous ray ids [begin, end) of `rank` among `world`: sizes differ by at most one
    and the ranges of ranks 0..world-1 tile [0, n_rays) in order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return n_rays * rank // world, n_rays * (rank + 1) // world


def pair_owner(tx, rx, nrx: int, world: int):
    """Rank owning the paths of pair (tx, rx): (tx * nrx + rx) mod world (the device rule of
    sbr_records_dedup)."""
    return (np.asarray(tx, np.int64) * nrx + np.asarray(rx, np.int64)) % world


def all_gather_records(local: torch.Tensor, count: int, group=None) -> tuple[torch.Tensor, int]:
    """All-gather variable-length record sets.  `local` holds at least `count` records of
    RECORD_BYTES bytes (uint8, on the device for NCCL, on the host for gloo).  Returns a
    uint8 tensor with every rank's records in rank order, and their total count."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = local.device
    n = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(max(counts), 1)
    send = torch.zeros(m * RECORD_BYTES, dtype=torch.uint8, device=dev)
    if count:
        send[: count * RECORD_BYTES] = local.reshape(-1)[: count * RECORD_BYTES]
    recv = [torch.empty(m * RECORD_BYTES, dtype=torch.uint8, device=dev) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    out = torch.cat([r[: c * RECORD_BYTES] for r, c in zip(recv, counts)])
    return out, sum(counts)


def sharded_launch(ctx, scene, tx, rxs, paths, n_div: int, max_order: int, rank: int, world: int, group=None,
                   buf: torch.Tensor | None = None, **launch_kw) -> dict:
    """One launch split over `world` ranks: trace this rank's ray range of every Tx (records
    only), all-gather the records, remove double counts over all of them for this rank's
    pairs.  `buf` (device uint8, record_cap * 64 bytes) receives the local records.
    Returns this rank's launch counters (segments of its own range)."""
    from . import _binding as B
    n_rays = B.load().sbr_num_rays_launcher(n_div, launch_kw.get("launcher", 0))
    ctx.launch(scene, tx, rxs, paths, n_div, max_order, ray_range=ray_range(n_rays, rank, world), records_only=True,
               **launch_kw)
    stats = ctx.launch_stats(paths)
    if buf is None:
        buf = torch.empty(paths.record_cap * RECORD_BYTES, dtype=torch.uint8, device=f"cuda:{ctx.device}")
    _, cnt = ctx.records(paths, buf)
    if world > 1:
        allrec, total = all_gather_records(buf, cnt, group)
    else:
        allrec, total = buf, cnt
    ctx.records_dedup(paths, allrec, total, rank, world)
    stats["gathered_records"] = total
    return stats
