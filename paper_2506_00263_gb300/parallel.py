"""Multi-GPU helpers: histories shard by contiguous index ranges.

Every history draws its random numbers from a Philox stream keyed by its own
index, so a fixed-source run of N histories split into contiguous shards
[first, first + count) gives exactly the histories of the single run.  The
only exchange is the final tally combination, done in fixed rank order so
the result does not depend on arrival order.  No collective touches the
transport loop itself.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous (first, count) of rank `rank` among `world` ranks."""
    base, extra = divmod(int(n), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def combine_means(parts: Sequence[Tuple[int, np.ndarray]]) -> np.ndarray:
    """Per-source-particle means of shards -> mean of the whole run, summed in
    the given (rank) order."""
    total = sum(int(c) for c, _ in parts)
    acc = None
    for c, m in parts:
        v = np.asarray(m, dtype=np.float64) * float(c)
        acc = v.copy() if acc is None else acc + v
    return acc / float(total) if total else acc


def gather_objects(obj, group=None) -> List:
    """All-gather of a picklable object over torch.distributed (rank order)."""
    import torch.distributed as dist
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def reduce_timing(seconds: float, events: float, histories: float, device=None):
    """Whole-job timing across ranks: the slowest rank's time, summed work."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    w = torch.tensor([events, histories], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0]), float(w[1])


def run_fixed_source_sharded(spec, opts, tally_ids=(0, 2), group=None):
    """Fixed-source run of opts.n_histories split over the ranks of `group`
    (one GPU per rank).  Returns the combined tallies on every rank."""
    import dataclasses

    import torch.distributed as dist

    from . import binding as tb
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, count = shard(opts.n_histories, rank, world)
    local = dataclasses.replace(opts, n_histories=count, first_history=opts.first_history + first)
    prob = tb.Problem(spec)
    stats = prob.run_fixed_source(local)
    mine = {t: prob.tally(t) for t in tally_ids}
    prob.close()
    parts = gather_objects((count, mine, int(stats["events"])), group)
    out = {t: combine_means([(c, d[t]) for c, d, _ in parts]) for t in tally_ids}
    out["events"] = sum(e for _, _, e in parts)
    return out
