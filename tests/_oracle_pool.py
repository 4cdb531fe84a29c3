"""The oracle over contiguous history shards in spawned worker processes.

Histories are keyed by their own index, so shards [first, first + count) run
separately give exactly the histories of one run; the per-shard means are
combined in shard order.  Workers are started with the spawn method (a fork
after the parent has touched CUDA can hang), and each rebuilds its problem
from the named input recipe, so no array crosses the process boundary on the
way in.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def _problem(recipe):
    from paper_2506_00263_gb300 import inputs
    name, kw = recipe
    return getattr(inputs, name)(**dict(kw))


def _shard(args):
    recipe, first, count, seed, max_events = args
    import oracle
    r = oracle.run_fixed_source(_problem(recipe), count, seed=seed, id_offset=first, max_events=max_events)
    return first, count, r


def fixed_source(recipe, n, seed=1, max_events=0, workers=None):
    """oracle.run_fixed_source over n histories, computed in shards.  recipe:
    (name of an inputs constructor, tuple of keyword items)."""
    from paper_2506_00263_gb300 import parallel
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    shards = [parallel.shard(n, r, workers) for r in range(workers)]
    jobs = [(recipe, f, c, seed, max_events) for f, c in shards if c > 0]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=ctx) as ex:
        parts = sorted(ex.map(_shard, jobs), key=lambda t: t[0])
    out = {"status": max(int(r["status"]) for _, _, r in parts)}
    for k in ("log_n", "log_cell", "log_type"):
        out[k] = np.concatenate([r[k] for _, _, r in parts])
    for k in ("mesh", "energy", "scalars", "time"):
        out[k] = parallel.combine_means([(c, r[k]) for _, c, r in parts])
    for k in ("events_by_type", "final_by_type"):
        out[k] = np.sum([r[k] for _, _, r in parts], axis=0).astype(np.uint64)
    return out


def _sens_shard(args):
    recipe, first, count, seed, g_mesh, g_scal = args
    import oracle
    r = oracle.sensitivities(_problem(recipe), count, g_mesh=g_mesh, g_scal=g_scal, seed=seed, id_offset=first)
    return first, count, r


def sensitivities(recipe, n, g_mesh=None, g_scal=None, seed=1, workers=None):
    """oracle.sensitivities over n histories, computed in shards (means per
    source particle combined in shard order)."""
    from paper_2506_00263_gb300 import parallel
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    shards = [parallel.shard(n, r, workers) for r in range(workers)]
    jobs = [(recipe, f, c, seed, g_mesh, g_scal) for f, c in shards if c > 0]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=ctx) as ex:
        parts = sorted(ex.map(_sens_shard, jobs), key=lambda t: t[0])
    out = {"status": max(int(r["status"]) for _, _, r in parts)}
    for k in ("d_sigt", "d_sigs", "d_nusigf"):
        out[k] = parallel.combine_means([(c, r[k]) for _, c, r in parts])
    out["value"] = float(parallel.combine_means([(c, np.array([r["value"]])) for _, c, r in parts])[0])
    return out
