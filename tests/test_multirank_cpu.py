"""The N > 1 path on CPU: two gloo ranks shard the histories by contiguous
index ranges, each computes its shard, and the tallies combine in rank order
to exactly the single-run result.  The per-rank computation here is the
oracle (the GPU library is exercised by the virtual-rank GPU test); what is
tested is the sharding, the exchange and the timing reduction that the
multi-GPU bench uses."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2506_00263_gb300 import parallel


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_path):
    import torch.distributed as dist

    import oracle
    from paper_2506_00263_gb300 import inputs, parallel as par
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = inputs.c5g7_lattice()
    first, count = par.shard(n, rank, world)
    r = oracle.run_fixed_source(p, count, seed=5, id_offset=first)
    parts = par.gather_objects((count, r["mesh"], r["scalars"], r["log_n"], r["log_type"]))
    t, ev, hi = par.reduce_timing(0.5 + rank, float(r["events_by_type"][1:].sum()), float(count))
    if rank == 0:
        mesh = par.combine_means([(c, m) for c, m, _, _, _ in parts])
        scal = par.combine_means([(c, s) for c, _, s, _, _ in parts])
        log_n = np.concatenate([ln for _, _, _, ln, _ in parts])
        log_t = np.concatenate([lt for _, _, _, _, lt in parts])
        np.savez(out_path, mesh=mesh, scal=scal, log_n=log_n, log_t=log_t, t=t, ev=ev, hi=hi)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 1000, 1_000_003):
        for w in (1, 2, 3, 8):
            parts = [parallel.shard(n, r, w) for r in range(w)]
            assert sum(c for _, c in parts) == n
            nxt = 0
            for f, c in parts:
                assert f == nxt
                nxt = f + c


def test_two_gloo_ranks_reproduce_single_run(tmp_path):
    import oracle
    from paper_2506_00263_gb300 import inputs
    n, world = 6001, 2
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(world, _free_port(), n, out), nprocs=world, join=True, start_method="spawn")
    res = np.load(out)
    ref = oracle.run_fixed_source(inputs.c5g7_lattice(), n, seed=5)
    assert np.array_equal(res["log_n"], ref["log_n"]) and np.array_equal(res["log_t"], ref["log_type"])
    assert np.allclose(res["mesh"], ref["mesh"], rtol=1e-12, atol=1e-15)
    assert np.allclose(res["scal"], ref["scalars"], rtol=1e-12)
    assert float(res["t"]) == 1.5                     # slowest rank's time
    assert float(res["hi"]) == n
    assert float(res["ev"]) == float(ref["events_by_type"][1:].sum())
