"""tr_run_batched: many independent multigroup box problems in one persistent
launch.  Each problem's counts and event log must equal, bit for bit, its own
single-problem run with random-stream tag problem_tag ^ i (and the oracle's),
its tallies within the parity tolerance; the captured graph must replay to
the same result, and autotuned settings must not change the result."""
import functools

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu

TAG = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _boxes(n=24):
    # small members of the batched workload: 1..20^3 voxels, 100..20000 histories
    return inputs.batched_boxes(n_problems=n, seed=7, max_vox=20, max_hist=20_000, min_hist=100)


def _read(prob, n):
    return {"mesh": prob.tally(tb.TALLY_MESH), "energy": prob.tally(tb.TALLY_ENERGY),
            "scalars": prob.tally(tb.TALLY_SCALARS), "log": prob.event_log(n) if n else None}


def _opts(**kw):
    base = dict(seed=11, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO, want_event_log=True,
                problem_tag=TAG, blocks_per_sm=1, stash_slots=512, remap_every=1)
    base.update(kw)
    return tb.RunOpts(**base)


def _check_against_single(probs, hist, got, stats, decomp):
    for i, (pd, n) in enumerate(zip(probs, hist)):
        single = tb.Problem(pd)
        st = single.run_fixed_source(tb.RunOpts(n_histories=n, seed=11, scheme=tb.SCHEME_ASYNC,
                                                decomposition=decomp, want_event_log=True,
                                                problem_tag=TAG ^ i))
        ref = _read(single, n)
        single.close()
        what = f"problem {i}"
        assert_logs_equal(got[i]["log"], ref["log"], what)
        assert np.array_equal(stats[i]["events_by_type"], st["events_by_type"]), what
        assert np.array_equal(stats[i]["final_by_type"], st["final_by_type"]), what
        for k in ("mesh", "energy", "scalars"):
            assert_tally_close(got[i][k], ref[k], f"{what} {k}")
            # the same contributions reduced the same way: the same bits
            assert np.array_equal(np.asarray(got[i][k]).view(np.uint64), np.asarray(ref[k]).view(np.uint64)), \
                f"{what} {k} bits"


@pytest.mark.parametrize("decomp", [tb.DECOMP_MONO, tb.DECOMP_SPLIT], ids=["mono", "split"])
def test_batched_equals_single_runs(decomp):
    probs, hist = _boxes()
    gp = [tb.Problem(p) for p in probs]
    stats = tb.run_batched(gp, hist, _opts(decomposition=decomp))
    got = [_read(p, n) for p, n in zip(gp, hist)]
    _check_against_single(probs, hist, got, stats, decomp)
    for p in gp:
        p.close()


def test_batched_members_match_oracle():
    probs, hist = _boxes()
    gp = [tb.Problem(p) for p in probs]
    stats = tb.run_batched(gp, hist, _opts())
    for i in (0, 3, len(probs) - 1):
        o = oracle.run_fixed_source(probs[i], hist[i], seed=11, tag=TAG ^ i)
        assert o["status"] == 0
        g = _read(gp[i], hist[i])
        assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]), f"problem {i}")
        assert np.array_equal(stats[i]["final_by_type"], o["final_by_type"])
        for k in ("mesh", "energy", "scalars"):
            assert_tally_close(g[k], o[k], f"problem {i} {k}")
    for p in gp:
        p.close()


def test_graph_replay_and_autotune():
    probs, hist = _boxes(12)
    gp = [tb.Problem(p) for p in probs]
    first = tb.run_batched(gp, hist, _opts())
    a = [_read(p, n) for p, n in zip(gp, hist)]
    # same batch again: replay of the captured graph, same launches, same results
    c0 = tb.kernel_launch_count()
    again = tb.run_batched(gp, hist, _opts())
    launches = tb.kernel_launch_count() - c0
    assert launches == 4          # the transport launch, the two-kernel per-history reduction, the normalisation
    b = [_read(p, n) for p, n in zip(gp, hist)]
    for i in range(len(gp)):
        assert_logs_equal(b[i]["log"], a[i]["log"], f"replay {i}")
        assert np.array_equal(again[i]["events_by_type"], first[i]["events_by_type"])
        for k in ("mesh", "energy", "scalars"):
            assert np.array_equal(b[i][k].view(np.uint64), a[i][k].view(np.uint64)), f"replay {i} {k}"
    # autotuned: every tuning field left at 0
    tuned = tb.run_batched(gp, hist, _opts(blocks_per_sm=0, stash_slots=0, remap_every=0))
    bps, slots, remap = tuned[0]["used"]
    assert bps >= 1 and slots >= 288 and remap >= 1
    assert all(t["used"] == tuned[0]["used"] for t in tuned)
    c = [_read(p, n) for p, n in zip(gp, hist)]
    for i in range(len(gp)):
        assert_logs_equal(c[i]["log"], a[i]["log"], f"tuned {i}")
        for k in ("mesh", "energy", "scalars"):
            assert np.array_equal(c[i][k].view(np.uint64), a[i][k].view(np.uint64)), f"tuned {i} {k}"
    for p in gp:
        p.close()


def test_batched_edge_cases():
    probs, hist = _boxes(4)
    gp = [tb.Problem(p) for p in probs]
    # a member with zero histories and a single-history member
    h = [0, 1, hist[2], 7]
    stats = tb.run_batched(gp, h, _opts())
    assert stats[0]["histories"] == 0 and stats[0]["events"] == 0
    assert not np.any(gp[0].tally(tb.TALLY_MESH))
    for i in (1, 2, 3):
        o = oracle.run_fixed_source(probs[i], h[i], seed=11, tag=TAG ^ i)
        g = _read(gp[i], h[i])
        assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]), f"problem {i}")
        assert_tally_close(g["mesh"], o["mesh"], f"problem {i} mesh")
    # refused on the host: duplicates, the stack scheme, a continuous-energy member
    for bad, opts in (([gp[0], gp[0]], _opts()), (gp[:2], _opts(scheme=tb.SCHEME_STACK))):
        with pytest.raises(tb.TransportError) as e:
            tb.run_batched(bad, [10] * len(bad), opts)
        assert e.value.status == tb.TR_ERR_INVALID
    ce = tb.Problem(inputs.ce_pin_cell(n_points=2000, n_res=10, n_ebins=10))
    with pytest.raises(tb.TransportError) as e:
        tb.run_batched([gp[1], ce], [10, 10], _opts())
    assert e.value.status == tb.TR_ERR_INVALID
    ce.close()
    for p in gp:
        p.close()
