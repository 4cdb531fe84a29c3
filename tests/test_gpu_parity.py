"""GPU vs. oracle parity through the C ABI (bit-exact integer outcomes,
1e-10 relative FP64 tallies), for both remapping schemes and both task
decompositions."""
import functools

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu

SCHEMES = [(tb.SCHEME_STACK, tb.DECOMP_MONO), (tb.SCHEME_STACK, tb.DECOMP_SPLIT),
           (tb.SCHEME_STACK, tb.DECOMP_SPLIT_LOOKUP),
           (tb.SCHEME_ASYNC, tb.DECOMP_MONO), (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT),
           (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT_LOOKUP), (tb.SCHEME_ASYNC, tb.DECOMP_STREAM)]
IDS = ["stack-mono", "stack-split", "stack-lookup", "async-mono", "async-split", "async-lookup", "async-stream"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _problem(name):
    if name == "cube":
        return inputs.cube_one_group()
    if name == "lattice":
        return inputs.c5g7_lattice()
    if name == "ce":
        return inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=100)
    if name == "ce_full":
        return inputs.ce_pin_cell()
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def _oracle_fixed(name, n, seed=1, max_events=0):
    r = oracle.run_fixed_source(_problem(name), n, seed=seed, max_events=max_events)
    assert r["status"] == 0
    return r


def _gpu_fixed(name, n, scheme, decomp, seed=1, **kw):
    prob = tb.Problem(_problem(name))
    opts = tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=decomp, want_event_log=True, **kw)
    st = prob.run_fixed_source(opts)
    out = {"stats": st, "log": prob.event_log(n) if n else None, "mesh": prob.tally(tb.TALLY_MESH),
           "energy": prob.tally(tb.TALLY_ENERGY), "scalars": prob.tally(tb.TALLY_SCALARS)}
    prob.close()
    return out


def _compare_fixed(g, o, n):
    assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]))
    assert np.array_equal(g["stats"]["final_by_type"], o["final_by_type"])
    assert np.array_equal(g["stats"]["events_by_type"], o["events_by_type"])
    assert_tally_close(g["mesh"], o["mesh"], "mesh")
    assert_tally_close(g["energy"], o["energy"], "energy")
    assert_tally_close(g["scalars"], o["scalars"], "scalars")
    assert g["stats"]["histories"] == n


@pytest.mark.parametrize("scheme,decomp", SCHEMES, ids=IDS)
def test_cube_parity(scheme, decomp):
    n = 100_003
    _compare_fixed(_gpu_fixed("cube", n, scheme, decomp), _oracle_fixed("cube", n), n)


@pytest.mark.parametrize("scheme,decomp", SCHEMES, ids=IDS)
def test_lattice_fixed_source_parity(scheme, decomp):
    n = 20_011
    _compare_fixed(_gpu_fixed("lattice", n, scheme, decomp), _oracle_fixed("lattice", n), n)


@pytest.mark.parametrize("scheme,decomp", SCHEMES, ids=IDS)
def test_ce_pin_cell_parity(scheme, decomp):
    n = 3_001
    _compare_fixed(_gpu_fixed("ce", n, scheme, decomp), _oracle_fixed("ce", n), n)


@pytest.mark.parametrize("scheme,decomp", SCHEMES, ids=IDS)
def test_power_iteration_parity(scheme, decomp):
    p = _problem("lattice")
    nper, ni, na = 3000, 2, 3
    o = oracle.power_iteration(p, nper, ni, na, seed=3, log_batch=ni + na - 1)
    assert o["status"] == 0
    prob = tb.Problem(p)
    g = prob.power_iteration(nper, ni, na, tb.RunOpts(seed=3, scheme=scheme, decomposition=decomp,
                                                      want_event_log=True))
    # per-batch sizes and k are integer-driven and bit-identical
    assert np.array_equal(g["n_source"], o["n_source"])
    assert np.array_equal(g["k_batch"], o["k_batch"])
    assert_tally_close(g["ktl_batch"], o["ktl_batch"], "ktl")
    assert abs(g["k_mean"] - o["k_mean"]) <= 1e-12 * abs(o["k_mean"])
    assert_tally_close(prob.tally(tb.TALLY_MESH), o["mesh_mean"], "mesh mean")
    sd = prob.tally(tb.TALLY_MESH, stddev=True)
    assert np.allclose(sd, o["mesh_std"], rtol=1e-6, atol=1e-12 * o["mesh_std"].max())
    assert_tally_close(prob.tally(tb.TALLY_SCALARS), o["scalars_mean"], "scalars mean")
    nlast = int(o["n_source"][-1])
    assert_logs_equal(prob.event_log(nlast), (o["log_n"], o["log_cell"], o["log_type"]), "last batch")
    assert np.array_equal(g["final_by_type"], o["final_by_type"])
    prob.close()


# ----------------------------------- the monolithic loop with deferred collisions
# (4 or more events between remaps: pending collisions batched in the warp,
# sources refilled in the loop, the batch tail consolidated; the benchmark
# runs 512, the CE benchmark 64)

@pytest.mark.parametrize("remap", [4, 64, 512])
@pytest.mark.parametrize("name,n", [("cube", 100_003), ("lattice", 20_011), ("ce", 3_001)])
def test_deferred_collision_loop_parity(name, n, remap):
    g = _gpu_fixed(name, n, tb.SCHEME_ASYNC, tb.DECOMP_MONO, remap_every=remap)
    _compare_fixed(g, _oracle_fixed(name, n), n)


def test_deferred_collision_loop_spills_and_tiny_stash():
    """Forced spills and a small stash with 512 events between remaps: the
    tail hands particles between warps and blocks, never changing a history."""
    n = 20_011
    o = _oracle_fixed("lattice", n)
    for kw in (dict(remap_every=512, spill_threshold=-32, queue_capacity=64 * 32),
               dict(remap_every=512, stash_slots=288, blocks_per_sm=1),
               dict(remap_every=64, stash_slots=288, spill_threshold=-32, queue_capacity=4096)):
        g = _gpu_fixed("lattice", n, tb.SCHEME_ASYNC, tb.DECOMP_MONO, **kw)
        _compare_fixed(g, o, n)


@pytest.mark.parametrize("remap", [64, 512])
def test_deferred_collision_loop_power_iteration(remap):
    p = _problem("lattice")
    nper, ni, na = 3000, 2, 3
    o = oracle.power_iteration(p, nper, ni, na, seed=3, log_batch=ni + na - 1)
    prob = tb.Problem(p)
    g = prob.power_iteration(nper, ni, na, tb.RunOpts(seed=3, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO,
                                                      remap_every=remap, want_event_log=True))
    assert np.array_equal(g["n_source"], o["n_source"])
    assert np.array_equal(g["k_batch"], o["k_batch"])
    assert_tally_close(prob.tally(tb.TALLY_MESH), o["mesh_mean"], "mesh mean")
    nlast = int(o["n_source"][-1])
    assert_logs_equal(prob.event_log(nlast), (o["log_n"], o["log_cell"], o["log_type"]), "last batch")
    prob.close()


# --------------------------------------------------------------- edge cases

@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000 + 7])
def test_tiny_and_ragged_counts(n):
    for scheme, decomp in SCHEMES:
        g = _gpu_fixed("lattice", n, scheme, decomp)
        if n == 0:
            assert g["stats"]["histories"] == 0 and g["stats"]["events"] == 0
            assert np.all(g["mesh"] == 0)
            continue
        _compare_fixed(g, _oracle_fixed("lattice", n), n)


def test_event_cap_maxev():
    n = 5000
    o = _oracle_fixed("lattice", n, max_events=4)
    assert o["final_by_type"][tb.EV_MAXEV] > 0
    for scheme, decomp in SCHEMES:
        _compare_fixed(_gpu_fixed("lattice", n, scheme, decomp, max_events=4), o, n)


def test_scheduler_invariance_tuning():
    """Remap frequency, tiny stacks, tiny stashes and forced spills change the
    schedule, never the histories."""
    n = 20_011
    o = _oracle_fixed("lattice", n)
    variants = [
        (tb.SCHEME_STACK, tb.DECOMP_MONO, dict(remap_every=5)),
        (tb.SCHEME_STACK, tb.DECOMP_MONO, dict(queue_capacity=64, blocks_per_sm=1)),
        (tb.SCHEME_STACK, tb.DECOMP_SPLIT, dict(queue_capacity=96)),
        (tb.SCHEME_ASYNC, tb.DECOMP_MONO, dict(remap_every=3, stash_slots=288, blocks_per_sm=1)),
        (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT, dict(stash_slots=288, spill_threshold=-32, queue_capacity=4096)),
        (tb.SCHEME_ASYNC, tb.DECOMP_MONO, dict(spill_threshold=-32, queue_capacity=64 * 32)),
        (tb.SCHEME_STACK, tb.DECOMP_SPLIT_LOOKUP, dict(queue_capacity=96)),
        (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT_LOOKUP, dict(stash_slots=288, spill_threshold=-32, queue_capacity=4096)),
        (tb.SCHEME_ASYNC, tb.DECOMP_STREAM, dict(remap_every=5)),
        (tb.SCHEME_ASYNC, tb.DECOMP_STREAM, dict(remap_every=2, stash_slots=288, spill_threshold=-32,
                                                 queue_capacity=4096)),
    ]
    for scheme, decomp, kw in variants:
        g = _gpu_fixed("lattice", n, scheme, decomp, **kw)
        _compare_fixed(g, o, n)
        if kw.get("spill_threshold", 0) < 0:
            assert g["stats"]["spills"] > 0 and g["stats"]["refills"] > 0, g["stats"]


def test_full_size_sampled_histories():
    """Lattice at 1e6 histories with the decomposed asynchronous scheme and
    the monolithic stack scheme: 3000 sampled histories recomputed one by one
    by the oracle, plus conservation and tally-sum checks.  (The benchmark's
    own configuration is compared in full in test_gpu_fullsize.py.)"""
    n = 1_000_000
    p = _problem("lattice")
    rng = np.random.default_rng(0)
    ids = np.unique(rng.integers(0, n, 3000))
    ref = [oracle.run_fixed_source(p, 1, seed=1, id_offset=int(i)) for i in ids]
    ref_log = tuple(np.array([r[k][0] for r in ref]) for k in ("log_n", "log_cell", "log_type"))
    for scheme, decomp in [(tb.SCHEME_ASYNC, tb.DECOMP_SPLIT), (tb.SCHEME_STACK, tb.DECOMP_MONO)]:
        g = _gpu_fixed("lattice", n, scheme, decomp)
        assert_logs_equal(tuple(a[ids] for a in g["log"]), ref_log, "sampled")
        fb = g["stats"]["final_by_type"]
        assert int(fb.sum()) == n and int(fb[tb.EV_ABSORB] + fb[tb.EV_LEAK]) == n
        assert int(g["log"][0].astype(np.int64).sum()) == int(g["stats"]["events_by_type"].sum())
        assert abs(g["mesh"].sum() - g["scalars"][0]) <= 1e-10 * g["scalars"][0]


def test_ce_full_size_sampled_histories():
    n = 200_000
    p = _problem("ce_full")
    rng = np.random.default_rng(1)
    ids = np.unique(rng.integers(0, n, 400))
    ref = [oracle.run_fixed_source(p, 1, seed=1, id_offset=int(i)) for i in ids]
    ref_log = tuple(np.array([r[k][0] for r in ref]) for k in ("log_n", "log_cell", "log_type"))
    for decomp in (tb.DECOMP_SPLIT, tb.DECOMP_SPLIT_LOOKUP):
        g = _gpu_fixed("ce_full", n, tb.SCHEME_ASYNC, decomp)
        assert_logs_equal(tuple(a[ids] for a in g["log"]), ref_log, "sampled CE")
        assert abs(g["energy"].sum() - g["scalars"][0]) <= 1e-10 * g["scalars"][0]


# --------------------------------------------------------------- error paths

def test_timeout_is_reported_and_problem_stays_usable():
    prob = tb.Problem(_problem("lattice"))
    with pytest.raises(tb.TransportError) as e:
        prob.run_fixed_source(tb.RunOpts(n_histories=200_000, scheme=tb.SCHEME_ASYNC,
                                         decomposition=tb.DECOMP_SPLIT, max_spin=1))
    assert e.value.status == tb.TR_ERR_TIMEOUT
    st = prob.run_fixed_source(tb.RunOpts(n_histories=1000, scheme=tb.SCHEME_ASYNC))
    assert st["histories"] == 1000
    prob.close()


def test_bank_overflow_is_capacity_error():
    prob = tb.Problem(_problem("lattice"))
    with pytest.raises(tb.TransportError) as e:
        prob.power_iteration(2000, 1, 2, tb.RunOpts(seed=1), bank_capacity_factor=0.01)
    assert e.value.status == tb.TR_ERR_CAPACITY
    prob.close()


def test_invalid_options_rejected():
    prob = tb.Problem(_problem("cube"))
    for bad in (dict(scheme=7), dict(decomposition=5), dict(decomposition=tb.DECOMP_SPLIT, remap_every=2),
                dict(decomposition=tb.DECOMP_SPLIT_LOOKUP, remap_every=2),
                dict(decomposition=tb.DECOMP_STREAM, scheme=tb.SCHEME_STACK), dict(n_histories=1 << 33)):
        kw = dict(n_histories=10)
        kw.update(bad)
        with pytest.raises(tb.TransportError) as e:
            prob.run_fixed_source(tb.RunOpts(**kw))
        assert e.value.status == tb.TR_ERR_INVALID
    with pytest.raises(tb.TransportError) as e:
        tb.lib()
        prob.tally(7)
    prob.close()


def test_invalid_energy_edges_rejected():
    """The energy tally's bin search compares bit patterns, so its edges must
    be ascending and non-negative; problem creation refuses others."""
    spec = inputs.ce_pin_cell(n_points=2000, n_res=10, n_ebins=4)
    for edges in (np.array([-1.0, 1.0, 10.0, 100.0, 1e3]), np.array([1.0, 10.0, 5.0, 100.0, 1e3])):
        with pytest.raises(tb.TransportError) as e:
            tb.Problem(spec.replace(energy_edges=edges))
        assert e.value.status == tb.TR_ERR_INVALID
    ok = tb.Problem(spec.replace(energy_edges=np.array([0.0, 1.0, 10.0, 100.0, 2e7])))
    ok.close()


def test_virtual_ranks_sum_equals_single_run():
    """Three contiguous shards (first_history) run separately and combined in
    rank order reproduce the single run: the multi-GPU replica/shard path
    emulated on one GPU, one shard after another."""
    from paper_2506_00263_gb300 import parallel
    n, world = 50_021, 3
    p = _problem("lattice")
    whole = _gpu_fixed("lattice", n, tb.SCHEME_ASYNC, tb.DECOMP_SPLIT)
    parts, logs = [], []
    for r in range(world):
        first, count = parallel.shard(n, r, world)
        g = _gpu_fixed("lattice", count, tb.SCHEME_STACK, tb.DECOMP_MONO, first_history=first)
        parts.append((count, g["mesh"], g["scalars"]))
        logs.append(g["log"])
    for k in range(3):
        assert np.array_equal(np.concatenate([l[k] for l in logs]), whole["log"][k])
    assert_tally_close(parallel.combine_means([(c, m) for c, m, _ in parts]), whole["mesh"], "sharded mesh")
    assert_tally_close(parallel.combine_means([(c, s) for c, _, s in parts]), whole["scalars"], "sharded scalars")
    # and against the oracle's shard of the middle rank
    first, count = parallel.shard(n, 1, world)
    o = oracle.run_fixed_source(p, count, seed=1, id_offset=first)
    assert_logs_equal(logs[1], (o["log_n"], o["log_cell"], o["log_type"]), "middle shard")
