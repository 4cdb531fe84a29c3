"""Full-size parity of the benchmark's own paths against the oracle.

The benchmark runs the asynchronous monolithic scheme with 512 events between
remaps on sources sampled ahead of the launch (the lattice), and 64 events
between remaps on the full continuous-energy grid.  At these sizes every
block's lanes refill from the source inside the loop and the batch tail
hands particles between warps, which the small parity cases never reach.
Here every history and every tally bin of the full-size runs is compared
with the oracle (computed over history shards on the host cores): per-history
event counts, final cells and final types bit-equal; tallies within 1e-10
relative (the floor of tests/_util.py)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests import _oracle_pool
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu

LATTICE = ("c5g7_lattice", ())
CE_FULL = ("ce_pin_cell", ())
CE_1E4_BINS = ("ce_pin_cell", (("n_ebins", 10_000),))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _spec(recipe):
    name, kw = recipe
    return getattr(inputs, name)(**dict(kw))


@functools.lru_cache(maxsize=None)
def _oracle(recipe, n, seed=1):
    r = _oracle_pool.fixed_source(recipe, n, seed=seed)
    assert r["status"] == 0
    return r


def _gpu(recipe, n, scheme, decomp, seed=1, **kw):
    prob = tb.Problem(_spec(recipe))
    st = prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=decomp,
                                          want_event_log=True, **kw))
    out = {"stats": st, "log": prob.event_log(n), "mesh": prob.tally(tb.TALLY_MESH),
           "energy": prob.tally(tb.TALLY_ENERGY), "scalars": prob.tally(tb.TALLY_SCALARS)}
    prob.close()
    return out


def _compare(g, o, n):
    assert g["stats"]["histories"] == n
    assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]), "full size")
    assert np.array_equal(g["stats"]["events_by_type"], o["events_by_type"])
    assert np.array_equal(g["stats"]["final_by_type"], o["final_by_type"])
    assert_tally_close(g["mesh"], o["mesh"], "mesh")
    assert_tally_close(g["energy"], o["energy"], "energy")
    assert_tally_close(g["scalars"], o["scalars"], "scalars")


def test_lattice_benchmark_path_full_size():
    """1e6 lattice histories, asynchronous monolithic, 512 events per remap,
    pre-sampled sources (the benchmark's kernel and launch configuration)."""
    n = 1_000_000
    g = _gpu(LATTICE, n, tb.SCHEME_ASYNC, tb.DECOMP_MONO, remap_every=512)
    _compare(g, _oracle(LATTICE, n), n)


def test_lattice_paper_setting_full_size():
    """The same histories at the paper's setting (one event per remap, whole
    events per pass) and with the stack-based scheme."""
    n = 1_000_000
    o = _oracle(LATTICE, n)
    for scheme, decomp, remap in ((tb.SCHEME_ASYNC, tb.DECOMP_MONO, 1), (tb.SCHEME_STACK, tb.DECOMP_MONO, 1)):
        _compare(_gpu(LATTICE, n, scheme, decomp, remap_every=remap), o, n)


def test_ce_full_grid_benchmark_path_full_size():
    """1e6 continuous-energy histories on the full grid (4 nuclides x 1e5
    points, union ~4e5), 100 energy bins, 64 events per remap."""
    n = 1_000_000
    g = _gpu(CE_FULL, n, tb.SCHEME_ASYNC, tb.DECOMP_MONO, remap_every=64)
    _compare(g, _oracle(CE_FULL, n), n)


def test_ce_energy_tally_1e4_bins():
    """The finest energy-tally resolution (1e4 bins per material) on the full
    grid, in both schedulers."""
    n = 200_000
    o = _oracle(CE_1E4_BINS, n)
    assert o["energy"].size == 2 * 10_000
    for scheme, decomp, remap in ((tb.SCHEME_ASYNC, tb.DECOMP_MONO, 64), (tb.SCHEME_STACK, tb.DECOMP_SPLIT, 1)):
        _compare(_gpu(CE_1E4_BINS, n, scheme, decomp, remap_every=remap), o, n)


def test_power_iteration_full_batch():
    """Power iteration at the benchmark's batch size (1e6 histories per batch,
    1 inactive + 2 active batches) in the benchmark's configuration: k per
    batch and source sizes bit-equal, the last batch's histories bit-equal,
    tallies within tolerance."""
    p = _spec(LATTICE)
    nper, ni, na = 1_000_000, 1, 2
    o = oracle.power_iteration(p, nper, ni, na, seed=1, log_batch=ni + na - 1)
    assert o["status"] == 0
    prob = tb.Problem(p)
    g = prob.power_iteration(nper, ni, na, tb.RunOpts(seed=1, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO,
                                                      remap_every=512, want_event_log=True))
    assert np.array_equal(g["n_source"], o["n_source"])
    assert np.array_equal(g["k_batch"], o["k_batch"])
    assert_tally_close(g["ktl_batch"], o["ktl_batch"], "ktl")
    assert_tally_close(prob.tally(tb.TALLY_MESH), o["mesh_mean"], "mesh mean")
    assert_tally_close(prob.tally(tb.TALLY_SCALARS), o["scalars_mean"], "scalars mean")
    nlast = int(o["n_source"][-1])
    assert_logs_equal(prob.event_log(nlast), (o["log_n"], o["log_cell"], o["log_type"]), "last batch")
    assert np.array_equal(g["final_by_type"], o["final_by_type"])
    prob.close()
