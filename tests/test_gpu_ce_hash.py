"""The continuous-energy lookup's union-grid hash, both placements, against
the oracle (whose lookup is a plain binary search over the union grid).

The asynchronous kernel copies the hash buckets into each block's shared
memory when they fit beside the stash (at most 64 KB); the pin cell's grids
span 41 octaves and their hash stays in global memory.  A pin cell whose
nuclide grids are cut to 1 eV .. 20 keV (14.3 octaves) has a hash that fits,
so these runs take the shared-memory path; the union index, and so every
history, must be the same as the oracle's either way."""
import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _narrow_pin_cell(lo=1.0, hi=2.0e4):
    base = inputs.ce_pin_cell(n_points=6000, n_res=40, n_ebins=50, source_energy=1.0e4)
    es, ss = [], []
    for E, S in zip(base.nuc_energy, base.nuc_sigma):
        keep = (E >= lo) & (E <= hi)
        es.append(np.ascontiguousarray(E[keep]))
        ss.append(np.ascontiguousarray(S[keep]))
    # the cutoff at the highest first grid point: every lookup stays inside every grid
    return base.replace(nuc_energy=es, nuc_sigma=ss, energy_cutoff=float(max(E[0] for E in es)))


def _run(spec, n, scheme, remap):
    prob = tb.Problem(spec)
    st = prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=4, scheme=scheme, decomposition=tb.DECOMP_MONO,
                                          remap_every=remap, want_event_log=True))
    out = {"stats": st, "log": prob.event_log(n), "energy": prob.tally(tb.TALLY_ENERGY),
           "scalars": prob.tally(tb.TALLY_SCALARS)}
    prob.close()
    return out


@pytest.mark.parametrize("name", ["narrow (hash in shared memory)", "full (hash in global memory)"])
def test_ce_lookup_hash_placements_match_the_oracle(name):
    spec = _narrow_pin_cell() if name.startswith("narrow") else inputs.ce_pin_cell(n_points=6000, n_res=40,
                                                                                   n_ebins=50)
    if name.startswith("narrow"):
        span = np.log2(max(E[-1] for E in spec.nuc_energy) / min(E[0] for E in spec.nuc_energy))
        assert span < 15.0                      # 2^10 buckets per octave: below 64 KB of buckets
    n = 4_001
    o = oracle.run_fixed_source(spec, n, seed=4)
    assert o["status"] == 0
    for scheme, remap in ((tb.SCHEME_ASYNC, 64), (tb.SCHEME_ASYNC, 1), (tb.SCHEME_STACK, 1)):
        g = _run(spec, n, scheme, remap)
        assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]), name)
        assert np.array_equal(g["stats"]["events_by_type"], o["events_by_type"])
        assert_tally_close(g["energy"], o["energy"], "energy")
        assert_tally_close(g["scalars"], o["scalars"], "scalars")
