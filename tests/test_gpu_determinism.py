"""Tallies are reduced in fixed-point integers (order-independent sums), so
they are bit-identical from run to run and across schedules: the same seed
gives the same bits whatever the scheme, decomposition, remap frequency,
stash size or spill pattern, because every scheme makes the same histories
and therefore the same set of track-length contributions."""
import numpy as np
import pytest

from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs

pytestmark = pytest.mark.gpu

SCHEMES = [(tb.SCHEME_STACK, tb.DECOMP_MONO, {}), (tb.SCHEME_STACK, tb.DECOMP_SPLIT, {}),
           (tb.SCHEME_STACK, tb.DECOMP_SPLIT_LOOKUP, {}),
           (tb.SCHEME_ASYNC, tb.DECOMP_MONO, {}), (tb.SCHEME_ASYNC, tb.DECOMP_MONO, {"remap_every": 512}),
           (tb.SCHEME_ASYNC, tb.DECOMP_MONO, {"remap_every": 64, "stash_slots": 288, "spill_threshold": -32,
                                              "queue_capacity": 4096}),
           (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT, {}), (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT_LOOKUP, {}),
           (tb.SCHEME_ASYNC, tb.DECOMP_STREAM, {"remap_every": 5})]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _tallies(spec, n, scheme, decomp, seed=1, **kw):
    prob = tb.Problem(spec)
    prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=decomp, **kw))
    out = [prob.tally(t) for t in (tb.TALLY_MESH, tb.TALLY_ENERGY, tb.TALLY_SCALARS)]
    prob.close()
    return out


def _same_bits(a, b, what):
    for name, x, y in zip(("mesh", "energy", "scalars"), a, b):
        assert x.shape == y.shape
        if not np.array_equal(x.view(np.uint64), y.view(np.uint64)):
            i = int(np.argmax(x.view(np.uint64) != y.view(np.uint64)))
            raise AssertionError(f"{what}/{name}: bin {i} differs: {x[i]!r} vs {y[i]!r}")


@pytest.mark.parametrize("name,n", [("lattice", 20_011), ("ce", 3_001), ("cube", 50_003)])
def test_tallies_bit_identical_across_runs_and_schedules(name, n):
    spec = {"lattice": inputs.c5g7_lattice, "cube": inputs.cube_one_group,
            "ce": lambda: inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=100)}[name]()
    ref = _tallies(spec, n, tb.SCHEME_ASYNC, tb.DECOMP_MONO)
    _same_bits(ref, _tallies(spec, n, tb.SCHEME_ASYNC, tb.DECOMP_MONO), "repeat")
    for scheme, decomp, kw in SCHEMES:
        _same_bits(ref, _tallies(spec, n, scheme, decomp, **kw), f"scheme {scheme} decomposition {decomp} {kw}")


def test_power_iteration_tallies_bit_identical_across_schemes():
    spec = inputs.c5g7_lattice()
    res = []
    for scheme, decomp, remap in ((tb.SCHEME_ASYNC, tb.DECOMP_MONO, 512), (tb.SCHEME_STACK, tb.DECOMP_MONO, 1),
                                  (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT, 1)):
        prob = tb.Problem(spec)
        r = prob.power_iteration(5000, 2, 3, tb.RunOpts(seed=2, scheme=scheme, decomposition=decomp,
                                                         remap_every=remap))
        res.append((r["k_batch"], r["ktl_batch"], prob.tally(tb.TALLY_MESH), prob.tally(tb.TALLY_MESH, stddev=True),
                    prob.tally(tb.TALLY_SCALARS)))
        prob.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def test_fixed_point_range_error_is_reported():
    """A track-length score of 2^39 or more lies outside the fixed-point
    range: the run reports TR_ERR_CAPACITY instead of a wrapped sum.  A
    beam along x from the centre of a 2^41 cm vacuum box with a negligible
    cross section makes one 2^40 cm segment per history."""
    big = 2.0 ** 41
    spec = inputs.box_mg("huge", (0.0, 0.0, 0.0), (big, big, big), sigma_t=[1e-300], sigma_s=[[0.0]],
                         bc=inputs.BC_VACUUM, src_kind=inputs.SRC_POINT, src_point=(big / 2, big / 2, big / 2),
                         src_direction=(1.0, 0.0, 0.0), src_group=0)
    prob = tb.Problem(spec)
    with pytest.raises(tb.TransportError) as e:
        prob.run_fixed_source(tb.RunOpts(n_histories=64, scheme=tb.SCHEME_ASYNC))
    assert e.value.status == tb.TR_ERR_CAPACITY
    prob.close()
