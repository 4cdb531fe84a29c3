"""Timed transport on the GPU (census and time bins, the paper's temporal
tally resolution): bit-exact histories and tallies within the parity
tolerance against the oracle for every scheme and decomposition, the
streaming closed form, and the host-side refusals."""
import functools

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu

ALL = [(s, d) for s in (tb.SCHEME_STACK, tb.SCHEME_ASYNC)
       for d in (tb.DECOMP_MONO, tb.DECOMP_SPLIT, tb.DECOMP_SPLIT_LOOKUP)]
IDS = [f"{'stack' if s == tb.SCHEME_STACK else 'async'}-{['mono', 'split', 'lookup'][d]}" for s, d in ALL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _mg_timed(nbins=6, t_cen=3.0, v=2.0):
    p = inputs.cube_one_group(n_mesh=8)
    return p.replace(inv_velocity=np.array([1.0 / v]), t_census=t_cen, n_time_bins=nbins)


@functools.lru_cache(maxsize=None)
def _ce_timed(nbins):
    p = inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=10, source_energy=14e6)
    return p.replace(t_census=2e-7, n_time_bins=nbins)


def _run(spec, n, scheme, decomp, seed=1, **kw):
    prob = tb.Problem(spec)
    st = prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=decomp,
                                          want_event_log=True, **kw))
    out = {"stats": st, "log": prob.event_log(n), "time": prob.tally(tb.TALLY_TIME),
           "scalars": prob.tally(tb.TALLY_SCALARS), "mesh": prob.tally(tb.TALLY_MESH),
           "energy": prob.tally(tb.TALLY_ENERGY)}
    prob.close()
    return out


def _compare(g, o):
    assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]))
    assert np.array_equal(g["stats"]["events_by_type"], o["events_by_type"])
    assert np.array_equal(g["stats"]["final_by_type"], o["final_by_type"])
    for k in ("time", "scalars", "mesh", "energy"):
        assert_tally_close(g[k], o[k], k)


@pytest.mark.parametrize("scheme,decomp", ALL, ids=IDS)
def test_timed_box_parity(scheme, decomp):
    spec = _mg_timed()
    n = 30_011
    o = oracle.run_fixed_source(spec, n, seed=1)
    assert o["status"] == 0 and o["final_by_type"][tb.EV_CUTOFF] > 0
    _compare(_run(spec, n, scheme, decomp), o)


@pytest.mark.parametrize("nbins", [1, 8, 128])
def test_timed_ce_parity(nbins):
    spec = _ce_timed(nbins)
    n = 5_003
    o = oracle.run_fixed_source(spec, n, seed=2)
    assert o["status"] == 0 and o["final_by_type"][tb.EV_CUTOFF] > 0
    for scheme, decomp in ((tb.SCHEME_ASYNC, tb.DECOMP_MONO), (tb.SCHEME_STACK, tb.DECOMP_SPLIT),
                           (tb.SCHEME_ASYNC, tb.DECOMP_SPLIT_LOOKUP)):
        _compare(_run(spec, n, scheme, decomp, seed=2), o)


@pytest.mark.parametrize("remap", [64, 512])
def test_timed_deferred_collision_loop(remap):
    """The monolithic loop with deferred collisions on timed problems."""
    spec = _mg_timed()
    _compare(_run(spec, 30_011, tb.SCHEME_ASYNC, tb.DECOMP_MONO, seed=1, remap_every=remap),
             oracle.run_fixed_source(spec, 30_011, seed=1))
    ce = _ce_timed(8)
    _compare(_run(ce, 5_003, tb.SCHEME_ASYNC, tb.DECOMP_MONO, seed=2, remap_every=remap),
             oracle.run_fixed_source(ce, 5_003, seed=2))


def test_streaming_closed_form_on_gpu():
    """No interactions: every history reaches census with track v T; each bin holds v T / n."""
    v, T, nb = 3.0, 2.0, 8
    spec = inputs.box_mg("stream", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1e-300], sigma_s=[[0.0]],
                         bc=inputs.BC_REFLECT, src_kind=inputs.SRC_POINT, src_point=(5.0, 5.0, 5.0), src_group=0,
                         inv_velocity=np.array([1.0 / v]), n_time_bins=nb, t_census=T)
    g = _run(spec, 1000, tb.SCHEME_ASYNC, tb.DECOMP_MONO)
    assert np.all(g["log"][2] == tb.EV_CUTOFF)
    assert np.allclose(g["time"], v * T / nb, rtol=1e-12)
    assert abs(g["scalars"][0] - v * T) <= 1e-12 * v * T


def test_timed_refusals():
    spec = _mg_timed()
    bad = spec.replace(inv_velocity=None)
    with pytest.raises(tb.TransportError) as e:
        tb.Problem(bad)
    assert e.value.status == tb.TR_ERR_INVALID
    prob = tb.Problem(spec)
    with pytest.raises(tb.TransportError) as e:
        prob.power_iteration(1000, 1, 2, tb.RunOpts(seed=1))
    assert e.value.status == tb.TR_ERR_INVALID
    import torch
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(tb.TransportError) as e:
        prob.run_fixed_source_noalloc(tb.RunOpts(n_histories=10, scheme=tb.SCHEME_ASYNC), buf.data_ptr(), 0,
                                      buf.data_ptr())
    assert e.value.status == tb.TR_ERR_INVALID
    prob.close()
