"""Weight-window closeout on the GPU against the oracle.

With windows the closeout runs after every event a particle survives:
roulette below the window, splitting above it, each split copy on its own
counter-based stream.  The source histories' logs (event counts, final cells,
final types) are bit-equal to the oracle's; the event and final-type counts,
which include every split copy, are equal; the tallies agree within 1e-10.
Both schedulers, the monolithic loop with deferred collisions (64 and 512
events per remap) and with whole events (one per remap)."""
import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal, assert_tally_close

pytestmark = pytest.mark.gpu

SCHEMES = [(tb.SCHEME_ASYNC, 512), (tb.SCHEME_ASYNC, 64), (tb.SCHEME_ASYNC, 1), (tb.SCHEME_STACK, 1)]
IDS = ["async-512", "async-64", "async-1", "stack-1"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _checkerboard_box():
    n = 4
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    even = ((i + j + k) % 2 == 0).transpose(2, 1, 0).reshape(-1)
    ww = np.where(even, 0.1, 1.5).reshape(-1, 1)
    p = inputs.box_mg("ww_box", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.5]],
                      bc=inputs.BC_REFLECT, mesh_n=(n, n, n), src_kind=inputs.SRC_POINT, src_point=(5.0, 5.0, 5.0),
                      src_group=0)
    return p.replace(ww_lower=ww, ww_upper=5.0, ww_survival=2.5, ww_max_split=4)


def _lattice_importance():
    """Importance rising toward the lattice's outer corner: windows fall
    with the distance from the origin (splitting outward, roulette inward)."""
    p = inputs.c5g7_lattice(fission=False)
    nx, ny, nz = p.mesh_n
    G = p.n_groups
    ix = np.arange(nx)[None, :]
    iy = np.arange(ny)[:, None]
    r = np.sqrt(ix ** 2 + iy ** 2) / np.hypot(nx, ny)          # 0 .. 1
    lo = (0.8 * np.exp(-3.0 * r)).reshape(-1)
    ww = np.repeat(lo[:, None], G, axis=1)
    return p.replace(ww_lower=ww, ww_upper=4.0, ww_survival=2.0, ww_max_split=8)


def _gpu(spec, n, scheme, remap, seed=1, **kw):
    prob = tb.Problem(spec)
    st = prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=tb.DECOMP_MONO,
                                          remap_every=remap, want_event_log=True, **kw))
    out = {"stats": st, "log": prob.event_log(n), "mesh": prob.tally(tb.TALLY_MESH),
           "energy": prob.tally(tb.TALLY_ENERGY), "scalars": prob.tally(tb.TALLY_SCALARS)}
    prob.close()
    return out


def _compare(g, o):
    assert_logs_equal(g["log"], (o["log_n"], o["log_cell"], o["log_type"]), "source histories")
    assert np.array_equal(g["stats"]["events_by_type"], o["events_by_type"])
    assert np.array_equal(g["stats"]["final_by_type"], o["final_by_type"])
    assert_tally_close(g["mesh"], o["mesh"], "mesh")
    assert_tally_close(g["energy"], o["energy"], "energy")
    assert_tally_close(g["scalars"], o["scalars"], "scalars")


@pytest.mark.parametrize("scheme,remap", SCHEMES, ids=IDS)
def test_box_with_splitting_and_roulette(scheme, remap):
    spec = _checkerboard_box()
    n = 20_011
    o = oracle.run_fixed_source(spec, n, seed=3)
    assert o["status"] == 0
    # both rules fire: roulette ends copies and histories, splitting adds events
    assert o["final_by_type"][tb.EV_CUTOFF] > 100 and o["final_by_type"].sum() > n
    _compare(_gpu(spec, n, scheme, remap, seed=3, stash_slots=1024), o)


@pytest.mark.parametrize("scheme,remap", SCHEMES, ids=IDS)
def test_lattice_with_an_importance_map(scheme, remap):
    spec = _lattice_importance()
    n = 10_007
    o = oracle.run_fixed_source(spec, n, seed=5)
    assert o["status"] == 0 and o["final_by_type"].sum() > n
    _compare(_gpu(spec, n, scheme, remap, seed=5, stash_slots=1024), o)


def test_continuous_energy_with_windows():
    base = inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=100)
    base = base.replace(mesh_lo=(-0.63, -0.63, -50.0), mesh_hi=(0.63, 0.63, 50.0), mesh_n=(4, 4, 1))
    ww = np.array([0.05, 0.4, 0.05, 0.4, 0.4, 0.05, 0.4, 0.05, 0.05, 0.4, 0.05, 0.4, 0.4, 0.05, 0.4, 0.05])
    spec = base.replace(ww_lower=ww.reshape(-1, 1), ww_upper=4.0, ww_survival=2.0, ww_max_split=4)
    n = 3_001
    o = oracle.run_fixed_source(spec, n, seed=2)
    assert o["status"] == 0 and o["final_by_type"].sum() > n
    for scheme, remap in ((tb.SCHEME_ASYNC, 64), (tb.SCHEME_STACK, 1)):
        _compare(_gpu(spec, n, scheme, remap, seed=2, stash_slots=1024), o)


def test_windows_with_forced_spills_through_the_global_links():
    """Split copies and window-weighted particles that travel through the
    global spill links (their records leave and re-enter the block stashes):
    the same histories and tallies as the oracle, multigroup and continuous
    energy (a continuous-energy record carries no group index)."""
    base = inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=100)
    base = base.replace(mesh_lo=(-0.63, -0.63, -50.0), mesh_hi=(0.63, 0.63, 50.0), mesh_n=(4, 4, 1))
    ww = np.array([0.05, 0.4, 0.05, 0.4, 0.4, 0.05, 0.4, 0.05, 0.05, 0.4, 0.05, 0.4, 0.4, 0.05, 0.4, 0.05])
    ce = base.replace(ww_lower=ww.reshape(-1, 1), ww_upper=4.0, ww_survival=2.0, ww_max_split=4)
    for spec, n, seed in ((_checkerboard_box(), 10_007, 3), (ce, 3_001, 2)):
        o = oracle.run_fixed_source(spec, n, seed=seed)
        assert o["status"] == 0
        for remap in (64, 512):
            g = _gpu(spec, n, tb.SCHEME_ASYNC, remap, seed=seed, stash_slots=512, spill_threshold=-32,
                     queue_capacity=8192 * 32)
            assert g["stats"]["spills"] > 0, g["stats"]
            _compare(g, o)


def test_inactive_windows_equal_the_analog_run():
    spec = _checkerboard_box()
    analog = inputs.box_mg("ww_box", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.5]],
                           bc=inputs.BC_REFLECT, mesh_n=(4, 4, 4), src_kind=inputs.SRC_POINT,
                           src_point=(5.0, 5.0, 5.0), src_group=0)
    a = _gpu(analog, 5_003, tb.SCHEME_ASYNC, 512)
    b = _gpu(spec.replace(ww_lower=np.zeros((64, 1))), 5_003, tb.SCHEME_ASYNC, 512)
    for x, y in zip(a["log"], b["log"]):
        assert np.array_equal(x, y)
    for k in ("mesh", "scalars"):
        assert np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)), k


def test_refusals_and_capacity():
    spec = _checkerboard_box()
    prob = tb.Problem(spec)
    for kw in (dict(decomposition=tb.DECOMP_SPLIT), dict(decomposition=tb.DECOMP_SPLIT_LOOKUP),
               dict(decomposition=tb.DECOMP_STREAM)):
        with pytest.raises(tb.TransportError) as e:
            prob.run_fixed_source(tb.RunOpts(n_histories=100, scheme=tb.SCHEME_ASYNC, **kw))
        assert e.value.status == tb.TR_ERR_INVALID
    with pytest.raises(tb.TransportError) as e:
        prob.power_iteration(100, 1, 2, tb.RunOpts(seed=1))
    assert e.value.status == tb.TR_ERR_INVALID
    prob.close()
    # windows far below the weight everywhere split every particle into 64
    # copies at its first event, and again at later ones: more copies than a
    # stash or an output stack holds, a capacity error in both schedulers,
    # after which the problem stays usable
    burst = tb.Problem(spec.replace(ww_lower=np.full((64, 1), 1e-3), ww_max_split=64))
    for scheme, kw in ((tb.SCHEME_ASYNC, dict(remap_every=512, stash_slots=288)),
                       (tb.SCHEME_STACK, dict(queue_capacity=4096))):
        with pytest.raises(tb.TransportError) as e:
            burst.run_fixed_source(tb.RunOpts(n_histories=20_000, seed=3, scheme=scheme, **kw))
        assert e.value.status == tb.TR_ERR_CAPACITY
    burst.close()
    prob = tb.Problem(spec)
    st = prob.run_fixed_source(tb.RunOpts(n_histories=1000, seed=3, scheme=tb.SCHEME_ASYNC, remap_every=512,
                                          stash_slots=1024))
    assert st["histories"] == 1000
    prob.close()
    for bad in (dict(ww_upper=1.0), dict(ww_survival=6.0), dict(ww_max_split=1), dict(ww_max_split=65),
                dict(ww_lower=-np.ones((64, 1)))):
        with pytest.raises(tb.TransportError) as e:
            tb.Problem(spec.replace(**bad))
        assert e.value.status == tb.TR_ERR_INVALID
