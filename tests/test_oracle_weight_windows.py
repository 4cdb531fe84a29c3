"""Pins of the oracle's weight-window closeout (the closeout event of the
paper's decomposed scheme, Sec. 4: weights and weight windows for the
particle's next loop iteration; the rules are our reading).

Splitting and Russian roulette change how a history's weight is carried, not
its expectation, so every tally keeps its analog mean:
  * infinite medium (reflective box, one group): the track length per source
    particle is 1/Sigma_a whatever the windows, under an importance map that
    forces both splitting and roulette;
  * windows that never trigger (all lower bounds 0, or bounds that bracket
    the weight 1 everywhere) give exactly the analog run.
A dropped 1/k on split copies, copies left untransported, or an inverted
roulette test bias the first pin by far more than its statistical margin."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import inputs


def _box(ww=None, n_mesh=4, **kw):
    p = inputs.box_mg("ww_box", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.5]],
                      bc=inputs.BC_REFLECT, mesh_n=(n_mesh, n_mesh, n_mesh),
                      src_kind=inputs.SRC_POINT, src_point=(5.0, 5.0, 5.0), src_group=0)
    if ww is not None:
        p = p.replace(ww_lower=np.ascontiguousarray(ww, np.float64).reshape(-1, 1), **kw)
    return p


def _checkerboard(n=4, low=0.05, high=2.0):
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # voxel index (k * n + j) * n + i with i fastest
    even = ((i + j + k) % 2 == 0).transpose(2, 1, 0).reshape(-1)
    return np.where(even, low, high)


def test_infinite_medium_flux_unbiased_under_splitting_and_roulette():
    ww = _checkerboard()
    p = _box(ww, ww_upper=5.0, ww_survival=3.0, ww_max_split=16)
    means, cutoffs, events = [], 0, 0
    for seed in range(1, 9):
        r = oracle.run_fixed_source(p, 4000, seed=seed)
        assert r["status"] == 0
        means.append(r["scalars"][0])
        cutoffs += int(r["final_by_type"][oracle.ORC_CUTOFF])
        events += int(r["events_by_type"][1:].sum())
    a = oracle.run_fixed_source(_box(), 4000 * 8, seed=1)
    analog_events = int(a["events_by_type"][1:].sum())
    # both rules fired: roulette ended histories, splitting multiplied the events
    assert cutoffs > 1000 and events > 1.2 * analog_events, (cutoffs, events, analog_events)
    m = np.array(means)
    se = m.std(ddof=1) / math.sqrt(len(m))
    assert abs(m.mean() - 2.0) < 5 * se + 1e-3, (m.mean(), se)
    # the absorption rate per source particle is 1 (every particle is absorbed in the end)
    r = oracle.run_fixed_source(p, 20000, seed=11)
    assert abs(r["scalars"][1] - 1.0) < 0.05, r["scalars"]


def test_inactive_windows_equal_the_analog_run():
    a = oracle.run_fixed_source(_box(), 3000, seed=5)
    for ww in (np.zeros(64), np.full(64, 0.5)):     # no window / bounds [0.5, 2.5] bracket w = 1
        b = oracle.run_fixed_source(_box(ww, ww_upper=5.0, ww_survival=3.0), 3000, seed=5)
        for k in ("log_n", "log_cell", "log_type"):
            assert np.array_equal(a[k], b[k])
        assert np.array_equal(a["mesh"], b["mesh"]) and np.array_equal(a["scalars"], b["scalars"])


def test_windows_refused_where_not_offered():
    p = _box(_checkerboard())
    assert oracle.power_iteration(p, 100, 1, 2)["status"] != 0
    assert oracle.sensitivities(p, 100)["status"] != 0
