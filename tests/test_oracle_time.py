"""Pins for the oracle's time-dependent transport (our reading of the paper's
temporal tally resolution and census, Sec. 4): histories start at t = 0, a
particle of speed v covers a flight of length d in d / v, the census ends
histories at t_census, and the time tally scores the track length spent in
each uniform time bin."""
import math

import numpy as np

import oracle
from paper_2506_00263_gb300 import inputs

EV_CUTOFF = 6


def _mg_box(sigma_t, sigma_s, v, t_cen, nbins, size=10.0):
    return inputs.box_mg("timed", (0.0, 0.0, 0.0), (size, size, size), sigma_t=[sigma_t], sigma_s=[[sigma_s]],
                         bc=inputs.BC_REFLECT, src_kind=inputs.SRC_POINT,
                         src_point=(size / 2, size / 2, size / 2), src_group=0,
                         inv_velocity=np.array([1.0 / v]), n_time_bins=nbins, t_census=t_cen)


def test_streaming_reaches_census_with_track_v_times_t():
    """No interactions (sigma_t ~ 0): every history ends at census, its track
    length is v T, and each of the n time bins holds v T / n."""
    v, T, nb = 3.0, 2.0, 8
    p = _mg_box(1e-300, 0.0, v, T, nb)
    r = oracle.run_fixed_source(p, 50, seed=3, per_history=True)
    assert r["status"] == 0
    assert np.all(r["log_type"] == EV_CUTOFF)
    assert np.allclose(r["hist_track"], v * T, rtol=1e-12, atol=0)
    assert np.allclose(r["time"], v * T / nb, rtol=1e-12, atol=0)
    assert abs(r["time"].sum() - r["scalars"][0]) <= 1e-12 * r["scalars"][0]


def test_ce_speed_is_the_textbook_thermal_speed():
    """Continuous energy: v = c sqrt(2 E / (m_n c^2)); a thermal (0.0253 eV)
    neutron streaming for T covers 2200 m/s * T (to 0.02 %)."""
    p = inputs.ce_pin_cell(n_points=2000, n_res=5, n_ebins=1, source_energy=0.0253)
    p = p.replace(mat_density=p.mat_density * 1e-30, t_census=1e-3, n_time_bins=4)
    r = oracle.run_fixed_source(p, 20, seed=5, per_history=True)
    assert r["status"] == 0
    assert np.all(r["log_type"] == EV_CUTOFF)
    speed = r["hist_track"] / 1e-3          # cm/s
    assert np.all(np.abs(speed - 2.2e5) < 0.0002 * 2.2e5), speed[:3]
    assert np.allclose(r["time"], speed[0] * 1e-3 / 4, rtol=1e-12)


def test_one_group_survival_and_time_bins_closed_form():
    """Infinite medium (reflective box), one group: the population decays as
    exp(-Sigma_a v t), so bin [a, b] holds (exp(-Sa v a) - exp(-Sa v b)) / Sa
    per source particle and exp(-Sa v T) of the histories reach census."""
    st, ss, v, T, nb = 1.0, 0.5, 2.0, 3.0, 6
    sa = st - ss
    p = _mg_box(st, ss, v, T, nb)
    runs = [oracle.run_fixed_source(p, 4000, seed=100 + s) for s in range(8)]
    for r in runs:
        assert r["status"] == 0
        assert abs(r["time"].sum() - r["scalars"][0]) <= 1e-12 * r["scalars"][0]
    tb = np.array([r["time"] for r in runs])
    mean, se = tb.mean(0), tb.std(0, ddof=1) / math.sqrt(len(runs))
    edges = np.linspace(0.0, T, nb + 1)
    ref = (np.exp(-sa * v * edges[:-1]) - np.exp(-sa * v * edges[1:])) / sa
    assert np.all(np.abs(mean - ref) < 5 * se + 1e-3 * ref.max()), (mean, ref)
    frac = np.array([r["final_by_type"][EV_CUTOFF] / 4000.0 for r in runs])
    assert abs(frac.mean() - math.exp(-sa * v * T)) < 5 * frac.std(ddof=1) / math.sqrt(len(runs)) + 1e-3


def test_census_changes_nothing_before_it():
    """A census later than every history's end leaves the histories as they
    are without one (same events and tallies, every history ends the same)."""
    p0 = inputs.cube_one_group(n_mesh=4)
    p1 = p0.replace(inv_velocity=np.array([1e-9]), t_census=1e6, n_time_bins=2)
    a = oracle.run_fixed_source(p0, 2000, seed=9)
    b = oracle.run_fixed_source(p1, 2000, seed=9)
    assert np.array_equal(a["log_n"], b["log_n"]) and np.array_equal(a["log_type"], b["log_type"])
    assert np.array_equal(a["events_by_type"], b["events_by_type"])
    assert np.allclose(a["mesh"], b["mesh"], rtol=0, atol=0)
    assert b["time"][1] == 0.0 and abs(b["time"].sum() - b["scalars"][0]) <= 1e-12 * b["scalars"][0]
