"""Pins for the oracle's transport results against closed forms.

Each check is chosen so that a plausible mistake in the oracle fails it: a
dropped path segment breaks the infinite-medium flux S/Sigma_a and the
exponential track-length law; a wrong sign or plane in the distance breaks the
uncollided transmission exp(-Sigma_t x); a transposed scatter matrix changes
the multigroup spectrum and k-infinity; a wrong elastic formula or energy bin
breaks the hydrogen slowing-down flux 1/(Sigma_t E); a mis-clipped segment
breaks the mesh length sums.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2506_00263_gb300 import inputs


def _z(mean, ref, se):
    return abs(mean - ref) / se


def test_infinite_medium_one_group_closed_forms():
    p = inputs.cube_one_group()
    N = 100_000
    r = oracle.run_fixed_source(p, N, seed=1, per_history=True)
    assert r["status"] == 0
    sig_a, c = 0.5, 0.5
    tr = r["hist_track"]
    # flux per source particle = 1/Sigma_a; track length per history ~ Exp(Sigma_a)
    assert _z(tr.mean(), 1.0 / sig_a, tr.std() / math.sqrt(N)) < 4.5
    assert stats.kstest(tr, stats.expon(scale=1.0 / sig_a).cdf).pvalue > 1e-4
    # collisions per history ~ geometric with mean 1/(1-c)
    k = r["hist_coll"].astype(float)
    assert _z(k.mean(), 1.0 / (1.0 - c), k.std() / math.sqrt(N)) < 4.5
    assert _z((k == 1).mean(), 1.0 - c, math.sqrt(c * (1 - c) / N)) < 4.5
    # conservation and tally consistency
    assert r["final_by_type"][oracle.ORC_ABSORB] == N and r["final_by_type"].sum() == N
    assert abs(r["mesh"].sum() - r["scalars"][0]) <= 1e-12 * r["scalars"][0]
    assert abs(r["scalars"][0] - tr.mean()) <= 1e-12 * tr.mean()
    assert abs(r["scalars"][1] - sig_a * r["scalars"][0]) <= 1e-12 * r["scalars"][1]
    assert r["scalars"][2] == 0.0


def test_uncollided_transmission_slab():
    L, N = 3.0, 200_000
    p = inputs.box_mg("slab", (0.0, 0.0, 0.0), (L, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.0]],
                      bc=inputs.BC_VACUUM, mesh_n=(12, 1, 1),
                      src_kind=inputs.SRC_POINT, src_point=(0.0, 5.3, 4.7), src_direction=(1.0, 0.0, 0.0),
                      src_group=0)
    r = oracle.run_fixed_source(p, N, seed=3)
    leak = r["final_by_type"][oracle.ORC_LEAK] / N
    pt = math.exp(-L)
    assert _z(leak, pt, math.sqrt(pt * (1 - pt) / N)) < 4.5
    assert r["final_by_type"][oracle.ORC_LEAK] + r["final_by_type"][oracle.ORC_ABSORB] == N
    # per-voxel track length: integral of exp(-x) over the voxel
    x = np.linspace(0.0, L, 13)
    exp_len = np.exp(-x[:-1]) - np.exp(-x[1:])
    w = L / 12
    se = np.sqrt(w * exp_len / N)
    assert np.all(np.abs(r["mesh"] - exp_len) < 5 * se)


def test_k_infinity_one_group():
    p = inputs.box_mg("kinf1", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.6]],
                      nu_sigma_f=[0.5], chi=[1.0], bc=inputs.BC_REFLECT, mesh_n=(2, 2, 2),
                      src_kind=inputs.SRC_BOX, src_lo=(0.0, 0.0, 0.0), src_hi=(10.0, 10.0, 10.0), src_group=0)
    e = oracle.power_iteration(p, 4000, 4, 40, seed=5)
    assert e["status"] == 0
    kinf = 0.5 / 0.4
    assert _z(e["k_mean"], kinf, e["k_std"]) < 4.5
    ktl = e["ktl_batch"][4:]
    assert _z(ktl.mean(), kinf, ktl.std(ddof=1) / math.sqrt(len(ktl))) < 4.5
    # every batch restarts from splitting-roulette copies of the bank
    assert np.all(e["n_source"][1:] > 0)


def _mg_material(m):
    st, ss, nsf, chi = inputs.c5g7_xs(2025)
    return st[m], ss[m], nsf[m], chi[m]


def test_multigroup_infinite_medium_spectrum():
    st, ss, nsf, chi = _mg_material(0)
    G = len(st)
    p = inputs.box_mg("mg_inf", (0.0, 0.0, 0.0), (20.0, 20.0, 20.0), sigma_t=st, sigma_s=ss, nu_sigma_f=nsf,
                      chi=chi, bc=inputs.BC_REFLECT, mesh_n=(1, 1, 1), mesh_by_group=True,
                      src_kind=inputs.SRC_POINT, src_point=(10.0, 10.0, 10.0), src_group=0)
    # balance: (diag(Sigma_t) - Sigma_s^T) phi = e_0 (fission counts as absorption here)
    A = np.diag(st) - ss.T
    phi = np.linalg.solve(A, np.eye(G)[0])
    runs = np.array([oracle.run_fixed_source(p, 20000, seed=100 + s, logs=False)["mesh"] for s in range(8)])
    mean, se = runs.mean(0), runs.std(0, ddof=1) / math.sqrt(len(runs))
    assert np.all(np.abs(mean - phi) < 5 * se + 1e-3 * phi), (mean, phi)
    # total absorption per source particle is exactly one in an infinite medium
    tot_abs = np.array([oracle.run_fixed_source(p, 5000, seed=s, logs=False)["scalars"][1] for s in range(4)])
    assert abs(tot_abs.mean() - 1.0) < 5 * tot_abs.std(ddof=1) / 2 + 1e-3


def test_multigroup_k_infinity():
    st, ss, nsf, chi = _mg_material(1)
    p = inputs.box_mg("mg_kinf", (0.0, 0.0, 0.0), (20.0, 20.0, 20.0), sigma_t=st, sigma_s=ss, nu_sigma_f=nsf,
                      chi=chi, bc=inputs.BC_REFLECT, mesh_n=(1, 1, 1),
                      src_kind=inputs.SRC_BOX, src_lo=(0.0, 0.0, 0.0), src_hi=(20.0, 20.0, 20.0), src_group=-1)
    A = np.diag(st) - ss.T
    F = np.outer(chi, nsf)
    kinf = max(abs(np.linalg.eigvals(np.linalg.solve(A, F))))
    e = oracle.power_iteration(p, 4000, 5, 40, seed=9)
    assert e["status"] == 0
    assert _z(e["k_mean"], kinf, e["k_std"]) < 4.5, (e["k_mean"], e["k_std"], kinf)
    # a transposed scatter matrix would give a clearly different k
    kt = max(abs(np.linalg.eigvals(np.linalg.solve(np.diag(st) - ss, F))))
    assert abs(kt - kinf) > 10 * e["k_std"]


def test_hydrogen_slowing_down():
    E0, Ec, sig = 1e6, 1.0, 20.0
    p = inputs.ce_box(A=1.0, sigma_el=sig, sigma_cap=0.0, energy=E0, cutoff=Ec)
    p.energy_edges = np.logspace(0.0, 6.0, 13)
    N = 20000
    runs = [oracle.run_fixed_source(p, N, seed=20 + s, per_history=True) for s in range(6)]
    coll = np.concatenate([r["hist_coll"] for r in runs]).astype(float)
    # E' = E U on hydrogen: collisions to fall below Ec = 1 + Poisson(ln(E0/Ec))
    lam = math.log(E0 / Ec)
    assert _z(coll.mean(), 1.0 + lam, math.sqrt(lam / len(coll))) < 4.5
    assert abs(coll.var() / lam - 1.0) < 0.05
    for r in runs:
        assert r["final_by_type"][oracle.ORC_CUTOFF] == N
    # collision density 1/E below the source: flux per bin = ln(E_b+1/E_b)/Sigma_t
    flux = np.array([r["energy"] for r in runs])
    mean, se = flux.mean(0), flux.std(0, ddof=1) / math.sqrt(len(runs))
    ref = np.log(p.energy_edges[1:] / p.energy_edges[:-1]) / sig
    assert np.all(np.abs(mean - ref) < 5 * se + 1e-9), (mean, ref)


def test_capture_branching_ratio():
    # constant elastic = capture on hydrogen: each collision absorbs with probability 1/2
    p = inputs.ce_box(A=1.0, sigma_el=10.0, sigma_cap=10.0, energy=1e6, cutoff=1e-5)
    N = 40000
    r = oracle.run_fixed_source(p, N, seed=2, per_history=True)
    k = r["hist_coll"].astype(float)
    assert _z(k.mean(), 2.0, k.std() / math.sqrt(N)) < 4.5
    assert r["final_by_type"][oracle.ORC_ABSORB] + r["final_by_type"][oracle.ORC_CUTOFF] == N


def _mesh_problem():
    p = inputs.cube_one_group()
    p.mesh_lo, p.mesh_hi, p.mesh_n = (1.0, -2.0, 0.5), (9.0, 7.0, 4.5), (7, 5, 3)
    return p


def _inside_length(lo, hi, p0, d, L):
    # slab method written with numpy for the whole mesh box
    t0, t1 = 0.0, L
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] <= p0[a] < hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - p0[a]) / d[a], (hi[a] - p0[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def test_mesh_clipping_lengths():
    p = _mesh_problem()
    rng = np.random.default_rng(11)
    lo, hi = np.array(p.mesh_lo), np.array(p.mesh_hi)
    for _ in range(300):
        p0 = rng.uniform(-1, 11, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        L = rng.uniform(0, 15)
        m = oracle.mesh_segment(p, p0, d, L)
        inside = _inside_length(lo, hi, p0, d, L)
        assert abs(m.sum() - inside) <= 1e-12 * max(1.0, L)
        assert np.all(m >= 0)
    # dense point sampling along a few segments (independent of slab clipping)
    n = p.mesh_n
    w = (hi - lo) / np.array(n)
    for _ in range(5):
        p0 = rng.uniform(lo, hi)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        L = 6.0
        m = oracle.mesh_segment(p, p0, d, L)
        K = 400_000
        t = (np.arange(K) + 0.5) * (L / K)
        pts = p0[None, :] + t[:, None] * d[None, :]
        ok = np.all((pts >= lo) & (pts < hi), axis=1)
        idx = np.floor((pts[ok] - lo) / w).astype(int)
        lin = (idx[:, 2] * n[1] + idx[:, 1]) * n[0] + idx[:, 0]
        ref = np.bincount(lin, minlength=int(np.prod(n))) * (L / K)
        assert np.all(np.abs(m - ref) < 3 * L / K + 1e-12)
    # an axis-parallel segment inside one row of voxels: closed-form pieces
    m = oracle.mesh_segment(p, (1.5, 0.1, 1.0), (1.0, 0.0, 0.0), 5.0)
    iy = int((0.1 - lo[1]) // w[1])
    row = m.reshape(n[2], n[1], n[0])[0, iy]
    assert m.sum() == pytest.approx(5.0, abs=1e-13)
    wx = w[0]
    expect = np.clip(np.minimum(6.5, lo[0] + wx * np.arange(1, 8)) - np.maximum(1.5, lo[0] + wx * np.arange(7)), 0, None)
    assert np.allclose(row, expect, rtol=0, atol=1e-13)


def test_lattice_conservation_and_bank_population():
    p = inputs.c5g7_lattice()
    N = 5000
    r = oracle.run_fixed_source(p, N, seed=1)
    fb = r["final_by_type"]
    assert fb.sum() == N and fb[oracle.ORC_ABSORB] + fb[oracle.ORC_LEAK] == N
    assert r["log_n"].min() >= 2
    # the mesh covers the whole domain: its sum is the total track length
    assert abs(r["mesh"].sum() - r["scalars"][0]) <= 1e-10 * r["scalars"][0]
    # every surface event and collision was counted once
    ev = r["events_by_type"]
    assert ev[oracle.ORC_SOURCE] == N
    assert int(r["log_n"].sum()) == int(ev.sum())
    # splitting roulette: E[N_{b+1}] = N with Var = M f (1 - f)
    e = oracle.power_iteration(p, 3000, 6, 2, seed=4)
    ns, ms = e["n_source"].astype(float), e["n_sites"].astype(float)
    zs = []
    for b in range(len(ns) - 1):
        r_ = 3000.0 / ms[b]
        f = r_ - math.floor(r_)
        zs.append((ns[b + 1] - 3000.0) / math.sqrt(max(ms[b] * f * (1 - f), 1e-9)))
        assert math.floor(r_) * ms[b] <= ns[b + 1] <= math.ceil(r_) * ms[b]
    assert max(abs(z) for z in zs) < 5
    # k follows k_b = k_{b-1} M / N exactly
    kprev = 1.0
    for b in range(len(ns)):
        assert e["k_batch"][b] == kprev * (ms[b] / ns[b])
        kprev = e["k_batch"][b]


def test_ce_pin_cell_conservation():
    p = inputs.ce_pin_cell(n_points=20000, n_res=60)
    N = 2000
    r = oracle.run_fixed_source(p, N, seed=1)
    fb = r["final_by_type"]
    assert fb.sum() == N and fb[oracle.ORC_ABSORB] + fb[oracle.ORC_CUTOFF] == N
    # energy edges span the whole grid: per-material energy tally sums to the flux
    assert abs(r["energy"].sum() - r["scalars"][0]) <= 1e-10 * r["scalars"][0]
    assert r["energy"].reshape(2, -1).sum(1).min() > 0


def _pin_cell(sig_pin, sig_mod, bc, b, z_half=5.0):
    half = 0.63
    p = inputs.box_mg("pin", (-half, -half, -z_half), (half, half, z_half), sigma_t=[sig_pin], sigma_s=[[0.0]],
                      bc=bc, mesh_n=(9, 1, 1))
    p.n_materials = 2
    p.sigma_t = np.array([[sig_pin], [sig_mod]])
    p.sigma_s = np.zeros((2, 1, 1))
    p.nu_sigma_f = np.zeros((2, 1))
    p.chi = np.ones((2, 1))
    p.cell_material = np.ones((1, 1, 1), np.int32)
    p.pin_material = np.zeros((1, 1, 1), np.int32)
    p.pin_radius = 0.54
    p.src_materials = np.ones(2, np.uint8)
    p.src_kind, p.src_point, p.src_direction, p.src_group = inputs.SRC_POINT, (-half, b, 0.25), (1.0, 0.0, 0.0), 0
    return p


@pytest.mark.parametrize("b", [0.0, 0.3, 0.5, 0.6])
def test_pin_chord_transmission(b):
    # pencil beam across a pin cell: transmission exp(-S_mod (1.26 - c) - S_pin c), chord c = 2 sqrt(r^2 - b^2)
    sp, sm, r = 2.0, 0.5, 0.54
    bc = [inputs.BC_VACUUM, inputs.BC_VACUUM, inputs.BC_REFLECT, inputs.BC_REFLECT, inputs.BC_REFLECT,
          inputs.BC_REFLECT]
    p = _pin_cell(sp, sm, np.array(bc, np.int32), b)
    N = 200_000
    res = oracle.run_fixed_source(p, N, seed=17)
    chord = 2.0 * math.sqrt(max(r * r - b * b, 0.0))
    pt = math.exp(-sm * (1.26 - chord) - sp * chord)
    leak = res["final_by_type"][oracle.ORC_LEAK] / N
    assert _z(leak, pt, math.sqrt(pt * (1 - pt) / N)) < 4.5
    # the track-length scalar equals the expected path: integral of survival along x
    x0, x1 = 0.63 - chord / 2, 0.63 + chord / 2
    def surv_int(a, c, s, base):  # integral over [a, c] of exp(-(base + s (x - a)))
        return math.exp(-base) * (1 - math.exp(-s * (c - a))) / s
    e1 = surv_int(0.0, x0, sm, 0.0)
    e2 = surv_int(x0, x1, sp, sm * x0) if chord > 0 else 0.0
    e3 = surv_int(x1, 1.26, sm, sm * x0 + sp * chord)
    mean_len = e1 + e2 + e3
    assert abs(res["scalars"][0] - mean_len) < 5 * math.sqrt(1.26 * mean_len / N)


def test_homogenised_lattice_is_infinite_medium():
    # every material equal and every face reflective: the lattice is an infinite
    # medium, so flux = 1/Sigma_a and track length ~ Exp(Sigma_a) despite thousands
    # of surface crossings (a lost or doubled segment would show here)
    p = inputs.c5g7_lattice()
    M = p.n_materials
    p = p.replace(n_groups=1, sigma_t=np.ones((M, 1)), sigma_s=np.full((M, 1, 1), 0.8),
                  nu_sigma_f=np.zeros((M, 1)), chi=np.ones((M, 1)), src_group=0,
                  bc=np.full(6, inputs.BC_REFLECT, np.int32))
    N = 20000
    r = oracle.run_fixed_source(p, N, seed=8, per_history=True)
    tr = r["hist_track"]
    assert _z(tr.mean(), 5.0, tr.std() / math.sqrt(N)) < 4.5
    assert stats.kstest(tr, stats.expon(scale=5.0).cdf).pvalue > 1e-4
    ev = r["events_by_type"]
    assert ev[oracle.ORC_SURF_INTERNAL] > 5 * N and ev[oracle.ORC_SURF_REFLECT] > 0
    assert abs(r["mesh"].sum() - r["scalars"][0]) <= 1e-10 * r["scalars"][0]


def test_ce_macroscopic_cross_sections_interpolate_linearly():
    """The continuous-energy lookup is linear interpolation in energy on each
    nuclide's own grid, weighted by the material's densities: against
    numpy's interp at random energies (inside every grid) and exactly at grid
    points, for sigma_t and sigma_a (capture + fission)."""
    p = inputs.ce_pin_cell(n_points=2000, n_res=20, n_ebins=10)
    lo = max(e[0] for e in p.nuc_energy)
    hi = min(e[-1] for e in p.nuc_energy)
    rng = np.random.default_rng(5)
    energies = list(np.exp(rng.uniform(math.log(lo), math.log(hi), 300)))
    energies += [float(p.nuc_energy[0][k]) for k in (1, 500, 1999)]
    for m in range(p.n_materials):
        for E in energies:
            ref_t = ref_a = 0.0
            for n, (e, s) in enumerate(zip(p.nuc_energy, p.nuc_sigma)):
                N = p.mat_density[m, n]
                if N <= 0.0:
                    continue
                sig = [np.interp(E, e, s[:, r]) for r in range(3)]
                ref_t += N * sum(sig)
                ref_a += N * (sig[1] + sig[2])
            st, sa = oracle.ce_macro(p, m, E)
            assert abs(st - ref_t) <= 1e-12 * ref_t, (m, E, st, ref_t)
            assert abs(sa - ref_a) <= 1e-12 * ref_a + 1e-300, (m, E, sa, ref_a)
