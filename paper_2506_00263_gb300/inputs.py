"""Seeded synthetic problem descriptions (inputs only).

This module builds the data that both the CUDA library and the CPU oracle
consume: geometry planes and cell maps, multigroup or continuous-energy cross
sections, the source definition and the tally definitions.  It contains no
transport arithmetic: nothing here samples a history, computes a distance,
looks up a cross section or scores a tally.  Every random draw uses numpy's
PCG64 generator with the stated seed, so a given builder call always yields the
same arrays.

Workloads (the paper runs 3D C5G7 k-eigenvalue and a continuous-energy
infinite pin cell, Sec. 4; their real geometry map and nuclear data are not
available, so these are synthetic stand-ins with the same structure):

* ``cube_one_group``: 10 cm reflective cube, one group, point source (Sec. 4 uses
  no such problem; it is the closed-form check case).
* ``c5g7_lattice``: 2x2 assemblies of 17x17 pins, 7 groups, axial and radial
  reflector, stand-in for the 3D C5G7 benchmark of Sec. 4 / Sec. 5.1.
* ``ce_pin_cell``: continuous-energy infinite pin cell with four synthetic
  nuclides, stand-in for the problem of Sec. 4 / Sec. 5.2.
* ``batched_boxes``: many voxelised box problems of uneven sizes.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# Boundary-condition codes per domain face (x-, x+, y-, y+, z-, z+).
BC_VACUUM = 0
BC_REFLECT = 1

# Source kinds.
SRC_POINT = 0  # fixed point, isotropic or given direction
SRC_BOX = 1    # uniform in an axis-aligned box
SRC_PINS = 2   # uniform in the pins whose material is flagged as a source material

XS_MG = 0
XS_CE = 1


@dataclass
class Problem:
    """One fixed-source or eigenvalue problem, as plain arrays.

    Geometry is a rectilinear grid of cells (planes ``x_planes``, ``y_planes``,
    ``z_planes``); each cell has an outer material and optionally a z-aligned
    cylinder ("pin") of radius ``pin_radius`` centred in the cell's x-y box with
    its own material.  ``pin_material[k, j, i] < 0`` means no pin.
    """

    name: str
    x_planes: np.ndarray
    y_planes: np.ndarray
    z_planes: np.ndarray
    bc: np.ndarray                 # (6,) int32
    cell_material: np.ndarray      # (nz, ny, nx) int32
    pin_material: np.ndarray       # (nz, ny, nx) int32, -1 = no pin
    pin_radius: float
    xs_kind: int
    n_materials: int
    # multigroup data: [m][g], [m][g][g'] (from g to g'), [m][g], [m][g]
    n_groups: int = 1
    sigma_t: Optional[np.ndarray] = None
    sigma_s: Optional[np.ndarray] = None
    nu_sigma_f: Optional[np.ndarray] = None
    chi: Optional[np.ndarray] = None
    # continuous-energy data
    nuc_energy: list = field(default_factory=list)   # per nuclide (K,) eV ascending
    nuc_sigma: list = field(default_factory=list)    # per nuclide (K, 3) barns: elastic, capture, fission
    nuc_awr: Optional[np.ndarray] = None             # (n_nuc,) target mass ratio A
    mat_density: Optional[np.ndarray] = None         # (n_materials, n_nuc) atoms / (barn cm)
    energy_cutoff: float = 1e-5
    # source
    src_kind: int = SRC_POINT
    src_point: tuple = (0.0, 0.0, 0.0)
    src_direction: Optional[tuple] = None            # None = isotropic
    src_lo: tuple = (0.0, 0.0, 0.0)
    src_hi: tuple = (0.0, 0.0, 0.0)
    src_group: int = 0                               # MG: fixed group, or -1 = sample chi
    src_materials: Optional[np.ndarray] = None       # (n_materials,) uint8 flags for SRC_PINS
    src_energy: float = 1e6                          # CE: mono-energetic source energy
    src_cdf_energy: Optional[np.ndarray] = None      # CE: tabulated CDF abscissae (eV)
    src_cdf_prob: Optional[np.ndarray] = None        # CE: CDF values, 0 .. 1
    # tallies
    mesh_lo: Optional[tuple] = None
    mesh_hi: Optional[tuple] = None
    mesh_n: Optional[tuple] = None
    mesh_by_group: bool = False
    energy_edges: Optional[np.ndarray] = None        # CE energy-bin tally, per material
    # time: histories start at t = 0 and end at the census time t_census (0 =
    # untimed); multigroup speeds from inv_velocity (G,) s/cm; n_time_bins
    # uniform flux bins over [0, t_census)
    inv_velocity: Optional[np.ndarray] = None
    n_time_bins: int = 0
    t_census: float = 0.0
    # weight windows (fixed source; None = analog): lower bound per tally-mesh
    # voxel and group, (mesh voxels, G) with 0 = no window; upper bound and
    # roulette survival weight as multiples of it; most copies per split
    ww_lower: Optional[np.ndarray] = None
    ww_upper: float = 5.0
    ww_survival: float = 3.0
    ww_max_split: int = 16

    @property
    def shape(self):
        return (len(self.z_planes) - 1, len(self.y_planes) - 1, len(self.x_planes) - 1)

    @property
    def mesh_size(self) -> int:
        if self.mesh_n is None:
            return 0
        n = int(np.prod(self.mesh_n))
        return n * (self.n_groups if (self.mesh_by_group and self.xs_kind == XS_MG) else 1)

    @property
    def energy_size(self) -> int:
        if self.energy_edges is None:
            return 0
        return self.n_materials * (len(self.energy_edges) - 1)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# --------------------------------------------------------------------------
# Small closed-form problems
# --------------------------------------------------------------------------

def box_mg(name, lo, hi, sigma_t, sigma_s, nu_sigma_f=None, chi=None, bc=BC_REFLECT,
           mesh_n=None, mesh_by_group=False, **src) -> Problem:
    """Homogeneous box of one material with G groups (G = len(sigma_t))."""
    sigma_t = _f64(sigma_t).reshape(1, -1)
    G = sigma_t.shape[1]
    sigma_s = _f64(sigma_s).reshape(1, G, G)
    nu_sigma_f = _f64(np.zeros((1, G)) if nu_sigma_f is None else nu_sigma_f).reshape(1, G)
    chi = _f64(np.eye(1, G) if chi is None else chi).reshape(1, G)
    bcs = np.full(6, bc, dtype=np.int32) if np.isscalar(bc) else _i32(bc)
    p = Problem(
        name=name,
        x_planes=_f64([lo[0], hi[0]]), y_planes=_f64([lo[1], hi[1]]), z_planes=_f64([lo[2], hi[2]]),
        bc=bcs, cell_material=np.zeros((1, 1, 1), np.int32), pin_material=-np.ones((1, 1, 1), np.int32),
        pin_radius=0.0, xs_kind=XS_MG, n_materials=1, n_groups=G,
        sigma_t=sigma_t, sigma_s=sigma_s, nu_sigma_f=nu_sigma_f, chi=chi,
        src_materials=np.ones(1, np.uint8),
    )
    if mesh_n is not None:
        p.mesh_lo, p.mesh_hi, p.mesh_n, p.mesh_by_group = tuple(lo), tuple(hi), tuple(mesh_n), mesh_by_group
    for k, v in src.items():
        setattr(p, k, v)
    return p


def cube_one_group(n_mesh: int = 16) -> Problem:
    """10 cm reflective cube, sigma_t = 1/cm, scatter ratio 0.5, no fission,
    isotropic point source at the centre, 16^3 track-length flux mesh."""
    return box_mg("cube_one_group", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0),
                  sigma_t=[1.0], sigma_s=[[0.5]], bc=BC_REFLECT,
                  mesh_n=(n_mesh, n_mesh, n_mesh),
                  src_kind=SRC_POINT, src_point=(5.0, 5.0, 5.0), src_direction=None, src_group=0)


# --------------------------------------------------------------------------
# C5G7-shaped 7-group lattice (synthetic data)
# --------------------------------------------------------------------------

C5G7_PITCH = 1.26
C5G7_RADIUS = 0.54
C5G7_NPIN = 34            # 2 assemblies x 17 pins per side
C5G7_FUEL = 42.84         # 34 * 1.26
C5G7_DOMAIN = 64.26       # fuel block + 21.42 cm reflector
MAT_FUEL1, MAT_FUEL2, MAT_FUEL3, MAT_FUEL4, MAT_MOD, MAT_GT, MAT_FC = range(7)


def c5g7_xs(seed: int = 2025, G: int = 7, n_mat: int = 7, n_fuel: int = 4):
    """Synthetic 7-group cross sections.

    sigma_t ~ U(0.2, 2.0); scatter ratio c ~ U(0.3, 0.95) per (material, group);
    scatter row weights U(0, 1) on g' >= g plus upscatter only from the last
    group to the one before it; rows scaled to c * sigma_t; fuel
    nu_sigma_f = 2.5 f sigma_a with f ~ U(0.2, 0.6); fuel chi proportional to
    U(0, 1) on the first three groups.  Non-fuel materials have no fission.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    st = rng.uniform(0.2, 2.0, size=(n_mat, G))
    c = rng.uniform(0.3, 0.95, size=(n_mat, G))
    ss = np.zeros((n_mat, G, G))
    for m in range(n_mat):
        for g in range(G):
            w = np.zeros(G)
            w[g:] = rng.uniform(0.0, 1.0, size=G - g)
            if G >= 2 and g == G - 1:
                w[G - 2] = rng.uniform(0.0, 1.0)   # upscatter between the two last groups
            w = w / w.sum()
            ss[m, g, :] = c[m, g] * st[m, g] * w
    nsf = np.zeros((n_mat, G))
    chi = np.zeros((n_mat, G))
    for m in range(n_fuel):
        f = rng.uniform(0.2, 0.6, size=G)
        nsf[m] = 2.5 * f * (1.0 - c[m]) * st[m]
        x = np.zeros(G)
        x[: min(3, G)] = rng.uniform(0.0, 1.0, size=min(3, G))
        chi[m] = x / x.sum()
    return st, ss, nsf, chi


def c5g7_pin_map() -> np.ndarray:
    """(34, 34) pin materials [j][i]: synthetic guide-tube rule (local indices in
    {2,5,8,11,14}^2 are guide tubes, the centre (8,8) is the fission chamber);
    assemblies (0,0),(1,1) are fuel-1; (0,1),(1,0) have fuel-2 on the outer ring,
    fuel-3 on the next two rings and fuel-4 inside."""
    pm = np.zeros((C5G7_NPIN, C5G7_NPIN), np.int32)
    gt = {2, 5, 8, 11, 14}
    for j in range(C5G7_NPIN):
        for i in range(C5G7_NPIN):
            ai, aj = i // 17, j // 17
            li, lj = i % 17, j % 17
            if li in gt and lj in gt:
                pm[j, i] = MAT_FC if (li == 8 and lj == 8) else MAT_GT
            elif ai == aj:
                pm[j, i] = MAT_FUEL1
            else:
                ring = min(li, lj, 16 - li, 16 - lj)
                pm[j, i] = MAT_FUEL2 if ring == 0 else (MAT_FUEL3 if ring <= 2 else MAT_FUEL4)
    return pm


def c5g7_lattice(xs_seed: int = 2025, fission: bool = True, mesh: bool = True) -> Problem:
    """C5G7-shaped 3D lattice (``fission=False`` only renames it: fixed-source
    runs never bank fission sites, nu_sigma_f stays as data for the production
    tally): 35x35x2 grid cells (34x34 pin cells plus one
    radial reflector slab per axis; fuel height 42.84 cm plus a 21.42 cm axial
    reflector).  Reflective at x=0, y=0, z=0; vacuum at 64.26 cm.  Source
    uniform in the fuel pins (materials 0-3) with the group from chi."""
    xp = np.concatenate([np.arange(C5G7_NPIN + 1) * C5G7_PITCH, [C5G7_DOMAIN]])
    zp = np.array([0.0, C5G7_FUEL, C5G7_DOMAIN])
    nx = len(xp) - 1
    cell = np.full((2, nx, nx), MAT_MOD, np.int32)
    pin = -np.ones((2, nx, nx), np.int32)
    pin[0, :C5G7_NPIN, :C5G7_NPIN] = c5g7_pin_map()
    st, ss, nsf, chi = c5g7_xs(xs_seed)
    p = Problem(
        name="c5g7_lattice" if fission else "c5g7_lattice_nofission",
        x_planes=_f64(xp), y_planes=_f64(xp), z_planes=_f64(zp),
        bc=_i32([BC_REFLECT, BC_VACUUM, BC_REFLECT, BC_VACUUM, BC_REFLECT, BC_VACUUM]),
        cell_material=cell, pin_material=pin, pin_radius=C5G7_RADIUS,
        xs_kind=XS_MG, n_materials=7, n_groups=7,
        sigma_t=_f64(st), sigma_s=_f64(ss), nu_sigma_f=_f64(nsf), chi=_f64(chi),
        src_kind=SRC_PINS, src_lo=(0.0, 0.0, 0.0), src_hi=(C5G7_FUEL, C5G7_FUEL, C5G7_FUEL),
        src_group=-1, src_materials=np.array([1, 1, 1, 1, 0, 0, 0], np.uint8),
    )
    if mesh:
        p.mesh_lo, p.mesh_hi, p.mesh_n = (0.0, 0.0, 0.0), (C5G7_DOMAIN,) * 3, (51, 51, 1)
    return p


# --------------------------------------------------------------------------
# Continuous-energy infinite pin cell (synthetic nuclides)
# --------------------------------------------------------------------------

CE_EMIN, CE_EMAX = 1e-5, 2e7
# name, A, potential elastic (b), capture at 0.0253 eV (b), fission at 0.0253 eV (b)
CE_NUCLIDES = (
    ("F1", 235.0, 11.5, 98.0, 585.0),
    ("F2", 238.0, 11.3, 2.7, 0.0),
    ("O", 16.0, 3.8, 0.0002, 0.0),
    ("H", 1.0, 20.4, 0.33, 0.0),
)


def ce_nuclide(k: int, rng, n_points: int, n_res: int, fissile: bool, pot: float, cap0: float, fis0: float):
    """One synthetic nuclide: log-spaced grid on [1e-5, 2e7] eV shifted by k/4
    of a log step (endpoints kept), elastic = potential + Lorentzian resonances,
    capture and fission = 1/sqrt(E) backgrounds + Lorentzian resonances
    (single-level Breit-Wigner shapes at 0 K without interference)."""
    lo, hi = np.log(CE_EMIN), np.log(CE_EMAX)
    h = (hi - lo) / (n_points - 1)
    inner = lo + (np.arange(1, n_points - 1) + 0.25 * k) * h
    inner = inner[inner < hi]
    E = np.concatenate([[CE_EMIN], np.exp(inner), [CE_EMAX]])
    E = np.unique(E)
    e0 = np.exp(rng.uniform(np.log(1.0), np.log(1e4), size=n_res))
    gam = np.exp(rng.uniform(np.log(0.02), np.log(0.5), size=n_res))
    peak = np.exp(rng.uniform(np.log(10.0), np.log(1e4), size=n_res))
    frac_n = rng.uniform(0.1, 0.9, size=n_res)
    frac_f = rng.uniform(0.0, 0.6, size=n_res) * (1.0 if fissile else 0.0)
    frac_g = 1.0 - frac_n - frac_f * (1.0 - frac_n)
    frac_f = frac_f * (1.0 - frac_n)
    el = np.full_like(E, pot)
    cap = cap0 * np.sqrt(0.0253 / E)
    fis = fis0 * np.sqrt(0.0253 / E)
    # accumulate resonances in chunks to bound memory
    for s in range(0, n_res, 32):
        x = 2.0 * (E[:, None] - e0[None, s:s + 32]) / gam[None, s:s + 32]
        shape = 1.0 / (1.0 + x * x)
        sq = np.sqrt(e0[None, s:s + 32] / E[:, None])
        el += (peak[None, s:s + 32] * frac_n[None, s:s + 32] * shape).sum(axis=1)
        cap += (peak[None, s:s + 32] * np.clip(frac_g[None, s:s + 32], 0.0, 1.0) * shape * sq).sum(axis=1)
        fis += (peak[None, s:s + 32] * frac_f[None, s:s + 32] * shape * sq).sum(axis=1)
    sig = np.stack([el, cap, fis if fissile else np.zeros_like(E)], axis=1)
    return _f64(E), _f64(sig)


def watt_cdf(n: int = 4001, a_mev: float = 0.988, b_per_mev: float = 2.249):
    """Tabulated CDF of p(E) ~ exp(-E/a) sinh(sqrt(b E)) on [1e-5 eV, 20 MeV]."""
    E = np.linspace(0.0, CE_EMAX, n)
    E[0] = CE_EMIN
    x = E * 1e-6
    pdf = np.exp(-x / a_mev) * np.sinh(np.sqrt(b_per_mev * x))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(x))])
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    return _f64(E), _f64(cdf)


def ce_pin_cell(seed: int = 11, n_points: int = 100_000, n_res: int = 300, n_ebins: int = 100,
                source_energy: Optional[float] = None) -> Problem:
    """Continuous-energy infinite pin cell: fuel cylinder r = 0.4 cm in a
    1.26 cm reflective square, z unbounded; fuel = F1 + F2 + O, moderator = H + O;
    source uniform in the fuel, energies from a Watt-like spectrum (or mono-
    energetic if ``source_energy`` is given); energy tally per material."""
    rng = np.random.Generator(np.random.PCG64(seed))
    E_list, S_list = [], []
    for k, (_, A, pot, cap0, fis0) in enumerate(CE_NUCLIDES):
        E, S = ce_nuclide(k, rng, n_points, n_res, fis0 > 0.0, pot, cap0, fis0)
        E_list.append(E)
        S_list.append(S)
    awr = _f64([n[1] for n in CE_NUCLIDES])
    dens = _f64([[5.7e-4, 2.3e-2, 4.7e-2, 0.0],      # fuel
                 [0.0, 0.0, 3.35e-2, 6.7e-2]])       # moderator
    half = 0.63
    cdfE, cdfP = watt_cdf()
    p = Problem(
        name="ce_pin_cell",
        x_planes=_f64([-half, half]), y_planes=_f64([-half, half]), z_planes=_f64([-np.inf, np.inf]),
        bc=_i32([BC_REFLECT, BC_REFLECT, BC_REFLECT, BC_REFLECT, BC_VACUUM, BC_VACUUM]),
        cell_material=np.ones((1, 1, 1), np.int32), pin_material=np.zeros((1, 1, 1), np.int32),
        pin_radius=0.4, xs_kind=XS_CE, n_materials=2, n_groups=1,
        nuc_energy=E_list, nuc_sigma=S_list, nuc_awr=awr, mat_density=dens, energy_cutoff=CE_EMIN,
        src_kind=SRC_PINS, src_lo=(-0.4, -0.4, 0.0), src_hi=(0.4, 0.4, 0.0),
        src_materials=np.array([1, 0], np.uint8),
        src_cdf_energy=None if source_energy else cdfE, src_cdf_prob=None if source_energy else cdfP,
        src_energy=float(source_energy or 1e6),
        energy_edges=_f64(np.logspace(np.log10(CE_EMIN), np.log10(CE_EMAX), n_ebins + 1)),
    )
    return p


def ce_box(A: float, sigma_el: float, sigma_cap: float, energy: float, cutoff: float = 1.0,
           n_points: int = 64, half: float = 50.0) -> Problem:
    """One-nuclide constant-cross-section reflective box (infinite medium) for
    slowing-down checks; density 1 atom/(barn cm) so Sigma = sigma."""
    E = _f64(np.logspace(np.log10(CE_EMIN), np.log10(CE_EMAX), n_points))
    S = np.zeros((n_points, 3))
    S[:, 0], S[:, 1] = sigma_el, sigma_cap
    return Problem(
        name="ce_box",
        x_planes=_f64([-half, half]), y_planes=_f64([-half, half]), z_planes=_f64([-half, half]),
        bc=np.full(6, BC_REFLECT, np.int32), cell_material=np.zeros((1, 1, 1), np.int32),
        pin_material=-np.ones((1, 1, 1), np.int32), pin_radius=0.0, xs_kind=XS_CE, n_materials=1,
        nuc_energy=[E], nuc_sigma=[_f64(S)], nuc_awr=_f64([A]), mat_density=_f64([[1.0]]),
        energy_cutoff=cutoff, src_kind=SRC_POINT, src_point=(0.0, 0.0, 0.0), src_energy=energy,
        src_materials=np.ones(1, np.uint8),
    )


# --------------------------------------------------------------------------
# Batched voxel boxes
# --------------------------------------------------------------------------

def voxel_box(rng, G: int, n_mat: int, nvox: tuple, mesh_n: int, size: float = 20.0, name="voxel_box") -> Problem:
    """Vacuum box split into a voxel grid with a random material per voxel
    (C5G7-style synthetic group constants); uniform volumetric source with the
    group sampled from the problem's chi."""
    st, ss, nsf, chi = c5g7_xs(int(rng.integers(1 << 31)), G=G, n_mat=n_mat, n_fuel=n_mat)
    nx, ny, nz = nvox
    p = Problem(
        name=name,
        x_planes=_f64(np.linspace(0.0, size, nx + 1)), y_planes=_f64(np.linspace(0.0, size, ny + 1)),
        z_planes=_f64(np.linspace(0.0, size, nz + 1)), bc=np.full(6, BC_VACUUM, np.int32),
        cell_material=_i32(rng.integers(0, n_mat, size=(nz, ny, nx))),
        pin_material=-np.ones((nz, ny, nx), np.int32), pin_radius=0.0, xs_kind=XS_MG,
        n_materials=n_mat, n_groups=G, sigma_t=_f64(st), sigma_s=_f64(ss), nu_sigma_f=_f64(nsf), chi=_f64(chi),
        src_kind=SRC_BOX, src_lo=(0.0, 0.0, 0.0), src_hi=(size, size, size), src_group=-1,
        src_materials=np.ones(n_mat, np.uint8),
        mesh_lo=(0.0, 0.0, 0.0), mesh_hi=(size, size, size), mesh_n=(mesh_n,) * 3,
    )
    return p


def batched_boxes(n_problems: int = 256, seed: int = 7, max_vox: int = 64, max_hist: int = 1_000_000,
                  min_hist: int = 1000):
    """(problems, histories): group counts from {1,2,7,20,70}, 1-8 materials,
    voxel layout up to max_vox^3, histories log-uniform in [min_hist, max_hist],
    tally mesh 8^3 - 32^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs, hist = [], []
    for b in range(n_problems):
        G = int(rng.choice([1, 2, 7, 20, 70]))
        n_mat = int(rng.integers(1, 9))
        nv = tuple(int(v) for v in rng.integers(1, max_vox + 1, size=3))
        mesh_n = int(rng.choice([8, 16, 32]))
        probs.append(voxel_box(rng, G, n_mat, nv, mesh_n, name=f"box{b}"))
        hist.append(int(np.exp(rng.uniform(np.log(min_hist), np.log(max_hist)))))
    return probs, hist
