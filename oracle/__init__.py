"""CPU oracle for the event-based Monte Carlo transport path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it; ``oracle.c`` implements the
arithmetic contract on its own.

``run_fixed_source`` and ``power_iteration`` take a
``paper_2506_00263_gb300.inputs.Problem`` (plain arrays) and return numpy
results.  The C library is built with ``gcc -O2 -ffp-contract=off`` so every
floating-point operation is a single IEEE-754 binary64 operation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ORC_SOURCE, ORC_SCATTER, ORC_ABSORB, ORC_SURF_INTERNAL, ORC_SURF_REFLECT, ORC_LEAK, ORC_CUTOFF, ORC_MAXEV = range(8)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, contraction off)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcProblem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("xp", C.POINTER(C.c_double)), ("yp", C.POINTER(C.c_double)), ("zp", C.POINTER(C.c_double)),
        ("bc", C.c_int32 * 6),
        ("cell_mat", C.POINTER(C.c_int32)), ("pin_mat", C.POINTER(C.c_int32)),
        ("pin_r", C.c_double),
        ("xs_kind", C.c_int32), ("n_mat", C.c_int32), ("n_grp", C.c_int32),
        ("sigt", C.POINTER(C.c_double)), ("sigs", C.POINTER(C.c_double)),
        ("nusigf", C.POINTER(C.c_double)), ("chi", C.POINTER(C.c_double)),
        ("n_nuc", C.c_int32),
        ("nuc_off", C.POINTER(C.c_int64)),
        ("nuc_e", C.POINTER(C.c_double)), ("nuc_sig", C.POINTER(C.c_double)),
        ("nuc_awr", C.POINTER(C.c_double)), ("mat_dens", C.POINTER(C.c_double)),
        ("e_cut", C.c_double),
        ("src_kind", C.c_int32), ("src_iso", C.c_int32), ("src_group", C.c_int32), ("n_cdf", C.c_int32),
        ("src_pt", C.c_double * 3), ("src_dir", C.c_double * 3), ("src_lo", C.c_double * 3),
        ("src_hi", C.c_double * 3), ("src_energy", C.c_double),
        ("src_mat", C.POINTER(C.c_uint8)),
        ("cdf_e", C.POINTER(C.c_double)), ("cdf_p", C.POINTER(C.c_double)),
        ("has_mesh", C.c_int32), ("mesh_n", C.c_int32 * 3), ("mesh_by_group", C.c_int32),
        ("n_ebins", C.c_int32),
        ("mesh_lo", C.c_double * 3), ("mesh_hi", C.c_double * 3),
        ("e_edges", C.POINTER(C.c_double)),
        ("inv_vel", C.POINTER(C.c_double)), ("n_tbins", C.c_int32), ("t_cen", C.c_double),
        ("ww_lo", C.POINTER(C.c_double)), ("ww_upper", C.c_double), ("ww_survival", C.c_double),
        ("ww_max_split", C.c_int32),
    ]


class OrcFixed(C.Structure):
    _fields_ = [
        ("n_hist", C.c_uint64), ("seed", C.c_uint64), ("tag", C.c_uint32), ("max_events", C.c_uint32),
        ("id_offset", C.c_uint64),
        ("mesh", C.POINTER(C.c_double)), ("energy", C.POINTER(C.c_double)),
        ("log_n", C.POINTER(C.c_uint32)), ("log_cell", C.POINTER(C.c_int32)), ("log_type", C.POINTER(C.c_uint8)),
        ("hist_track", C.POINTER(C.c_double)), ("hist_coll", C.POINTER(C.c_uint32)),
        ("scalars", C.c_double * 3),
        ("events_by_type", C.c_uint64 * 8), ("final_by_type", C.c_uint64 * 8),
        ("time_tally", C.POINTER(C.c_double)),
    ]


class OrcEig(C.Structure):
    _fields_ = [
        ("n_per_batch", C.c_uint64), ("seed", C.c_uint64), ("bank_capacity", C.c_uint64),
        ("n_inactive", C.c_uint32), ("n_active", C.c_uint32), ("max_events", C.c_uint32),
        ("k0", C.c_double),
        ("k_batch", C.POINTER(C.c_double)), ("ktl_batch", C.POINTER(C.c_double)),
        ("n_source", C.POINTER(C.c_uint64)), ("n_sites", C.POINTER(C.c_uint64)),
        ("mesh_mean", C.POINTER(C.c_double)), ("mesh_std", C.POINTER(C.c_double)),
        ("energy_mean", C.POINTER(C.c_double)), ("energy_std", C.POINTER(C.c_double)),
        ("scalars_mean", C.c_double * 3), ("scalars_std", C.c_double * 3),
        ("k_mean", C.c_double), ("k_std", C.c_double),
        ("log_batch", C.c_uint32),
        ("log_n", C.POINTER(C.c_uint32)), ("log_cell", C.POINTER(C.c_int32)), ("log_type", C.POINTER(C.c_uint8)),
        ("log_count", C.c_uint64),
        ("events_by_type", C.c_uint64 * 8), ("final_by_type", C.c_uint64 * 8),
    ]


class OrcSens(C.Structure):
    _fields_ = [
        ("n_hist", C.c_uint64), ("seed", C.c_uint64), ("tag", C.c_uint32), ("max_events", C.c_uint32),
        ("g_mesh", C.POINTER(C.c_double)), ("g_scal", C.POINTER(C.c_double)),
        ("d_sigt", C.POINTER(C.c_double)), ("d_sigs", C.POINTER(C.c_double)), ("d_nusigf", C.POINTER(C.c_double)),
        ("value", C.c_double), ("id_offset", C.c_uint64),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.orc_fixed_source.argtypes = [C.POINTER(OrcProblem), C.POINTER(OrcFixed)]
        L.orc_fixed_source.restype = C.c_int
        L.orc_sensitivities.argtypes = [C.POINTER(OrcProblem), C.POINTER(OrcSens)]
        L.orc_sensitivities.restype = C.c_int
        L.orc_power_iteration.argtypes = [C.POINTER(OrcProblem), C.POINTER(OrcEig)]
        L.orc_power_iteration.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_uniform.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_uniform.restype = C.c_double
        L.orc_log.argtypes = [C.c_double]
        L.orc_log.restype = C.c_double
        L.orc_iso_dir.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]
        L.orc_exp_event.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32]
        L.orc_exp_event.restype = C.c_double
        L.orc_zig_table.argtypes = [C.POINTER(C.c_double)]
        L.orc_ce_macro.argtypes = [C.POINTER(OrcProblem), C.c_int, C.c_double, C.POINTER(C.c_double)]
        L.orc_ce_macro.restype = C.c_int
        L.orc_elastic.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_rotate.argtypes = [C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.orc_azimuth.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]
        L.orc_elastic_scatter.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_double, C.c_double,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_cdf_sample.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32, C.c_double]
        L.orc_cdf_sample.restype = C.c_double
        L.orc_mesh_segment.argtypes = [C.POINTER(OrcProblem), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.c_double, C.POINTER(C.c_double)]
        L.orc_mesh_segment.restype = C.c_double
        L.orc_nuclide_index.argtypes = [C.POINTER(C.c_double), C.c_int64, C.c_double]
        L.orc_nuclide_index.restype = C.c_int64
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


class _Marshalled:
    """Keeps the numpy buffers referenced by an OrcProblem alive."""

    def __init__(self, prob):
        self.keep = []
        s = OrcProblem()
        k = self.keep

        def f64(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            k.append(a)
            return _dp(a)

        def i32(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
            k.append(a)
            return _ip(a)

        s.nz, s.ny, s.nx = prob.shape
        s.xp, s.yp, s.zp = f64(prob.x_planes), f64(prob.y_planes), f64(prob.z_planes)
        for i in range(6):
            s.bc[i] = int(prob.bc[i])
        s.cell_mat, s.pin_mat = i32(prob.cell_material), i32(prob.pin_material)
        s.pin_r = float(prob.pin_radius)
        s.xs_kind, s.n_mat = int(prob.xs_kind), int(prob.n_materials)
        if prob.xs_kind == 0:
            s.n_grp = int(prob.n_groups)
            s.sigt, s.sigs = f64(prob.sigma_t), f64(prob.sigma_s)
            s.nusigf, s.chi = f64(prob.nu_sigma_f), f64(prob.chi)
        else:
            s.n_grp = 1
            s.n_nuc = len(prob.nuc_energy)
            off = np.zeros(s.n_nuc + 1, np.int64)
            off[1:] = np.cumsum([len(e) for e in prob.nuc_energy])
            offa = np.ascontiguousarray(off)
            k.append(offa)
            s.nuc_off = offa.ctypes.data_as(C.POINTER(C.c_int64))
            s.nuc_e = f64(np.concatenate(prob.nuc_energy))
            s.nuc_sig = f64(np.concatenate(prob.nuc_sigma, axis=0))
            s.nuc_awr, s.mat_dens = f64(prob.nuc_awr), f64(prob.mat_density)
            s.e_cut = float(prob.energy_cutoff)
        s.src_kind = int(prob.src_kind)
        s.src_iso = 1 if prob.src_direction is None else 0
        s.src_group = int(prob.src_group)
        for i in range(3):
            s.src_pt[i] = prob.src_point[i]
            s.src_lo[i], s.src_hi[i] = prob.src_lo[i], prob.src_hi[i]
            s.src_dir[i] = 0.0 if prob.src_direction is None else prob.src_direction[i]
        s.src_energy = float(prob.src_energy)
        sm = np.ascontiguousarray(np.asarray(prob.src_materials if prob.src_materials is not None
                                             else np.ones(prob.n_materials), dtype=np.uint8))
        k.append(sm)
        s.src_mat = sm.ctypes.data_as(C.POINTER(C.c_uint8))
        if prob.src_cdf_energy is not None:
            s.n_cdf = len(prob.src_cdf_energy)
            s.cdf_e, s.cdf_p = f64(prob.src_cdf_energy), f64(prob.src_cdf_prob)
        if prob.mesh_n is not None:
            s.has_mesh = 1
            for i in range(3):
                s.mesh_n[i] = int(prob.mesh_n[i])
                s.mesh_lo[i], s.mesh_hi[i] = prob.mesh_lo[i], prob.mesh_hi[i]
            s.mesh_by_group = 1 if prob.mesh_by_group else 0
        if prob.energy_edges is not None:
            s.n_ebins = len(prob.energy_edges) - 1
            s.e_edges = f64(prob.energy_edges)
        s.t_cen = float(getattr(prob, "t_census", 0.0) or 0.0)
        s.n_tbins = int(getattr(prob, "n_time_bins", 0) or 0)
        if getattr(prob, "inv_velocity", None) is not None:
            s.inv_vel = f64(prob.inv_velocity)
        if getattr(prob, "ww_lower", None) is not None:
            s.ww_lo = f64(prob.ww_lower)
            s.ww_upper, s.ww_survival = float(prob.ww_upper), float(prob.ww_survival)
            s.ww_max_split = int(prob.ww_max_split)
        self.s = s


def ce_macro(prob, m: int, E: float):
    """Macroscopic (sigma_t, sigma_a) of material m at energy E (continuous energy)."""
    mm = _Marshalled(prob)
    out = (C.c_double * 2)()
    if lib().orc_ce_macro(C.byref(mm.s), int(m), float(E), out) != 0:
        raise ValueError("orc_ce_macro failed")
    return out[0], out[1]


def run_fixed_source(prob, n_hist: int, seed: int = 1, tag: int = 0, max_events: int = 0, logs: bool = True,
                     per_history: bool = False, id_offset: int = 0) -> dict:
    """History-based fixed-source run of histories id_offset .. id_offset + n_hist - 1;
    tallies are means per source particle."""
    L = lib()
    m = _Marshalled(prob)
    o = OrcFixed()
    o.n_hist, o.seed, o.tag, o.max_events, o.id_offset = n_hist, seed, tag, max_events, id_offset
    out = {"mesh": np.zeros(prob.mesh_size), "energy": np.zeros(prob.energy_size),
           "time": np.zeros(int(getattr(prob, "n_time_bins", 0) or 0))}
    o.mesh, o.energy = _dp(out["mesh"]), _dp(out["energy"])
    o.time_tally = _dp(out["time"]) if out["time"].size else None
    if logs:
        out["log_n"] = np.zeros(n_hist, np.uint32)
        out["log_cell"] = np.zeros(n_hist, np.int32)
        out["log_type"] = np.zeros(n_hist, np.uint8)
        o.log_n = out["log_n"].ctypes.data_as(C.POINTER(C.c_uint32))
        o.log_cell = _ip(out["log_cell"])
        o.log_type = out["log_type"].ctypes.data_as(C.POINTER(C.c_uint8))
    if per_history:
        out["hist_track"] = np.zeros(n_hist)
        out["hist_coll"] = np.zeros(n_hist, np.uint32)
        o.hist_track = _dp(out["hist_track"])
        o.hist_coll = out["hist_coll"].ctypes.data_as(C.POINTER(C.c_uint32))
    st = L.orc_fixed_source(C.byref(m.s), C.byref(o))
    out["status"] = st
    out["scalars"] = np.array(o.scalars[:])
    out["events_by_type"] = np.array(o.events_by_type[:], np.uint64)
    out["final_by_type"] = np.array(o.final_by_type[:], np.uint64)
    return out


def sensitivities(prob, n_hist: int, g_mesh=None, g_scal=None, seed: int = 1, tag: int = 0,
                  max_events: int = 0, id_offset: int = 0) -> dict:
    """Score-function + pathwise derivatives of L = g . tallies with respect to
    sigma_t [m][g], sigma_s [m][g][g'] and nu_sigma_f [m][g]."""
    L = lib()
    m = _Marshalled(prob)
    o = OrcSens()
    o.n_hist, o.seed, o.tag, o.max_events, o.id_offset = n_hist, seed, tag, max_events, id_offset
    keep = []
    if g_mesh is not None:
        gm = np.ascontiguousarray(g_mesh, np.float64)
        keep.append(gm)
        o.g_mesh = _dp(gm)
    if g_scal is not None:
        gs = np.ascontiguousarray(g_scal, np.float64)
        keep.append(gs)
        o.g_scal = _dp(gs)
    M, G = prob.n_materials, prob.n_groups
    out = {"d_sigt": np.zeros((M, G)), "d_sigs": np.zeros((M, G, G)), "d_nusigf": np.zeros((M, G))}
    o.d_sigt, o.d_sigs, o.d_nusigf = _dp(out["d_sigt"]), _dp(out["d_sigs"]), _dp(out["d_nusigf"])
    out["status"] = L.orc_sensitivities(C.byref(m.s), C.byref(o))
    out["value"] = o.value
    return out


def power_iteration(prob, n_per_batch: int, n_inactive: int, n_active: int, seed: int = 1, k0: float = 1.0,
                    max_events: int = 0, log_batch: int = 0, bank_capacity: int = 0) -> dict:
    """k-eigenvalue power iteration with splitting-roulette population control."""
    L = lib()
    m = _Marshalled(prob)
    o = OrcEig()
    nb = n_inactive + n_active
    cap = bank_capacity or 4 * n_per_batch + 64
    o.n_per_batch, o.seed, o.bank_capacity = n_per_batch, seed, cap
    o.n_inactive, o.n_active, o.max_events, o.k0 = n_inactive, n_active, max_events, k0
    out = {"k_batch": np.zeros(nb), "ktl_batch": np.zeros(nb), "n_source": np.zeros(nb, np.uint64),
           "n_sites": np.zeros(nb, np.uint64), "mesh_mean": np.zeros(prob.mesh_size),
           "mesh_std": np.zeros(prob.mesh_size), "log_n": np.zeros(cap, np.uint32),
           "log_cell": np.zeros(cap, np.int32), "log_type": np.zeros(cap, np.uint8)}
    o.k_batch, o.ktl_batch = _dp(out["k_batch"]), _dp(out["ktl_batch"])
    o.n_source = out["n_source"].ctypes.data_as(C.POINTER(C.c_uint64))
    o.n_sites = out["n_sites"].ctypes.data_as(C.POINTER(C.c_uint64))
    o.mesh_mean, o.mesh_std = _dp(out["mesh_mean"]), _dp(out["mesh_std"])
    o.log_batch = log_batch
    o.log_n = out["log_n"].ctypes.data_as(C.POINTER(C.c_uint32))
    o.log_cell = _ip(out["log_cell"])
    o.log_type = out["log_type"].ctypes.data_as(C.POINTER(C.c_uint8))
    st = L.orc_power_iteration(C.byref(m.s), C.byref(o))
    n = int(o.log_count)
    for key in ("log_n", "log_cell", "log_type"):
        out[key] = out[key][:n]
    out.update(status=st, k_mean=o.k_mean, k_std=o.k_std, scalars_mean=np.array(o.scalars_mean[:]),
               scalars_std=np.array(o.scalars_std[:]), events_by_type=np.array(o.events_by_type[:], np.uint64),
               final_by_type=np.array(o.final_by_type[:], np.uint64))
    return out


# ---- unit-level helpers used by the pin tests ----

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


def uniform(lo, hi):
    return lib().orc_uniform(lo, hi)


def log(x: float) -> float:
    return lib().orc_log(float(x))


def exp_event(seed, tag, hid, n):
    """The exponential variate (ziggurat) of event n of history hid."""
    return lib().orc_exp_event(seed, tag, hid, n)


def zig_table():
    """The ziggurat's per-layer table: widths W, inner widths C, lower
    heights f and height steps df (256 each)."""
    out = (C.c_double * 1024)()
    lib().orc_zig_table(out)
    a = np.array(out[:])
    return a[:256], a[256:512], a[512:768], a[768:]


def iso_dir(seed, tag, hid, n):
    d = (C.c_double * 3)()
    lib().orc_iso_dir(seed, tag, hid, n, d)
    return np.array(d[:])


def elastic(A, E, mu_cm):
    e, mu = C.c_double(), C.c_double()
    lib().orc_elastic(A, E, mu_cm, C.byref(e), C.byref(mu))
    return e.value, mu.value


def azimuth(seed, tag, hid, n):
    """(cos phi, sin phi) of event n of history hid (the CE scatter azimuth)."""
    o = (C.c_double * 2)()
    lib().orc_azimuth(seed, tag, hid, n, o)
    return o[0], o[1]


def elastic_scatter(seed, tag, hid, n, A, E, d):
    """The continuous-energy elastic scatter of event n of history hid off a
    target of mass ratio A: (outgoing direction, outgoing energy)."""
    a = (C.c_double * 3)(*d)
    o = (C.c_double * 3)()
    e = C.c_double()
    lib().orc_elastic_scatter(seed, tag, hid, n, float(A), float(E), a, o, C.byref(e))
    return np.array(o[:]), e.value


def rotate(d, mu, cphi, sphi):
    a = (C.c_double * 3)(*d)
    o = (C.c_double * 3)()
    lib().orc_rotate(a, mu, cphi, sphi, o)
    return np.array(o[:])


def cdf_sample(e, p, xi):
    e = np.ascontiguousarray(e, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    return lib().orc_cdf_sample(_dp(e), _dp(p), len(e), xi)


def nuclide_index(e, E):
    e = np.ascontiguousarray(e, np.float64)
    return lib().orc_nuclide_index(_dp(e), len(e), E)


def mesh_segment(prob, p0, d, length):
    m = _Marshalled(prob)
    out = np.zeros(int(np.prod(prob.mesh_n)))
    a = (C.c_double * 3)(*p0)
    b = (C.c_double * 3)(*d)
    lib().orc_mesh_segment(C.byref(m.s), a, b, float(length), _dp(out))
    return out
