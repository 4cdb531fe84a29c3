"""Thin Python binding of the C ABI in ``include/tr.h`` (argument marshalling only).

Every step of the transport path runs in the CUDA library ``libtr.so``; this
module converts a :class:`paper_2506_00263_gb300.inputs.Problem` into the C
descriptions, wires device allocation to PyTorch's caching allocator and the
work to PyTorch's current CUDA stream, and returns numpy arrays.  It raises if
the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import inputs as _inp

_HERE = os.path.dirname(os.path.abspath(__file__))
# TR_LIBRARY selects another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("TR_LIBRARY") or os.path.join(_HERE, "libtr.so")

TR_OK, TR_ERR_INVALID, TR_ERR_NOMEM, TR_ERR_CAPACITY, TR_ERR_TIMEOUT, TR_ERR_CUDA, TR_ERR_STATE = range(7)
STATUS_NAMES = {0: "TR_OK", 1: "TR_ERR_INVALID", 2: "TR_ERR_NOMEM", 3: "TR_ERR_CAPACITY", 4: "TR_ERR_TIMEOUT",
                5: "TR_ERR_CUDA", 6: "TR_ERR_STATE"}
EV_SOURCE, EV_SCATTER, EV_ABSORB, EV_SURF_INTERNAL, EV_SURF_REFLECT, EV_LEAK, EV_CUTOFF, EV_MAXEV = range(8)
SCHEME_STACK, SCHEME_ASYNC = 0, 1
DECOMP_MONO, DECOMP_SPLIT, DECOMP_SPLIT_LOOKUP, DECOMP_STREAM = 0, 1, 2, 3
TALLY_MESH, TALLY_ENERGY, TALLY_SCALARS, TALLY_TIME = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class GeometryDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x_planes", _dp), ("y_planes", _dp), ("z_planes", _dp),
                ("bc", C.c_int32 * 6), ("cell_material", _ip), ("pin_material", _ip), ("pin_radius", C.c_double)]


class XsDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_materials", C.c_int32), ("n_groups", C.c_int32),
                ("sigma_t", _dp), ("sigma_s", _dp), ("nu_sigma_f", _dp), ("chi", _dp),
                ("n_nuclides", C.c_int32), ("nuc_offset", C.POINTER(C.c_int64)), ("nuc_energy", _dp),
                ("nuc_sigma", _dp), ("nuc_awr", _dp), ("density", _dp), ("energy_cutoff", C.c_double),
                ("inv_velocity", _dp)]


class SourceDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("isotropic", C.c_int32), ("group", C.c_int32), ("n_cdf", C.c_int32),
                ("point", C.c_double * 3), ("direction", C.c_double * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("energy", C.c_double), ("source_material", C.POINTER(C.c_uint8)),
                ("cdf_energy", _dp), ("cdf_prob", _dp)]


class TallyDesc(C.Structure):
    _fields_ = [("has_mesh", C.c_int32), ("mesh_n", C.c_int32 * 3), ("by_group", C.c_int32),
                ("n_energy_bins", C.c_int32), ("mesh_lo", C.c_double * 3), ("mesh_hi", C.c_double * 3),
                ("energy_edges", _dp), ("n_time_bins", C.c_int32), ("t_census", C.c_double),
                ("ww_lower", _dp), ("ww_upper", C.c_double), ("ww_survival", C.c_double),
                ("ww_max_split", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class DeviceCtx(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("user", C.c_void_p)]


class RunOptsC(C.Structure):
    _fields_ = [("n_histories", C.c_uint64), ("seed", C.c_uint64), ("scheme", C.c_int32),
                ("decomposition", C.c_int32), ("queue_capacity", C.c_uint64), ("blocks_per_sm", C.c_int32),
                ("remap_every", C.c_int32), ("stash_slots", C.c_int32), ("max_spin", C.c_int64),
                ("max_events", C.c_uint32), ("want_event_log", C.c_int32), ("spill_threshold", C.c_int32),
                ("problem_tag", C.c_uint32), ("first_history", C.c_uint64), ("max_wait_ms", C.c_uint32),
                ("reserved", C.c_uint32)]


class RunStats(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("events", C.c_uint64), ("events_by_type", C.c_uint64 * 8),
                ("final_by_type", C.c_uint64 * 8), ("launches", C.c_uint64), ("spills", C.c_uint64),
                ("refills", C.c_uint64), ("seconds", C.c_double), ("transport_seconds", C.c_double),
                ("used_blocks_per_sm", C.c_int32), ("used_stash_slots", C.c_int32),
                ("used_remap_every", C.c_int32), ("reserved", C.c_int32)]


class EigOptsC(C.Structure):
    _fields_ = [("n_per_batch", C.c_uint64), ("n_inactive", C.c_uint32), ("n_active", C.c_uint32),
                ("k0", C.c_double), ("bank_capacity_factor", C.c_double), ("run", RunOptsC),
                ("stop_after", C.c_uint32), ("resume_from", C.c_void_p), ("resume_bytes", C.c_size_t)]


class EigResultC(C.Structure):
    _fields_ = [("k_mean", C.c_double), ("k_std", C.c_double), ("k_batch", _dp), ("ktl_batch", _dp),
                ("n_source", C.POINTER(C.c_uint64)), ("histories", C.c_uint64), ("events", C.c_uint64),
                ("final_by_type", C.c_uint64 * 8), ("seconds", C.c_double), ("transport_seconds", C.c_double),
                ("transport_launches", C.c_uint64), ("batches_done", C.c_uint32)]


_lib = None


def lib():
    """Load libtr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2506_00263_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    L.tr_problem_create.argtypes = [C.POINTER(GeometryDesc), C.POINTER(XsDesc), C.POINTER(SourceDesc),
                                    C.POINTER(TallyDesc), C.c_int32, C.POINTER(DeviceCtx), C.POINTER(C.c_void_p)]
    L.tr_problem_create.restype = C.c_int
    L.tr_problem_destroy.argtypes = [C.c_void_p]
    L.tr_problem_destroy.restype = None
    L.tr_run_fixed_source.argtypes = [C.c_void_p, C.POINTER(RunOptsC), C.POINTER(RunStats)]
    L.tr_run_fixed_source.restype = C.c_int
    L.tr_run_power_iteration.argtypes = [C.c_void_p, C.POINTER(EigOptsC), C.POINTER(EigResultC)]
    L.tr_run_power_iteration.restype = C.c_int
    for fn in ("tr_tallies", "tr_tally_stddev"):
        getattr(L, fn).argtypes = [C.c_void_p, C.c_int32, _dp, C.c_size_t, C.c_int32]
        getattr(L, fn).restype = C.c_int
    L.tr_tally_size.argtypes = [C.c_void_p, C.c_int32]
    L.tr_tally_size.restype = C.c_size_t
    L.tr_event_log.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), _ip, C.POINTER(C.c_uint8), C.c_size_t]
    L.tr_event_log.restype = C.c_int
    L.tr_last_error.restype = C.c_char_p
    L.tr_kernel_launch_count.restype = C.c_uint64
    L.tr_sensitivities.argtypes = [C.c_void_p, C.POINTER(RunOptsC), _dp, _dp, _dp, _dp, _dp]
    L.tr_sensitivities.restype = C.c_int
    L.tr_run_fixed_source_noalloc.argtypes = [C.c_void_p, C.POINTER(RunOptsC), _dp, _dp, _dp, C.POINTER(RunStats)]
    L.tr_run_fixed_source_noalloc.restype = C.c_int
    L.tr_run_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_uint64), C.POINTER(RunOptsC),
                                 C.POINTER(RunStats)]
    L.tr_run_batched.restype = C.c_int
    L.tr_eig_checkpoint.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    L.tr_eig_checkpoint.restype = C.c_int
    L.tr_problem_set_xs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.tr_problem_set_xs.restype = C.c_int
    L.tr_version.restype = C.c_char_p
    L.tr_selftest_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_size_t,
                                     C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.tr_selftest_philox.restype = C.c_int
    L.tr_selftest_log.argtypes = [C.c_void_p, _dp, C.c_size_t, _dp]
    L.tr_selftest_log.restype = C.c_int
    L.tr_selftest_zig_table.argtypes = [C.c_void_p, _dp]
    L.tr_selftest_zig_table.restype = C.c_int
    L.tr_selftest_issue_rate.argtypes = [C.c_int32, C.c_int32, _dp]
    L.tr_selftest_issue_rate.restype = C.c_int
    L.tr_selftest_softfp.argtypes = [C.c_int32, _dp, C.c_size_t, _dp]
    L.tr_selftest_softfp.restype = C.c_int
    _lib = L
    return L


def softfp(op: int, x) -> np.ndarray:
    """tr_selftest_softfp: 0 sf_rcp, 1 1/x, 2 sf_sqrt, 3 sqrt, elementwise on
    the device; 4 sf_div, 5 division, of the pairs (x[2i], x[2i+1])."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(x.size // 2 if op >= 4 else x.size)
    _check(lib().tr_selftest_softfp(op, x.ctypes.data_as(_dp), x.size, out.ctypes.data_as(_dp)))
    return out


def issue_rate(op: int, lanes: int = 32) -> float:
    """tr_selftest_issue_rate: operations (op 7: FP64 warp instructions) per second."""
    v = C.c_double()
    _check(lib().tr_selftest_issue_rate(op, lanes, C.byref(v)))
    return v.value


def selftest_philox(ctr, key):
    """tr_selftest_philox: (library Philox, curand Philox) on n counters (n x 4
    uint32) and keys (n x 2 uint32), each n x 4 uint32."""
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    n = ctr.shape[0]
    ours = np.zeros((n, 4), np.uint32)
    lib_out = np.zeros((n, 4), np.uint32)
    u32 = C.POINTER(C.c_uint32)
    _check(lib().tr_selftest_philox(ctr.ctypes.data_as(u32), key.ctypes.data_as(u32), n,
                                    ours.ctypes.data_as(u32), lib_out.ctypes.data_as(u32)))
    return ours, lib_out


class TransportError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st):
    if st != TR_OK:
        raise TransportError(st, lib().tr_last_error().decode())


@dataclass
class RunOpts:
    n_histories: int = 0
    seed: int = 1
    scheme: int = SCHEME_STACK
    decomposition: int = DECOMP_MONO
    queue_capacity: int = 0
    blocks_per_sm: int = 0
    remap_every: int = 1
    stash_slots: int = 0
    max_spin: int = 0
    max_events: int = 0
    want_event_log: bool = False
    spill_threshold: int = 0
    problem_tag: int = 0
    first_history: int = 0
    max_wait_ms: int = 0
    reserved: int = 0

    def to_c(self) -> RunOptsC:
        c = RunOptsC()
        for f in RunOptsC._fields_:
            setattr(c, f[0], int(getattr(self, f[0])))
        return c


def _torch_ctx(device=None):
    """Device context wired to PyTorch's caching allocator and current stream."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    stream = torch.cuda.current_stream(dev)
    live = {}

    def _alloc(size, _stream, _user):
        try:
            p = torch.cuda.caching_allocator_alloc(int(size), dev, stream)
        except Exception:  # allocation failure is reported as NULL
            return None
        live[p] = True
        return p

    def _free(ptr, _stream, _user):
        if ptr and ptr in live:
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    ctx = DeviceCtx()
    ctx.device = dev
    ctx.stream = stream.cuda_stream
    ctx.alloc = ALLOC_FN(_alloc)
    ctx.free = FREE_FN(_free)
    ctx.user = None
    return ctx, (_alloc, _free, live, stream)


class Problem:
    """A problem resident on the GPU (``tr_problem``)."""

    def __init__(self, prob: "_inp.Problem", device=None, use_torch_allocator: bool = True):
        L = lib()
        self.spec = prob
        self.xs_generation = 0            # tr_problem_set_xs calls so far
        keep = []

        def f64(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            keep.append(a)
            return a.ctypes.data_as(_dp)

        def i32(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
            keep.append(a)
            return a.ctypes.data_as(_ip)

        g = GeometryDesc()
        g.nz, g.ny, g.nx = prob.shape
        g.x_planes, g.y_planes, g.z_planes = f64(prob.x_planes), f64(prob.y_planes), f64(prob.z_planes)
        for i in range(6):
            g.bc[i] = int(prob.bc[i])
        g.cell_material = i32(prob.cell_material)
        g.pin_material = i32(prob.pin_material)
        g.pin_radius = float(prob.pin_radius)

        x = XsDesc()
        x.kind, x.n_materials = int(prob.xs_kind), int(prob.n_materials)
        if prob.xs_kind == _inp.XS_MG:
            x.n_groups = int(prob.n_groups)
            x.sigma_t, x.sigma_s = f64(prob.sigma_t), f64(prob.sigma_s)
            x.nu_sigma_f, x.chi = f64(prob.nu_sigma_f), f64(prob.chi)
            if getattr(prob, "inv_velocity", None) is not None:
                x.inv_velocity = f64(prob.inv_velocity)
        else:
            x.n_groups = 1
            x.n_nuclides = len(prob.nuc_energy)
            off = np.zeros(x.n_nuclides + 1, np.int64)
            off[1:] = np.cumsum([len(e) for e in prob.nuc_energy])
            keep.append(off)
            x.nuc_offset = off.ctypes.data_as(C.POINTER(C.c_int64))
            x.nuc_energy = f64(np.concatenate(prob.nuc_energy))
            x.nuc_sigma = f64(np.concatenate(prob.nuc_sigma, axis=0))
            x.nuc_awr, x.density = f64(prob.nuc_awr), f64(prob.mat_density)
            x.energy_cutoff = float(prob.energy_cutoff)

        s = SourceDesc()
        s.kind = int(prob.src_kind)
        s.isotropic = 1 if prob.src_direction is None else 0
        s.group = int(prob.src_group)
        for i in range(3):
            s.point[i] = prob.src_point[i]
            s.lo[i], s.hi[i] = prob.src_lo[i], prob.src_hi[i]
            s.direction[i] = 0.0 if prob.src_direction is None else prob.src_direction[i]
        s.energy = float(prob.src_energy)
        sm = np.ascontiguousarray(np.asarray(prob.src_materials if prob.src_materials is not None
                                             else np.ones(prob.n_materials), dtype=np.uint8))
        keep.append(sm)
        s.source_material = sm.ctypes.data_as(C.POINTER(C.c_uint8))
        if prob.src_cdf_energy is not None:
            s.n_cdf = len(prob.src_cdf_energy)
            s.cdf_energy, s.cdf_prob = f64(prob.src_cdf_energy), f64(prob.src_cdf_prob)

        t = TallyDesc()
        n_t = 0
        if prob.mesh_n is not None:
            n_t = 1
            t.has_mesh = 1
            for i in range(3):
                t.mesh_n[i] = int(prob.mesh_n[i])
                t.mesh_lo[i], t.mesh_hi[i] = prob.mesh_lo[i], prob.mesh_hi[i]
            t.by_group = 1 if prob.mesh_by_group else 0
        if prob.energy_edges is not None:
            n_t = 1
            t.n_energy_bins = len(prob.energy_edges) - 1
            t.energy_edges = f64(prob.energy_edges)
        if getattr(prob, "t_census", 0.0):
            n_t = 1
            t.t_census = float(prob.t_census)
            t.n_time_bins = int(prob.n_time_bins)
        if getattr(prob, "ww_lower", None) is not None:
            n_t = 1
            t.ww_lower = f64(prob.ww_lower)
            t.ww_upper, t.ww_survival = float(prob.ww_upper), float(prob.ww_survival)
            t.ww_max_split = int(prob.ww_max_split)

        if use_torch_allocator:
            self._ctx, self._keep_ctx = _torch_ctx(device)
        else:
            import torch
            self._ctx = DeviceCtx()
            self._ctx.device = torch.cuda.current_device() if device is None else int(device)
            self._ctx.stream = torch.cuda.current_stream(self._ctx.device).cuda_stream
            self._keep_ctx = None
        h = C.c_void_p()
        _check(L.tr_problem_create(C.byref(g), C.byref(x), C.byref(s), C.byref(t), n_t, C.byref(self._ctx),
                                   C.byref(h)))
        self._h = h
        self.last_stats = None
        Problem.live += 1

    # problems created and not yet closed in this process
    live = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().tr_problem_destroy(self._h)
            self._h = None
            Problem.live -= 1

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def run_fixed_source(self, opts: RunOpts) -> dict:
        st = RunStats()
        c = opts.to_c()
        _check(lib().tr_run_fixed_source(self._h, C.byref(c), C.byref(st)))
        self.last_stats = stats_dict(st)
        return self.last_stats

    def run_fixed_source_noalloc(self, opts: RunOpts, mesh_ptr: int, energy_ptr: int, scalars_ptr: int) -> dict:
        """tr_run_fixed_source_noalloc: the asynchronous fixed-source run with
        its scratch in the library's static device array; the tallies go to the
        given device pointers (0 for an absent tally).  Allocates nothing."""
        st = RunStats()
        c = opts.to_c()

        def ptr(v):
            return C.cast(C.c_void_p(int(v)), _dp) if v else None

        _check(lib().tr_run_fixed_source_noalloc(self._h, C.byref(c), ptr(mesh_ptr), ptr(energy_ptr),
                                                 ptr(scalars_ptr), C.byref(st)))
        return stats_dict(st)

    def sensitivities(self, opts: RunOpts, g_mesh_ptr: int, g_scal_ptr: int, d_sigt_ptr: int, d_sigs_ptr: int,
                      d_nusigf_ptr: int) -> None:
        """tr_sensitivities with device pointers (0 for an absent upstream gradient)."""
        def ptr(v):
            return C.cast(C.c_void_p(int(v)), _dp) if v else None

        c = opts.to_c()
        _check(lib().tr_sensitivities(self._h, C.byref(c), ptr(g_mesh_ptr), ptr(g_scal_ptr), ptr(d_sigt_ptr),
                                      ptr(d_sigs_ptr), ptr(d_nusigf_ptr)))

    def power_iteration(self, n_per_batch, n_inactive, n_active, opts: RunOpts, k0=1.0,
                        bank_capacity_factor=0.0, stop_after: int = 0, resume: bytes = None) -> dict:
        """tr_run_power_iteration; stop_after > 0 ends early keeping the state
        (read it with eig_checkpoint), resume continues from such a state."""
        eo = EigOptsC()
        eo.n_per_batch, eo.n_inactive, eo.n_active = n_per_batch, n_inactive, n_active
        eo.k0, eo.bank_capacity_factor = k0, bank_capacity_factor
        eo.run = opts.to_c()
        eo.stop_after = stop_after
        if resume is not None:
            rbuf = C.create_string_buffer(bytes(resume), len(resume))
            eo.resume_from = C.cast(rbuf, C.c_void_p)
            eo.resume_bytes = len(resume)
        nb = n_inactive + n_active
        kb, ktl, ns = np.zeros(nb), np.zeros(nb), np.zeros(nb, np.uint64)
        r = EigResultC()
        r.k_batch, r.ktl_batch = kb.ctypes.data_as(_dp), ktl.ctypes.data_as(_dp)
        r.n_source = ns.ctypes.data_as(C.POINTER(C.c_uint64))
        _check(lib().tr_run_power_iteration(self._h, C.byref(eo), C.byref(r)))
        return {"k_mean": r.k_mean, "k_std": r.k_std, "k_batch": kb, "ktl_batch": ktl, "n_source": ns,
                "histories": r.histories, "events": r.events,
                "final_by_type": np.array(r.final_by_type[:], np.uint64), "seconds": r.seconds,
                "transport_seconds": r.transport_seconds, "transport_launches": r.transport_launches,
                "batches_done": r.batches_done}

    def eig_checkpoint(self) -> bytes:
        """tr_eig_checkpoint: the state of the last power iteration stopped early."""
        n = C.c_size_t(0)
        _check(lib().tr_eig_checkpoint(self._h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().tr_eig_checkpoint(self._h, buf, n.value, C.byref(n)))
        return buf.raw[:n.value]

    def selftest_log(self, x) -> np.ndarray:
        """tr_selftest_log: the device logarithm of the transport kernels."""
        x = np.ascontiguousarray(x, np.float64)
        out = np.empty_like(x)
        _check(lib().tr_selftest_log(self._h, x.ctypes.data_as(_dp), x.size, out.ctypes.data_as(_dp)))
        return out

    def zig_table(self) -> np.ndarray:
        """tr_selftest_zig_table: the ziggurat table the transport kernels read."""
        out = np.empty(1024, np.float64)
        _check(lib().tr_selftest_zig_table(self._h, out.ctypes.data_as(_dp)))
        return out

    def set_xs(self, sigma_t, sigma_s, nu_sigma_f):
        """tr_problem_set_xs: new multigroup cross sections, either numpy
        arrays (host) or contiguous float64 CUDA tensors on the problem's
        device (passed by pointer, no host copy).  Shapes as at creation."""
        arrs = (sigma_t, sigma_s, nu_sigma_f)
        on_dev = all(hasattr(a, "data_ptr") and getattr(a, "is_cuda", False) for a in arrs)
        if on_dev:
            for a in arrs:
                if str(a.dtype) != "torch.float64" or not a.is_contiguous():
                    raise ValueError("device cross sections must be contiguous float64 tensors")
            ptrs = [a.data_ptr() for a in arrs]
            keep = arrs
        else:
            keep = [np.ascontiguousarray(a, np.float64) for a in arrs]
            ptrs = [k.ctypes.data for k in keep]
        _check(lib().tr_problem_set_xs(self._h, ptrs[0], ptrs[1], ptrs[2], 1 if on_dev else 0))
        del keep
        self.xs_generation += 1

    def tally_size(self, tally_id: int) -> int:
        """tr_tally_size: bins of one tally (0 if absent)."""
        return int(lib().tr_tally_size(self._h, tally_id))

    def tally(self, tally_id: int, stddev: bool = False) -> np.ndarray:
        n = lib().tr_tally_size(self._h, tally_id)
        out = np.zeros(n)
        fn = lib().tr_tally_stddev if stddev else lib().tr_tallies
        _check(fn(self._h, tally_id, out.ctypes.data_as(_dp), n, 0))
        return out

    def tally_to_device(self, tally_id: int, out_ptr: int, n: int):
        _check(lib().tr_tallies(self._h, tally_id, C.cast(C.c_void_p(out_ptr), _dp), n, 1))

    def event_log(self, n: int):
        a = np.zeros(n, np.uint32)
        b = np.zeros(n, np.int32)
        c = np.zeros(n, np.uint8)
        _check(lib().tr_event_log(self._h, a.ctypes.data_as(C.POINTER(C.c_uint32)), b.ctypes.data_as(_ip),
                                  c.ctypes.data_as(C.POINTER(C.c_uint8)), n))
        return a, b, c


def stats_dict(st: RunStats) -> dict:
    return {"histories": st.histories, "events": st.events,
            "events_by_type": np.array(st.events_by_type[:], np.uint64),
            "final_by_type": np.array(st.final_by_type[:], np.uint64), "launches": st.launches,
            "spills": st.spills, "refills": st.refills, "seconds": st.seconds,
            "transport_seconds": st.transport_seconds,
            "used": (st.used_blocks_per_sm, st.used_stash_slots, st.used_remap_every)}


def run_batched(problems, n_histories, opts: RunOpts) -> list:
    """tr_run_batched: transport several problems in one persistent launch;
    problem i uses the random-stream tag opts.problem_tag ^ i.  Returns the
    per-problem statistics; each problem's tallies are read as after a single
    run."""
    n = len(problems)
    if n != len(n_histories):
        raise ValueError("one history count per problem")
    hs = (C.c_void_p * n)(*[p._h for p in problems])
    nh = (C.c_uint64 * n)(*[int(v) for v in n_histories])
    st = (RunStats * n)()
    c = opts.to_c()
    _check(lib().tr_run_batched(hs, n, nh, C.byref(c), st))
    return [stats_dict(st[i]) for i in range(n)]


def kernel_launch_count() -> int:
    return int(lib().tr_kernel_launch_count())


def version() -> str:
    return lib().tr_version().decode()
