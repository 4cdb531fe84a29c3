"""GPU derivatives (tr_sensitivities / TransportFn.backward) against the
oracle's estimator, the infinite-medium closed form and common-random-number
central finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_tally_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _gpu_sens(spec, n, g_mesh, g_scal, seed=1, scheme=tb.SCHEME_ASYNC):
    import torch
    prob = tb.Problem(spec)
    opts = tb.RunOpts(n_histories=n, seed=seed, scheme=scheme, decomposition=tb.DECOMP_MONO)
    prob.run_fixed_source(opts)
    M, G = spec.n_materials, spec.n_groups
    d_st = torch.empty((M, G), dtype=torch.float64, device="cuda")
    d_ss = torch.empty((M, G, G), dtype=torch.float64, device="cuda")
    d_nf = torch.empty((M, G), dtype=torch.float64, device="cuda")
    gm = torch.tensor(g_mesh, dtype=torch.float64, device="cuda") if g_mesh is not None else None
    gs = torch.tensor(g_scal, dtype=torch.float64, device="cuda") if g_scal is not None else None
    prob.sensitivities(opts, gm.data_ptr() if gm is not None else 0, gs.data_ptr() if gs is not None else 0,
                       d_st.data_ptr(), d_ss.data_ptr(), d_nf.data_ptr())
    out = {"d_sigt": d_st.cpu().numpy(), "d_sigs": d_ss.cpu().numpy(), "d_nusigf": d_nf.cpu().numpy()}
    prob.close()
    return out


def _close(g, o, what):
    # 1e-10 relative per entry, floor 1e-12 of the array's largest entry: every
    # entry is a sum of terms of both signs, and summation order differs
    g, o = np.ravel(g), np.ravel(o)
    tol = 1e-10 * np.abs(o) + 1e-12 * np.abs(o).max()
    bad = np.abs(g - o) > tol
    assert not bad.any(), (what, int(bad.sum()), g[bad][:4], o[bad][:4])


def test_lattice_sensitivities_match_oracle():
    spec = inputs.c5g7_lattice(fission=False)
    n = 20011
    rng = np.random.default_rng(5)
    g_mesh = rng.uniform(-1.0, 1.0, spec.mesh_size)
    g_scal = [0.3, 1.0, 0.7]
    o = oracle.sensitivities(spec, n, g_mesh=g_mesh, g_scal=g_scal, seed=1)
    assert o["status"] == 0
    for scheme in (tb.SCHEME_ASYNC, tb.SCHEME_STACK):
        g = _gpu_sens(spec, n, g_mesh, g_scal, scheme=scheme)
        for key in ("d_sigt", "d_sigs", "d_nusigf"):
            _close(g[key], o[key], key)


def test_autograd_infinite_medium_closed_form():
    import torch
    from paper_2506_00263_gb300.autograd import transport
    spec = inputs.box_mg("inf1", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[1.0], sigma_s=[[0.5]],
                         nu_sigma_f=[0.5], bc=inputs.BC_REFLECT, mesh_n=(2, 2, 2),
                         src_kind=inputs.SRC_POINT, src_point=(5.0, 5.0, 5.0), src_group=0)
    vals = []
    for s in range(6):
        st = torch.tensor([[1.0]], dtype=torch.float64, device="cuda", requires_grad=True)
        ss = torch.tensor([[[0.5]]], dtype=torch.float64, device="cuda", requires_grad=True)
        nf = torch.tensor([[0.5]], dtype=torch.float64, device="cuda", requires_grad=True)
        mesh, scal = transport(st, ss, nf, spec, tb.RunOpts(n_histories=200_000, seed=10 + s,
                                                            scheme=tb.SCHEME_ASYNC))
        (mesh.sum() + scal[2]).backward()      # total flux (mesh covers the box) + production
        vals.append([st.grad.item(), ss.grad.item(), nf.grad.item()])
    v = np.array(vals)
    mean, se = v.mean(0), v.std(0, ddof=1) / math.sqrt(len(v))
    sa, nsf = 0.5, 0.5
    ref = [-1.0 / sa ** 2 - nsf / sa ** 2, 1.0 / sa ** 2 + nsf / sa ** 2, 1.0 / sa]
    assert np.all(np.abs(mean - ref) < 5 * se + 2e-3 * np.abs(ref)), (mean, se, ref)


def test_adjoint_matches_crn_finite_differences():
    """Central differences with common random numbers (h = 1e-4 relative) on
    sigma_t of fuel-1, group 3, for the total absorption rate in the lattice."""
    spec = inputs.c5g7_lattice(fission=False)
    m, g, h = 0, 2, 1e-4
    n, seeds = 100_000, 6
    fd, ad = [], []
    for s in range(seeds):
        vals = []
        for sign in (+1, -1):
            st = spec.sigma_t.copy()
            st[m, g] *= 1.0 + sign * h
            prob = tb.Problem(spec.replace(sigma_t=st))
            prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=100 + s, scheme=tb.SCHEME_ASYNC))
            vals.append(prob.tally(tb.TALLY_SCALARS)[1])
            prob.close()
        fd.append((vals[0] - vals[1]) / (2 * h * spec.sigma_t[m, g]))
        ad.append(_gpu_sens(spec, n, None, [0.0, 1.0, 0.0], seed=100 + s)["d_sigt"][m, g])
    fd, ad = np.array(fd), np.array(ad)
    se = math.sqrt(fd.var(ddof=1) / seeds + ad.var(ddof=1) / seeds)
    assert abs(fd.mean() - ad.mean()) < 5 * se + 1e-4, (fd.mean(), ad.mean(), se)


def test_sensitivities_require_matching_forward_run():
    spec = inputs.cube_one_group()
    prob = tb.Problem(spec)
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(tb.TransportError) as e:
        prob.sensitivities(tb.RunOpts(n_histories=10), 0, 0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
    assert e.value.status == tb.TR_ERR_STATE
    prob.close()


def test_lattice_sensitivities_match_oracle_at_benchmark_size():
    """The benchmark's backward pass (1e6 histories, pre-sampled sources, the
    per-row shared-memory accumulators) against the oracle's estimator over
    the same histories (computed in shards on the host cores)."""
    from tests import _oracle_pool
    spec = inputs.c5g7_lattice(fission=False)
    n = 1_000_000
    rng = np.random.default_rng(6)
    g_mesh = rng.uniform(-1.0, 1.0, spec.mesh_size)
    g_scal = [0.2, 1.0, 0.5]
    o = _oracle_pool.sensitivities(("c5g7_lattice", (("fission", False),)), n, g_mesh=g_mesh, g_scal=g_scal, seed=3)
    assert o["status"] == 0
    g = _gpu_sens(spec, n, g_mesh, g_scal, seed=3)
    for key in ("d_sigt", "d_sigs", "d_nusigf"):
        _close(g[key], o[key], key)


def test_set_xs_equals_a_problem_created_with_those_values():
    """tr_problem_set_xs from device tensors (and from host arrays) gives the
    histories and tallies of a problem created with the new cross sections;
    invalid values are refused and leave the problem as it was."""
    import torch
    a = inputs.c5g7_lattice()
    other = inputs.c5g7_lattice(xs_seed=7)
    # set_xs replaces sigma_t, sigma_s and nu_sigma_f; chi (which samples the
    # source groups) stays a's
    b = a.replace(sigma_t=other.sigma_t, sigma_s=other.sigma_s, nu_sigma_f=other.nu_sigma_f)
    n = 20_011
    opts = tb.RunOpts(n_histories=n, seed=4, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO,
                      remap_every=64, want_event_log=True)
    ref = tb.Problem(b)
    ref.run_fixed_source(opts)
    want = (ref.event_log(n), ref.tally(tb.TALLY_MESH), ref.tally(tb.TALLY_SCALARS))
    ref.close()
    for on_device in (True, False):
        p = tb.Problem(a)
        xs = (b.sigma_t, b.sigma_s, b.nu_sigma_f)
        if on_device:
            xs = tuple(torch.tensor(x, dtype=torch.float64, device="cuda") for x in xs)
        p.set_xs(*xs)
        p.run_fixed_source(opts)
        got = (p.event_log(n), p.tally(tb.TALLY_MESH), p.tally(tb.TALLY_SCALARS))
        for x, y in zip(got[0], want[0]):
            assert np.array_equal(x, y)
        assert np.array_equal(got[1].view(np.uint64), want[1].view(np.uint64))
        assert np.array_equal(got[2].view(np.uint64), want[2].view(np.uint64))
        bad = b.sigma_t.copy()
        bad[0, 0] = -1.0
        with pytest.raises(tb.TransportError) as e:
            p.set_xs(bad, b.sigma_s, b.nu_sigma_f)
        assert e.value.status == tb.TR_ERR_INVALID
        # a refused update changes nothing: the results stay readable, and a
        # new run still uses b's values
        assert np.array_equal(p.tally(tb.TALLY_MESH).view(np.uint64), want[1].view(np.uint64))
        p.run_fixed_source(opts)
        assert np.array_equal(p.tally(tb.TALLY_MESH).view(np.uint64), want[1].view(np.uint64))
        # an accepted update drops the earlier run's results
        p.set_xs(b.sigma_t, b.sigma_s, b.nu_sigma_f)
        with pytest.raises(tb.TransportError):
            p.tally(tb.TALLY_MESH)
        p.close()


def test_autograd_keeps_one_problem_and_matches_direct_derivatives():
    """Fifty forward and backward passes through TransportFn with one problem:
    no problem and no device memory accumulate, and each gradient equals the
    derivative kernel called directly on a problem with those cross
    sections; with a problem description the problem made for the call is
    closed after the backward pass."""
    import torch
    from paper_2506_00263_gb300.autograd import transport
    spec = inputs.c5g7_lattice(fission=False)
    n = 20_011
    opts = tb.RunOpts(n_histories=n, seed=8, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO, remap_every=64)
    g_mesh = np.random.default_rng(2).uniform(-1.0, 1.0, spec.mesh_size)
    gm = torch.tensor(g_mesh, dtype=torch.float64, device="cuda")
    prob = tb.Problem(spec)
    live0 = tb.Problem.live
    base = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in (spec.sigma_t, spec.sigma_s,
                                                                          spec.nu_sigma_f)]
    mem = []
    for it in range(50):
        scale = 1.0 + 0.01 * (it % 5)
        st = (base[0] * scale).requires_grad_(True)
        ss = base[1].clone().requires_grad_(True)
        nf = base[2].clone().requires_grad_(True)
        mesh, scal = transport(st, ss, nf, prob, opts)
        ((mesh * gm).sum() + scal[1]).backward()
        torch.cuda.synchronize()
        mem.append(torch.cuda.memory_allocated())
        if it in (0, 3):
            direct = _gpu_sens(spec.replace(sigma_t=spec.sigma_t * scale), n, g_mesh, [0.0, 1.0, 0.0], seed=8)
            _close(st.grad.cpu().numpy(), direct["d_sigt"], "d_sigt")
            _close(ss.grad.cpu().numpy(), direct["d_sigs"], "d_sigs")
    assert tb.Problem.live == live0
    assert max(mem[5:]) == min(mem[5:]), (min(mem[5:]), max(mem[5:]))
    prob.close()
    # a problem description: one problem per call, closed after backward
    live1 = tb.Problem.live
    st = base[0].clone().requires_grad_(True)
    mesh, scal = transport(st, base[1], base[2], spec, opts)
    assert tb.Problem.live == live1 + 1
    scal[1].backward()
    assert tb.Problem.live == live1
    with torch.no_grad():
        transport(base[0], base[1], base[2], spec, opts)
    assert tb.Problem.live == live1
