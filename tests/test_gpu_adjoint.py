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
