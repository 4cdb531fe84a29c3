"""Pins for the oracle's derivative estimator (score function in causal form
plus pathwise reaction-rate terms) against closed-form derivatives of
infinite-medium solutions."""
import math

import numpy as np

import oracle
from paper_2506_00263_gb300 import inputs


def _runs(p, n, k, **kw):
    return [oracle.sensitivities(p, n, seed=1000 + s, **kw) for s in range(k)]


def _stat(runs, key):
    a = np.array([r[key] for r in runs])
    return a.mean(0), a.std(0, ddof=1) / math.sqrt(len(runs))


def test_one_group_infinite_medium_derivatives():
    st, ss, nsf = 1.0, 0.5, 0.5
    p = inputs.box_mg("inf1", (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), sigma_t=[st], sigma_s=[[ss]],
                      nu_sigma_f=[nsf], bc=inputs.BC_REFLECT, mesh_n=(1, 1, 1),
                      src_kind=inputs.SRC_POINT, src_point=(5.0, 5.0, 5.0), src_group=0)
    sa = st - ss
    # L = total flux = 1/Sa
    runs = _runs(p, 20000, 8, g_scal=[1.0, 0.0, 0.0])
    for r in runs:
        assert r["status"] == 0
    m, e = _stat(runs, "d_sigt")
    assert abs(m[0, 0] - (-1.0 / sa ** 2)) < 5 * e[0, 0] + 1e-3
    m, e = _stat(runs, "d_sigs")
    assert abs(m[0, 0, 0] - (1.0 / sa ** 2)) < 5 * e[0, 0, 0] + 1e-3
    assert np.all(np.array([r["d_nusigf"] for r in runs]) == 0.0)
    # L = absorption rate = 1 exactly: every derivative is zero in expectation
    runs = _runs(p, 20000, 8, g_scal=[0.0, 1.0, 0.0])
    for key in ("d_sigt", "d_sigs"):
        m, e = _stat(runs, key)
        assert np.all(np.abs(m) < 5 * e + 1e-3), (key, m, e)
    v = np.array([r["value"] for r in runs])       # track-length estimate of the absorption rate
    assert abs(v.mean() - 1.0) < 5 * v.std(ddof=1) / math.sqrt(len(v)) + 1e-3
    # L = production = nuSf/Sa: d/dnuSf = 1/Sa (pathwise only), d/dSt = -nuSf/Sa^2
    runs = _runs(p, 20000, 8, g_scal=[0.0, 0.0, 1.0])
    m, e = _stat(runs, "d_nusigf")
    assert abs(m[0, 0] - 1.0 / sa) < 5 * e[0, 0] + 1e-3
    m, e = _stat(runs, "d_sigt")
    assert abs(m[0, 0] - (-nsf / sa ** 2)) < 5 * e[0, 0] + 1e-3


def test_multigroup_infinite_medium_adjoint_closed_form():
    st, ss, nsf, chi = inputs.c5g7_xs(2025)
    st, ss = st[0], ss[0]
    G = len(st)
    p = inputs.box_mg("mg_inf", (0.0, 0.0, 0.0), (20.0, 20.0, 20.0), sigma_t=st, sigma_s=ss,
                      bc=inputs.BC_REFLECT, mesh_n=(1, 1, 1), src_kind=inputs.SRC_POINT,
                      src_point=(10.0, 10.0, 10.0), src_group=0)
    A = np.diag(st) - ss.T
    phi = np.linalg.solve(A, np.eye(G)[0])        # forward flux
    psi = np.linalg.solve(A.T, np.ones(G))        # adjoint of total flux
    d_st = -psi * phi                              # dL/dSt[g]
    d_ss = np.outer(phi, psi)                      # dL/dSs[g->h] = phi_g psi_h
    runs = _runs(p, 8000, 10, g_scal=[1.0, 0.0, 0.0])
    m, e = _stat(runs, "d_sigt")
    assert np.all(np.abs(m[0] - d_st) < 5 * e[0] + 2e-3 * np.abs(d_st).max()), (m[0], d_st)
    m, e = _stat(runs, "d_sigs")
    mask = ss > 0
    assert np.all(np.abs(m[0][mask] - d_ss[mask]) < 5 * e[0][mask] + 2e-3 * np.abs(d_ss).max())
    # a transposed transfer index would disagree clearly
    assert np.abs(d_ss.T[mask] - d_ss[mask]).max() > 10 * e[0][mask].max()


def test_mesh_weights_match_scalar_flux_weights():
    p = inputs.cube_one_group(n_mesh=1)
    a = oracle.sensitivities(p, 3000, g_mesh=np.ones(1), seed=4)
    b = oracle.sensitivities(p, 3000, g_scal=[1.0, 0.0, 0.0], seed=4)
    for key in ("d_sigt", "d_sigs"):
        assert np.allclose(a[key], b[key], rtol=1e-11, atol=0)
    assert abs(a["value"] - b["value"]) < 1e-12 * b["value"]
