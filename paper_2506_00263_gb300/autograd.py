"""Differentiable fixed-source transport: ``torch.autograd.Function`` over the C ABI.

``transport(sigma_t, sigma_s, nu_sigma_f, spec, opts)`` runs the fixed-source
problem ``spec`` (multigroup) with the given cross sections and returns the
mesh flux tally and the scalar tallies (flux, absorption rate, production
rate) per source particle.  Its backward pass calls ``tr_sensitivities``: the
score-function + pathwise estimator over the same histories, recomputed on
the GPU from their random-number keys.  Gradients flow to sigma_t [m][g],
sigma_s [m][g][g'] and nu_sigma_f [m][g].
"""
from __future__ import annotations

import dataclasses

import torch

from . import binding as tb


class TransportFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, nu_sigma_f, spec, opts):
        dev = sigma_t.device
        data = {k: v.detach().to("cpu", torch.float64).contiguous().numpy()
                for k, v in (("sigma_t", sigma_t), ("sigma_s", sigma_s), ("nu_sigma_f", nu_sigma_f))}
        prob = tb.Problem(dataclasses.replace(spec, **data), device=dev.index if dev.type == "cuda" else None)
        prob.run_fixed_source(opts)
        n_mesh = prob.spec.mesh_size
        mesh = torch.empty(n_mesh, dtype=torch.float64, device=dev)
        scal = torch.empty(3, dtype=torch.float64, device=dev)
        if n_mesh:
            prob.tally_to_device(tb.TALLY_MESH, mesh.data_ptr(), n_mesh)
        prob.tally_to_device(tb.TALLY_SCALARS, scal.data_ptr(), 3)
        ctx.prob, ctx.opts = prob, opts
        ctx.shapes = (sigma_t.shape, sigma_s.shape, nu_sigma_f.shape)
        return mesh, scal

    @staticmethod
    def backward(ctx, g_mesh, g_scal):
        prob, opts = ctx.prob, ctx.opts
        dev = g_scal.device if g_scal is not None else g_mesh.device
        st_shape, ss_shape, nf_shape = ctx.shapes
        d_st = torch.empty(st_shape, dtype=torch.float64, device=dev)
        d_ss = torch.empty(ss_shape, dtype=torch.float64, device=dev)
        d_nf = torch.empty(nf_shape, dtype=torch.float64, device=dev)
        gm = g_mesh.contiguous().to(torch.float64) if (g_mesh is not None and g_mesh.numel()) else None
        gs = g_scal.contiguous().to(torch.float64) if g_scal is not None else None
        prob.sensitivities(opts, gm.data_ptr() if gm is not None else 0, gs.data_ptr() if gs is not None else 0,
                           d_st.data_ptr(), d_ss.data_ptr(), d_nf.data_ptr())
        return d_st, d_ss, d_nf, None, None


def transport(sigma_t, sigma_s, nu_sigma_f, spec, opts: tb.RunOpts):
    """(mesh flux, scalar tallies) of a fixed-source run, differentiable in the cross sections."""
    return TransportFn.apply(sigma_t, sigma_s, nu_sigma_f, spec, opts)
