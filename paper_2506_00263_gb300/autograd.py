"""Differentiable fixed-source transport: ``torch.autograd.Function`` over the C ABI.

``transport(sigma_t, sigma_s, nu_sigma_f, problem, opts)`` runs a multigroup
fixed-source problem with the given cross sections and returns the mesh flux
tally and the scalar tallies (flux, absorption rate, production rate) per
source particle.  ``problem`` is a ``binding.Problem`` kept by the caller
(the cross sections are written into it on the device with
``tr_problem_set_xs``: no host copy, no new problem per step), or a problem
description, for which a problem is made for this call and closed once the
backward pass has run (or at once when no gradient is wanted).  The backward
pass calls ``tr_sensitivities``: the score-function + pathwise estimator over
the same histories, recomputed on the GPU from their random-number keys.
Gradients flow to sigma_t [m][g], sigma_s [m][g][g'] and nu_sigma_f [m][g].
"""
from __future__ import annotations

import torch

from . import binding as tb


def _xs(t):
    return t.detach().to(torch.float64).contiguous()


class TransportFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, nu_sigma_f, problem, opts):
        dev = sigma_t.device
        owned = not isinstance(problem, tb.Problem)
        if owned:
            problem = tb.Problem(problem, device=dev.index if dev.type == "cuda" else None)
        st, ss, nf = _xs(sigma_t), _xs(sigma_s), _xs(nu_sigma_f)
        if st.is_cuda:
            problem.set_xs(st, ss, nf)
        else:
            problem.set_xs(st.numpy(), ss.numpy(), nf.numpy())
        problem.run_fixed_source(opts)
        n_mesh = problem.tally_size(tb.TALLY_MESH)
        out_dev = dev if dev.type == "cuda" else torch.device("cuda", torch.cuda.current_device())
        mesh = torch.empty(n_mesh, dtype=torch.float64, device=out_dev)
        scal = torch.empty(3, dtype=torch.float64, device=out_dev)
        if n_mesh:
            problem.tally_to_device(tb.TALLY_MESH, mesh.data_ptr(), n_mesh)
        problem.tally_to_device(tb.TALLY_SCALARS, scal.data_ptr(), 3)
        if any(ctx.needs_input_grad[:3]):
            ctx.save_for_backward(st, ss, nf)
            ctx.problem, ctx.owned, ctx.opts, ctx.gen = problem, owned, opts, problem.xs_generation
        elif owned:
            problem.close()
        return mesh.to(dev), scal.to(dev)

    @staticmethod
    def backward(ctx, g_mesh, g_scal):
        prob, opts = ctx.problem, ctx.opts
        st, ss, nf = ctx.saved_tensors
        if prob.xs_generation != ctx.gen:
            # another forward pass rewrote this problem since: restore this
            # pass's cross sections and histories before differentiating
            prob.set_xs(st, ss, nf) if st.is_cuda else prob.set_xs(st.numpy(), ss.numpy(), nf.numpy())
            prob.run_fixed_source(opts)
            ctx.gen = prob.xs_generation
        dev = torch.device("cuda", torch.cuda.current_device()) if not st.is_cuda else st.device
        d_st = torch.empty(st.shape, dtype=torch.float64, device=dev)
        d_ss = torch.empty(ss.shape, dtype=torch.float64, device=dev)
        d_nf = torch.empty(nf.shape, dtype=torch.float64, device=dev)
        gm = g_mesh.to(dev, torch.float64).contiguous() if (g_mesh is not None and g_mesh.numel()) else None
        gs = g_scal.to(dev, torch.float64).contiguous() if g_scal is not None else None
        prob.sensitivities(opts, gm.data_ptr() if gm is not None else 0, gs.data_ptr() if gs is not None else 0,
                           d_st.data_ptr(), d_ss.data_ptr(), d_nf.data_ptr())
        if ctx.owned:
            prob.close()
            ctx.problem = None
        to = st.device
        return d_st.to(to), d_ss.to(to), d_nf.to(to), None, None


def transport(sigma_t, sigma_s, nu_sigma_f, problem, opts: tb.RunOpts):
    """(mesh flux, scalar tallies) of a fixed-source run, differentiable in
    the cross sections; problem: a binding.Problem or a problem description."""
    return TransportFn.apply(sigma_t, sigma_s, nu_sigma_f, problem, opts)
