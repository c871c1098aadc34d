"""torch.autograd wrapper: (nodal log-viscosity) -> (u, p) through the library's Stokes
solver, with the hand-written adjoint (mfs_adjoint_solve + mfs_grad_log_eta) as backward.

The forward solution, the viscosity it was computed with and a checkpoint of the
viscosity-dependent multigrid state (every level's viscosity, inverse diagonal and Chebyshev
interval, the coarse inverse and the mass-matrix weights: mfs_mg_checkpoint) are saved for the
backward pass; if the problem's viscosity has been changed in between, backward restores the
checkpoint (mfs_mg_restore) before the adjoint solve instead of rebuilding the hierarchy.
"""
from __future__ import annotations

import torch


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_eta, f, g, problem, opts, l_min):
        opts = dict(opts or {})
        problem.set_viscosity(log_eta.detach().contiguous(), is_log=True)
        problem.setup_multigrid(l_min)
        problem._visc_token = object()
        u = torch.zeros_like(f)
        p = torch.zeros_like(g)
        problem.solve(f.detach().contiguous(), g.detach().contiguous(), u, p, **opts)
        ctx.problem, ctx.opts, ctx.l_min, ctx.token = problem, opts, l_min, problem._visc_token
        ctx.state = problem.mg_checkpoint()
        ctx.save_for_backward(log_eta.detach().clone(), u)
        return u, p

    @staticmethod
    def backward(ctx, gu, gp):
        log_eta, u = ctx.saved_tensors
        prob = ctx.problem
        if getattr(prob, "_visc_token", None) is not ctx.token:
            prob.mg_restore(ctx.state)
            prob._visc_token = ctx.token
        gu = torch.zeros_like(u) if gu is None else gu.contiguous()
        gp = torch.zeros(prob.mesh.info(prob.mesh.l_max).n_p1, dtype=torch.float64, device=u.device) \
            if gp is None else gp.contiguous()
        lam_u = torch.zeros_like(u)
        lam_p = torch.zeros_like(gp)
        opts = dict(ctx.opts)
        prob.adjoint_solve(gu, gp, lam_u, lam_p, **opts)
        grad = torch.empty_like(log_eta)
        prob.grad_log_eta(u, lam_u, grad)
        ctx.state = None
        # K x = b: dJ/db = lam (projected), returned for f and g
        return grad, lam_u, lam_p, None, None, None


def stokes_solve(log_eta, f, g, problem, opts=None, l_min=1):
    """(u, p) = solve of the Stokes system with viscosity exp(log_eta); differentiable in
    log_eta (and in f, g)."""
    return StokesSolve.apply(log_eta, f, g, problem, opts, l_min)
