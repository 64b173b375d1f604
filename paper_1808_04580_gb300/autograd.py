"""Differentiable solve of (beta L_s + diag(s)) u = f (Sec. 6.2.2) for torch autograd.

Forward: nfl_cg_solve.  Backward: nfl_cg_solve_backward, which runs the
adjoint solve (the operator is symmetric) and assembles dl/df, dl/ds,
dl/dbeta and dl/dsigma in the library's kernels, and nfl_form_grad_nodes for
dl/dv = beta d(lambda^T A u)/dv; this module only passes tensors and scalars
between torch and the library.
"""
import torch

from .nfl import Plan


class _CGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, shift, beta, sigma, v, plan, dplan, tol, maxit):
        u, _, _, _ = plan.cg_solve(f.detach(), beta=float(beta), shift=shift.detach(), tol=tol, maxit=maxit)
        ctx.save_for_backward(u, shift, v)
        ctx.plan, ctx.dplan, ctx.beta, ctx.tol, ctx.maxit = plan, dplan, float(beta), tol, maxit
        return u

    @staticmethod
    def backward(ctx, g):
        u, shift, v = ctx.saved_tensors
        want_sigma = ctx.dplan is not None and ctx.needs_input_grad[3]
        want_v = ctx.needs_input_grad[4]
        gf, gs, gb, gsig, _, _ = ctx.plan.cg_solve_backward(
            u, g.contiguous(), beta=ctx.beta, shift=shift, dplan=ctx.dplan if want_sigma else None,
            tol=ctx.tol, maxit=ctx.maxit, want_shift=ctx.needs_input_grad[1])
        dev, dt = g.device, g.dtype
        grad_beta = torch.tensor(gb, device=dev, dtype=dt) if ctx.needs_input_grad[2] else None
        grad_sigma = torch.tensor(gsig, device=dev, dtype=dt) if want_sigma else None
        # dl/dv = -beta lambda^T (dL_s/dv) u = beta d(lambda^T A u)/dv
        grad_v = ctx.beta * ctx.plan.form_grad_nodes(v.detach(), gf, u) if want_v else None
        return gf, gs, grad_beta, grad_sigma, grad_v, None, None, None, None


def cg_solve(plan, f, shift, beta, sigma=None, dplan=None, tol=1e-10, maxit=1000, v=None):
    """u = (beta L_s + diag(shift))^{-1} f, differentiable in f, shift, beta, sigma and v.

    plan   the Gaussian Plan of the nodes (built with the value of sigma).
    beta   a 0-d tensor (or float); sigma a 0-d tensor holding the plan's sigma,
           whose gradient needs dplan, the GAUSSIAN_DSIGMA Plan of the same nodes
           and parameters.
    v      the (n, d) node tensor the plan was built from, when dl/dv is wanted.
    """
    if not isinstance(plan, Plan):
        raise TypeError("plan must be a Plan")
    dev = f.device
    beta_t = beta if isinstance(beta, torch.Tensor) else torch.tensor(float(beta), device=dev, dtype=torch.float64)
    sigma_t = sigma if isinstance(sigma, torch.Tensor) else torch.tensor(0.0, device=dev, dtype=torch.float64)
    v_t = v if v is not None else torch.zeros((), device=dev, dtype=torch.float64)
    return _CGSolve.apply(f, shift, beta_t, sigma_t, v_t, plan, dplan, tol, maxit)
