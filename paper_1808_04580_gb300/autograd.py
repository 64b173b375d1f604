"""Differentiable solve of (beta L_s + diag(s)) u = f (Sec. 6.2.2) for torch autograd.

Forward: nfl_cg_solve.  Backward: nfl_cg_solve_backward, which runs the
adjoint solve (the operator is symmetric) and assembles dl/df, dl/ds,
dl/dbeta and dl/dsigma in the library's kernels; this module only passes
tensors and scalars between torch and the library.
"""
import torch

from .nfl import Plan


class _CGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, shift, beta, sigma, plan, dplan, tol, maxit):
        u, _, _, _ = plan.cg_solve(f.detach(), beta=float(beta), shift=shift.detach(), tol=tol, maxit=maxit)
        ctx.save_for_backward(u, shift)
        ctx.plan, ctx.dplan, ctx.beta, ctx.tol, ctx.maxit = plan, dplan, float(beta), tol, maxit
        return u

    @staticmethod
    def backward(ctx, g):
        u, shift = ctx.saved_tensors
        want_sigma = ctx.dplan is not None and ctx.needs_input_grad[3]
        gf, gs, gb, gsig, _, _ = ctx.plan.cg_solve_backward(
            u, g.contiguous(), beta=ctx.beta, shift=shift, dplan=ctx.dplan if want_sigma else None,
            tol=ctx.tol, maxit=ctx.maxit, want_shift=ctx.needs_input_grad[1])
        dev, dt = g.device, g.dtype
        grad_beta = torch.tensor(gb, device=dev, dtype=dt) if ctx.needs_input_grad[2] else None
        grad_sigma = torch.tensor(gsig, device=dev, dtype=dt) if want_sigma else None
        return gf, gs, grad_beta, grad_sigma, None, None, None, None


def cg_solve(plan, f, shift, beta, sigma=None, dplan=None, tol=1e-10, maxit=1000):
    """u = (beta L_s + diag(shift))^{-1} f, differentiable in f, shift, beta and sigma.

    plan   the Gaussian Plan of the nodes (built with the value of sigma).
    beta   a 0-d tensor (or float); sigma a 0-d tensor holding the plan's sigma,
           whose gradient needs dplan, the GAUSSIAN_DSIGMA Plan of the same nodes
           and parameters.
    """
    if not isinstance(plan, Plan):
        raise TypeError("plan must be a Plan")
    dev = f.device
    beta_t = beta if isinstance(beta, torch.Tensor) else torch.tensor(float(beta), device=dev, dtype=torch.float64)
    sigma_t = sigma if isinstance(sigma, torch.Tensor) else torch.tensor(0.0, device=dev, dtype=torch.float64)
    return _CGSolve.apply(f, shift, beta_t, sigma_t, plan, dplan, tol, maxit)
