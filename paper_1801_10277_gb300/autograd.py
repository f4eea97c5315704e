"""torch.autograd.Function for the ELBO: the forward pass evaluates the ELBO (E / Var
maps and the expected log-likelihood), the backward pass runs the hand-written adjoint
kernel, which recomputes every mixture term from the forward's E / Var maps instead of
storing them.  Argument marshalling only: both passes run in libceleste's kernels."""
from __future__ import annotations

import torch

from . import celeste


class ELBO(torch.autograd.Function):
    """ELBO(theta) for a celeste.Problem; theta is a CUDA float64 tensor [n_src, 44]."""

    @staticmethod
    def forward(ctx, theta, problem, precision=celeste.FP32):
        if not (theta.is_cuda and theta.dtype == torch.float64):
            raise TypeError("theta must be a CUDA float64 tensor")
        th = theta.detach().contiguous()
        total = torch.zeros(1, dtype=torch.float64, device=theta.device)
        problem.elbo_device(th, total, None, precision=precision)
        ctx.problem, ctx.precision = problem, precision
        ctx.generation = problem.generation
        ctx.save_for_backward(th)
        return total[0]

    @staticmethod
    def backward(ctx, grad_out):
        (th,) = ctx.saved_tensors
        pr = ctx.problem
        if pr.generation != ctx.generation:
            # another evaluation replaced the maps: rebuild this theta's maps first
            total = torch.zeros(1, dtype=torch.float64, device=th.device)
            pr.elbo_device(th, total, None, precision=ctx.precision)
        g = torch.empty_like(th)
        pr.grad_device(th, g, precision=ctx.precision)
        return grad_out * g, None, None


def elbo(theta, problem, precision=celeste.FP32):
    """Differentiable ELBO of `problem` at `theta` (see ELBO)."""
    return ELBO.apply(theta, problem, precision)
