"""torch.autograd.Function over the likelihood kernels.

LogLik.apply(theta, model, precision, obs) returns log p(y | theta_p) for each
row of theta ([P, d] float64, CUDA).  The forward pass runs the adjoint kernel
(smc_loglik_grad), which produces the log likelihood and its gradient in one
sweep when theta requires a gradient (the plain likelihood kernel otherwise);
backward scales the saved gradient by the incoming one.  All arithmetic is in
libsmc.so; torch supplies the buffers and the stream.
"""
from __future__ import annotations

import torch

from . import smc


class LogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model, precision, obs):
        if theta.dim() != 2 or theta.dtype != torch.float64 or not theta.is_cuda:
            raise ValueError("theta must be a CUDA float64 tensor of shape [P, d]")
        P, d = theta.shape
        th = theta.detach().t().contiguous()
        ll = torch.empty(P, dtype=torch.float64, device=theta.device)
        if theta.requires_grad:
            grad = torch.empty((d, P), dtype=torch.float64, device=theta.device)
            smc.loglik_grad(model, precision, obs, th, ll, grad)
            ctx.save_for_backward(grad)
        else:
            smc.loglik(model, precision, obs, th, ll)
        return ll

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return g_out[:, None] * grad.t(), None, None, None


def loglik(theta, model, precision, obs):
    return LogLik.apply(theta, model, precision, obs)
