"""log Z as a differentiable function of a likelihood or prior parameter.

Forward: one nested-sampling run on the GPU (nss_create, nss_run).
Backward: the Fisher identity (the gradient of log Z is the posterior mean of
the gradient of log L + log Pi), estimated over the run's weighted dead points
by the library's device kernel (nss_posterior_expectation); no autodiff
through the sampler, which is not differentiable.

    theta = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    z = logz(theta, lambda s: workload.with_(sigma=float(s)), native.GRAD_LIK_SIGMA)
    z.backward()            # theta.grad = d log Z / d sigma

The estimate carries the run's statistical error (``last_logz_err``); the
gradient's own spread is of the same order relative to its scale.
"""
from __future__ import annotations

import torch

from . import native

last_logz_err = None


class LogZ(torch.autograd.Function):
    """log Z(theta) by one run; theta's gradient from the device Fisher kernel."""

    @staticmethod
    def forward(ctx, theta, build, kind):
        global last_logz_err
        wl = build(theta.detach().cpu().numpy())
        with native.Sampler(wl) as s:
            r = s.run()[0]
            g = s.posterior(kind)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device).reshape(theta.shape))
        last_logz_err = r["logZ_err"]
        return torch.tensor(r["logZ"], dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None


def logz(theta, build, kind):
    """log Z at theta: build(theta as numpy) returns the workload; kind is one
    of native.GRAD_LIK_SIGMA, GRAD_LIK_MU, GRAD_PRIOR_LOG_PREC (the parameter
    theta stands for, in the units that kind differentiates)."""
    return LogZ.apply(theta, build, kind)
