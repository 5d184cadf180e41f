"""log Z of the SV auxiliary LGSSM as a differentiable function of theta.

theta = (mu, phi, L, delta) of the multivariate stochastic-volatility model
(Section 4.1): F = diag(phi), b = (I - F) mu, Q = L L^T, stationary p_0,
R = (delta/2) I; the pseudo-observations ytilde are held fixed. The forward
pass, the gradient and the theta -> model map all run in the CUDA library
(aux_loglik_grad, aux_set_sv_theta); this module marshals theta and applies the
chain rule to the upstream gradient. sv_model_arrays states the same map on the
host for callers that build a model description themselves.
"""
import numpy as np
import torch

from . import _binding as B


def sv_model_arrays(mu, phi, L, delta):
    """Host LGSSM arrays (float64 numpy) of theta."""
    mu = np.asarray(mu, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    L = np.tril(np.asarray(L, dtype=np.float64))
    Q = L @ L.T
    return dict(m0=mu.copy(), P0=Q / (1.0 - np.outer(phi, phi)), F=np.diag(phi),
                b=(1.0 - phi) * mu, Q=Q, delta=float(delta))


def set_theta(sampler, mu, phi, L, delta):
    """Write theta into an existing AuxKalman handle (aux_set_sv_theta: the library
    forms F, b, Q and the stationary p_0 on the device)."""
    B.aux_set_sv_theta(sampler.handle, mu, phi, L, delta)


class SVLogZ(torch.autograd.Function):
    """logZ[c] = log p(ytilde[c] | theta) for every chain c; differentiable in theta."""

    @staticmethod
    def forward(ctx, mu, phi, L, delta, ytilde, sampler):
        set_theta(sampler, mu.detach().cpu().numpy(), phi.detach().cpu().numpy(),
                  L.detach().cpu().numpy(), float(delta))
        C, d = sampler.C, sampler.d
        dev = ytilde.device
        logZ = torch.empty(C, dtype=torch.float64, device=dev)
        g_mu = torch.empty(C, d, dtype=torch.float64, device=dev)
        g_phi = torch.empty(C, d, dtype=torch.float64, device=dev)
        g_L = torch.empty(C, d, d, dtype=torch.float64, device=dev)
        g_delta = torch.empty(C, dtype=torch.float64, device=dev)
        B.aux_loglik_grad(sampler.handle, ytilde, g_mu, g_phi, g_L, g_delta, logZ)
        ctx.save_for_backward(g_mu, g_phi, g_L, g_delta)
        ctx.dtypes = (mu.dtype, mu.device)
        return logZ

    @staticmethod
    def backward(ctx, grad_out):
        g_mu, g_phi, g_L, g_delta = ctx.saved_tensors
        dt, dev = ctx.dtypes
        w = grad_out.to(torch.float64)
        return ((w[:, None] * g_mu).sum(0).to(dev, dt), (w[:, None] * g_phi).sum(0).to(dev, dt),
                (w[:, None, None] * g_L).sum(0).to(dev, dt), (w * g_delta).sum().to(dev, dt),
                None, None)
