"""The potential Phi(x) as a differentiable torch function.

Forward and backward both come from the library's adjoint gradient
(``smc_gradient``: a forward and an adjoint Darcy solve per row, then the
transposed KL synthesis), computed once in the forward pass; the backward pass
only scales the stored gradient.  The drift D Phi of a Langevin-type mutation
(the Langevin equation of App. B with gamma != 0).
"""
import torch


class PotentialFunction(torch.autograd.Function):
    """Phi for each row of X (FP64, on the sampler's device); dPhi/dX in backward."""

    @staticmethod
    def forward(ctx, X, sampler):
        if X.dtype != torch.float64 or not X.is_cuda or X.dim() != 2:
            raise ValueError("X must be a 2-D float64 CUDA tensor (rows of KL coordinates)")
        X = X.contiguous()
        Phi = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        G = torch.empty_like(X)
        sampler.smc_gradient(X, Phi, G)
        ctx.save_for_backward(G)
        return Phi

    @staticmethod
    def backward(ctx, grad_phi):
        (G,) = ctx.saved_tensors
        return grad_phi.to(G.dtype)[:, None] * G, None


def potential(X, sampler):
    """Phi(X) with autograd support; ``sampler`` is a ``smcgm.Sampler`` built with gradient=1."""
    return PotentialFunction.apply(X, sampler)
