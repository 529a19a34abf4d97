"""Differentiable LR-SPIKE solve: x = A(theta)^{-1} f with theta the band
values of A, as a torch.autograd.Function.

Forward: LR-SPIKE factorisation of A and the outer iteration to the handle's
tolerance (x = A^{-1} f, not M^{-1} f).  Backward, for an incoming gradient
g = dL/dx: the adjoint solve A^T lambda = g with the same factors
(lrspike_solve_transpose: the outer iteration with M^{-T}), then
dL/df = lambda and dL/dA = -lambda x^T restricted to the band
(lrspike_band_outer).  Every step runs in the CUDA library; this module only
marshals tensors.
"""
from __future__ import annotations

import torch

from .solver import LRSpike, band_outer


class LRSpikeSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, band, f, k, p, r, kwargs):
        n = band.shape[1]
        A = band.detach().contiguous()
        s = LRSpike(n, k, p, r, **kwargs)
        s.factor(A)
        x, _ = s.solve(f.detach().contiguous())
        x = x.clone()
        ctx.solver, ctx.band, ctx.k = s, A, k   # the library borrows A until the handle closes
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, _ = ctx.solver.solve_transpose(gx.contiguous())
        grad_band = grad_f = None
        if ctx.needs_input_grad[0]:
            grad_band = torch.empty_like(ctx.band)
            band_outer(lam, x, ctx.k, -1.0, grad_band)
        if ctx.needs_input_grad[1]:
            grad_f = lam.clone()
        return grad_band, grad_f, None, None, None, None


def solve(band: torch.Tensor, f: torch.Tensor, k: int, p: int, r: int, **kwargs) -> torch.Tensor:
    """x = A^{-1} f, differentiable in the band values of A and in f.
    band: (2k+1, n) float64 on the GPU, band[k + i - j, j] = A[i, j];
    f: (n,) or (nrhs, n) float64; kwargs: LRSpike options (precision, tol,
    reduced, outer, ...).  The default tolerance is 1e-12 (FP64)."""
    return LRSpikeSolveFn.apply(band, f, k, p, r, kwargs)
