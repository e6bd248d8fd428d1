"""Dose as a differentiable function of the voxel densities.

``dose(rho, engine, ...)`` runs the forward transport with the densities
``rho`` (a float32 CUDA tensor shaped like the phantom) and returns the dose
per voxel (MeV/g per history, float64). Its backward pass calls the library's
path-replay adjoint (``gbmc_adjoint``): each history of a second, independent
set is run twice from its Philox key, and dL/drho is the likelihood-ratio
estimate for the incoming dL/dD. The forward and adjoint histories are
different sets (different seeds), so the gradient estimate is unbiased for the
dose's expectation. All arithmetic runs in the library's kernels; this module
only moves pointers.
"""
from __future__ import annotations

import torch

from . import Engine


class _Dose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, engine: Engine, phantom, mat, n_hist, seed, first_hist,
                adj_hist, adj_seed, adj_first):
        rho_c = rho.detach().contiguous()
        engine.load_phantom(phantom, mat=mat, rho=rho_c)
        engine.run(n_hist, seed=seed, first_hist=first_hist)
        out = torch.empty(rho_c.numel(), dtype=torch.float64, device=rho_c.device)
        engine.dose(out=out, var=None)
        ctx.engine, ctx.phantom, ctx.mat = engine, phantom, mat
        ctx.adj = (adj_hist, adj_seed, adj_first)
        ctx.save_for_backward(rho_c)
        return out.view(rho.shape)

    @staticmethod
    def backward(ctx, grad_dose):
        (rho_c,) = ctx.saved_tensors
        eng = ctx.engine
        # the engine may have been used since: put this call's densities back
        eng.load_phantom(ctx.phantom, mat=ctx.mat, rho=rho_c)
        g = grad_dose.detach().to(torch.float64).contiguous().view(-1)
        grad = torch.empty_like(g)
        n, seed, first = ctx.adj
        eng.adjoint(g, n, seed=seed, first_hist=first, out=grad, var=None)
        return (grad.view(rho_c.shape).to(rho_c.dtype),) + (None,) * 9


def dose(rho: torch.Tensor, engine: Engine, phantom, mat: torch.Tensor, n_hist: int,
         seed: int = 1, first_hist: int = 0, adj_hist: int | None = None,
         adj_seed: int | None = None, adj_first: int = 0) -> torch.Tensor:
    """Dose (MeV/g per history) of ``n_hist`` histories with densities ``rho``;
    differentiable in ``rho`` through the path-replay adjoint with ``adj_hist``
    histories (default ``n_hist``) of seed ``adj_seed`` (default seed + 1).
    ``phantom`` supplies the grid (shape, dx, dy, dz); ``mat`` is the uint8
    material tensor on the same device as ``rho``."""
    if not rho.is_cuda or rho.dtype != torch.float32:
        raise ValueError("rho must be a float32 CUDA tensor")
    return _Dose.apply(rho, engine, phantom, mat, n_hist, seed, first_hist,
                       adj_hist if adj_hist is not None else n_hist,
                       adj_seed if adj_seed is not None else seed + 1, adj_first)
