"""torch.autograd.Function over the energy+gradient kernel (adg_score).

Forward evaluates the docking energy E(genes) of a batch of genotypes
[t(3), q(4), theta(T)] in one launch that also forms the analytic gradient
dE/dgenes (the gradient the ADADELTA local search of the paper's Sec. 1.1
follows); backward returns grad_output * dE/dgenes.  Both run in libadg.so;
PyTorch only carries the tensors.
"""
from __future__ import annotations

import torch

from . import adg


class ScoreFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, genes, ctx, rec, lig):
        if genes.dtype != torch.float32 or not genes.is_cuda:
            raise TypeError("genes must be a float32 CUDA tensor")
        g = genes.detach().contiguous()
        energy, grad = adg.score(ctx, rec, lig, g, adg.GRAD_GENES)
        fctx.save_for_backward(grad)
        return energy

    @staticmethod
    def backward(fctx, grad_energy):
        (grad,) = fctx.saved_tensors
        return grad_energy.to(grad.dtype)[:, None] * grad, None, None, None


def score(genes: torch.Tensor, ctx: "adg.Context", rec: "adg.Receptor", lig: "adg.Ligand") -> torch.Tensor:
    """Differentiable docking energy of genotypes [npose, 7+T] (float32, CUDA)."""
    return ScoreFn.apply(genes, ctx, rec, lig)
