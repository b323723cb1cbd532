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


class ScoreBatchFn(torch.autograd.Function):
    """The energies of several ligands' poses in one launch per
    atoms-per-lane width (adg_score_multi); rows padded to MAX_GENES."""

    @staticmethod
    def forward(fctx, genes, ctx, rec, ligs, npose):
        if genes.dtype != torch.float32 or not genes.is_cuda:
            raise TypeError("genes must be a float32 CUDA tensor")
        energy, grad = adg.score_multi(ctx, rec, ligs, genes.detach().contiguous(), npose, adg.GRAD_GENES)
        fctx.save_for_backward(grad)
        return energy

    @staticmethod
    def backward(fctx, grad_energy):
        (grad,) = fctx.saved_tensors
        return grad_energy.to(grad.dtype)[:, None] * grad, None, None, None, None


def score_rows(rows: torch.Tensor, ctx: "adg.Context", rec: "adg.Receptor", ligs, npose) -> torch.Tensor:
    """Differentiable docking energies of packed genotype rows (float32 CUDA
    [sum(npose), MAX_GENES]; ligand i owns npose[i] consecutive rows, its 7+T
    genes in front) in one launch per atoms-per-lane width."""
    return ScoreBatchFn.apply(rows, ctx, rec, list(ligs), [int(k) for k in npose])


def score_batch(genes_list, ctx: "adg.Context", rec: "adg.Receptor", ligs) -> list:
    """Differentiable docking energies of several ligands' genotypes
    (genes_list[i]: float32 CUDA [npose_i, 7+T_i]) in one launch per width;
    returns the per-ligand energy tensors.  Gradients flow back to every
    genes_list[i] through the padding and concatenation."""
    npose = [int(g.shape[0]) for g in genes_list]
    rows = torch.cat([torch.nn.functional.pad(g, (0, adg.MAX_GENES - g.shape[1])) for g in genes_list], 0)
    energy = ScoreBatchFn.apply(rows, ctx, rec, list(ligs), npose)
    return list(torch.split(energy, npose))

