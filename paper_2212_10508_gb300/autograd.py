"""SNAP energy as a differentiable torch function over the library's kernels.

forward : E[b] = sum_i (beta_0 + sum_t beta_t B_t^i) -- the U_tot and bispectrum stages only;
          dE/dbeta = (natoms, sum_i B_t^i) comes out of the same launch and is kept.
backward: dE/dr from the adjoint pass (Y = dE/dU, then the per-neighbour contraction and the
          deterministic force gather), dE/dbeta from the kept bispectrum sums; both are scaled
          by the incoming gradient.  A second derivative is not provided.
"""
import torch

from . import snap_energy_forces


class SnapEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, beta, snap, box):
        E, _, S = snap_energy_forces(snap, pos, box, beta, energy=True, forces=False, sumB=True)
        ctx.save_for_backward(pos, beta, S)
        ctx.snap = snap
        ctx.box = tuple(float(x) for x in box)
        return E

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gE):
        pos, beta, S = ctx.saved_tensors
        gpos = gbeta = None
        if ctx.needs_input_grad[0]:
            _, F, _ = snap_energy_forces(ctx.snap, pos, ctx.box, beta, energy=False, forces=True)
            gpos = -gE.to(F.dtype)[:, None, None] * F
        if ctx.needs_input_grad[1]:
            gbeta = (gE.to(S.dtype)[:, None] * S).sum(0)
        return gpos, gbeta, None, None


def snap_energy(pos, beta, snap, box):
    """Differentiable SNAP energies [nbatch] of positions pos [nbatch,3,natoms] (float64, CUDA)."""
    return SnapEnergy.apply(pos.contiguous(), beta.contiguous(), snap, box)
