"""Exact-exchange energy as a differentiable PyTorch function.

The gradient of the discrete exchange energy is the exchange action itself
(arXiv 1712.07973, Eq. daction, the Fock operator being the functional
derivative of E_X with respect to the density matrix): for real orbitals and a
symmetric kernel G,

    E_x = -(alpha/2) sum_ij f_i f_j h^3 rho_ij^T G rho_ij
    dE_x/dpsi_k = -2 alpha h^3 f_k sum_j f_j V_kj psi_j = 2 f_k h^3 (Vx psi)_k.

``ExxEnergy.forward`` runs exx_apply when a gradient is needed (E_x and
Vx psi from the same pair solves; Vx psi is kept for backward) and exx_energy
otherwise.  With ``recompute=True`` the forward runs exx_energy only and the
backward recomputes the pair solves with exx_apply, so nothing the size of the
orbitals is kept between the two passes.  No V_ij is ever stored.
"""

import torch

from .exx import ExxPlan

__all__ = ["ExxEnergy", "exx_energy"]


class ExxEnergy(torch.autograd.Function):
    """E_x(psi) with its gradient dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k.

    forward: exx_apply when a gradient will be needed (the action is kept for
    the backward), exx_energy otherwise or with recompute=True (the backward
    then runs exx_apply again).  backward: the library's exchange action
    times the per-orbital factor 2 f_k h^3 grad_out (one elementwise product
    on the returned tensor; every pair solve runs in the library).
    """

    @staticmethod
    def forward(ctx, psi, plan, recompute=False):
        if not isinstance(plan, ExxPlan):
            raise TypeError("plan must be an ExxPlan")
        ctx.plan = plan
        ctx.recompute = bool(recompute)
        need_grad = ctx.needs_input_grad[0]
        if need_grad and not recompute:
            E, vx = plan.apply(psi)
            ctx.save_for_backward(vx)
        else:
            E = plan.energy(psi)
            if need_grad:
                ctx.save_for_backward(psi)
        return torch.tensor(E, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        (saved,) = ctx.saved_tensors
        if ctx.recompute:
            _, vx = plan.apply(saved)
        else:
            vx = saved
        occ = torch.as_tensor(plan.occ, dtype=torch.float64, device=vx.device)
        scale = (2.0 * plan.h ** 3) * occ.view(-1, 1, 1, 1) * grad_out.to(torch.float64)
        grad = (vx.to(torch.float64) * scale).to(plan.dtype)
        return grad, None, None


def exx_energy(psi, plan, recompute=False):
    """Differentiable E_x(psi) for a plan (see ExxEnergy)."""
    return ExxEnergy.apply(psi, plan, recompute)
