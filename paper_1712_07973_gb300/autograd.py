"""Exact-exchange energy as a differentiable PyTorch function.

The gradient of the discrete exchange energy is the exchange action itself
(arXiv 1712.07973, Eq. daction, the Fock operator being the functional
derivative of E_X with respect to the density matrix): for real orbitals and a
symmetric kernel G,

    E_x = -(alpha/2) sum_ij f_i f_j h^3 rho_ij^T G rho_ij
    dE_x/dpsi_k = -2 alpha h^3 f_k sum_j f_j V_kj psi_j = 2 f_k h^3 (Vx psi)_k.

The library computes that gradient directly (exx_gradient: the per-orbital
factor 2 f_k h^3 is folded into its FP64 accumulation), from the same pair
solves as E_x.  ``ExxEnergy.forward`` runs exx_gradient when a gradient is
needed (the gradient is kept for backward) and exx_energy otherwise.  With
``recompute=True`` the forward runs exx_energy only and the backward recomputes
the pair solves with exx_gradient, so nothing the size of the orbitals is kept
between the two passes.  No V_ij is ever stored.  The backward's only tensor
operation is the chain rule's product with the incoming scalar grad_out, in
the orbitals' own dtype.

``ExxBatchEnergy`` does the same for a batch of molecules of uneven size
(ExxBatch, exx_batch_gradient): one CUDA-graph launch per call gives every
molecule's E_x and gradient.
"""

import torch

from .exx import ExxBatch, ExxPlan

__all__ = ["ExxEnergy", "exx_energy", "ExxBatchEnergy", "exx_batch_energy"]


def _chain(g, grad_out):
    # dL/dpsi = dL/dE * dE/dpsi; grad_out is a device scalar (1 for E.backward())
    return g * grad_out.to(g.dtype)


class ExxEnergy(torch.autograd.Function):
    """E_x(psi) with its gradient dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k.

    forward: exx_gradient when a gradient will be needed (the library returns
    E_x and the gradient; the gradient is kept for the backward), exx_energy
    otherwise or with recompute=True (the backward then runs exx_gradient).
    backward: the library's gradient times grad_out.
    """

    @staticmethod
    def forward(ctx, psi, plan, recompute=False):
        if not isinstance(plan, ExxPlan):
            raise TypeError("plan must be an ExxPlan")
        ctx.plan = plan
        ctx.recompute = bool(recompute)
        need_grad = ctx.needs_input_grad[0]
        if need_grad and not recompute:
            E, g = plan.gradient(psi)
            ctx.save_for_backward(g)
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
            _, g = plan.gradient(saved)
        else:
            g = saved
        grad = _chain(g, grad_out)
        if grad.dtype != plan.dtype:  # FP32 plans with FP64 output
            grad = grad.to(plan.dtype)
        return grad, None, None


def exx_energy(psi, plan, recompute=False):
    """Differentiable E_x(psi) for a plan (see ExxEnergy)."""
    return ExxEnergy.apply(psi, plan, recompute)


class ExxBatchEnergy(torch.autograd.Function):
    """E_x of every molecule of a batch (FP64 tensor [nmol]) with the gradients
    2 f_k h^3 (Vx psi)_k of each molecule's orbitals (exx_batch_gradient).

    forward(batch, *psis): binds the orbitals (and, when gradients are
    needed, fresh output tensors) to the batch and runs one batched call;
    backward: each molecule's gradient times its entry of grad_out.
    """

    @staticmethod
    def forward(ctx, batch, *psis):
        if not isinstance(batch, ExxBatch):
            raise TypeError("batch must be an ExxBatch")
        need = any(ctx.needs_input_grad[1:])
        # one energy buffer per batch, so that a captured graph (which embeds
        # its address) is replayed rather than captured again
        E = getattr(batch, "_autograd_E", None)
        if E is None or E.device != psis[0].device:
            E = torch.zeros(batch.nmol, dtype=torch.float64, device=psis[0].device)
            batch._autograd_E = E
        if need:
            gs = [torch.empty_like(p) for p in psis]
            batch.set_buffers(list(psis), gs)
            batch.gradient(E)
            ctx.save_for_backward(*gs)
        else:
            batch.set_buffers(list(psis), None)
            batch.energy(E)
        return E.clone()

    @staticmethod
    def backward(ctx, grad_E):
        gs = ctx.saved_tensors
        return (None,) + tuple(_chain(g, grad_E[m]) for m, g in enumerate(gs))


def exx_batch_energy(batch, psis):
    """Differentiable per-molecule E_x of a batch (see ExxBatchEnergy)."""
    return ExxBatchEnergy.apply(batch, *psis)
