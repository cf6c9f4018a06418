"""Exact exchange sharded over ranks with torch.distributed.

Pair solves are independent (arXiv 1712.07973, Sec. 2.1: the paper
distributes orbital pairs over MPI ranks in a round-robin and sends the
potentials back); here each rank processes its own pair tiles
(exx_plan_set_shard: largest-first assignment, balanced to one tile) on its own
GPU, and the only exchange is one all-reduce of the partial E_x and one of the
partial Vx psi (or gradient).  Use a plan with FP64 output (``vx_fp64=True``
or FP64 precision) to sum the partial actions in FP64.
"""

import torch
import torch.distributed as dist

__all__ = ["sharded_apply"]


def sharded_apply(plan, psi, group=None, out=None, gradient=False, sync=True):
    """Full E_x and Vx psi (gradient=True: dE_x/dpsi = 2 f_k h^3 (Vx psi)_k)
    on every rank of ``group``.  Returns (E_x, out): E_x a float when sync,
    else the one-element FP64 device tensor (no host synchronisation)."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    plan.set_shard(rank, world)
    if out is None:
        out = torch.empty(psi.shape, dtype=plan.vx_dtype, device=psi.device)
    E = torch.zeros(1, dtype=torch.float64, device=psi.device)
    if gradient:
        plan.gradient_async(psi, out, E)
    else:
        plan.apply_async(psi, out, E)
    dist.all_reduce(E, group=group)
    dist.all_reduce(out, group=group)
    return (float(E.item()) if sync else E), out
