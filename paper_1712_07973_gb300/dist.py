"""Exact exchange sharded over ranks with torch.distributed.

Each rank processes its own pair tiles (exx_plan_set_shard: largest-first
assignment, balanced to one tile) on its own GPU; the partial E_x and Vx psi
are summed with one all-reduce each.  Use a plan with FP64 output
(``vx_fp64=True`` or FP64 precision) so the partial actions are summed in FP64.
"""

import torch
import torch.distributed as dist

__all__ = ["sharded_apply"]


def sharded_apply(plan, psi, group=None, out=None):
    """Full E_x (float) and Vx psi on every rank of ``group``."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    plan.set_shard(rank, world)
    if out is None:
        out = torch.empty(psi.shape, dtype=plan.vx_dtype, device=psi.device)
    E = torch.zeros(1, dtype=torch.float64, device=psi.device)
    plan.apply_async(psi, out, E)
    dist.all_reduce(E, group=group)
    dist.all_reduce(out, group=group)
    return float(E.item()), out
