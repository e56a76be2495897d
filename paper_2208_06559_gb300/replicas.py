"""Replica (multi-GPU) bookkeeping for independent chain ensembles.

The paper distributes independent chains over MPI ranks with no messages
between them (Sec. 4, simulation methodology).  Here each rank drives one GPU
with its own batch of chains; the only collectives are the timing barrier and
the max-over-ranks reduction of the measured time, so the data path has no
exchange step (weak scaling).
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed: int, rank: int) -> int:
    """Disjoint seeds per rank: the ranks simulate different chains."""
    return int(base_seed) + 1000003 * int(rank)


def aggregate(ms_local: float, units_local: float, world: int, device=None):
    """Whole-job throughput of independent replicas: total units over the
    slowest rank's time.  Returns (units_total, ms_max)."""
    import torch
    if world <= 1:
        return float(units_local), float(ms_local)
    import torch.distributed as dist
    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(sm[1].item()), float(mx[0].item())
