"""Host-side logic of multi-GPU runs: replicas only.

The docking path shards into independent (ligand, run) units with no
exchange during a run (paper Sec. 1.1: nrun independent LGA runs; Sec. 2.2:
one job per ligand), so N GPUs run N independent replicas: each rank docks
its own share of the ligands and the only collective is the end-of-run
reduction of timings and counts for reporting -- none on the data path.
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> list:
    """Round-robin share of item indices for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, n_items, world))


def reduce_run(total_ms: float, units: float, dist=None, device=None):
    """(max over ranks of the elapsed time, sum over ranks of the units).
    `dist` is torch.distributed (any backend) or None for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return total_ms, units
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
