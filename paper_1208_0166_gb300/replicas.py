"""Replica bookkeeping for multi-GPU runs.

The multilevel path is run as independent replicas, one Markov chain per GPU with its
own seed, and no collective on the data path.  The only cross-rank operations are the
barrier around the timed region and this aggregation: the whole-job time is the slowest
rank's time and the whole-job work is the sum over ranks.
"""
from __future__ import annotations


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of the chain on `rank`: distinct per rank, base_seed on rank 0."""
    return int(base_seed) + int(rank)


def aggregate(local_seconds: float, local_units: float, dist=None, device=None):
    """(max over ranks of local_seconds, sum over ranks of local_units); the local values
    when dist is None (single process)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_seconds), float(local_units)
    import torch

    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
