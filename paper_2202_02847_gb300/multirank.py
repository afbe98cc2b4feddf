"""Multi-GPU bookkeeping of the benchmark: one independent problem per rank.

Translations never exchange data, so the ranks shard the work as independent
octrees (weak scaling) and only two collectives run, both outside the data
path: a barrier around the timed region and the maximum of the per-rank
times.  The aggregate rate is the sum of all ranks' units over that maximum.
"""
import torch
import torch.distributed as dist


def rank_seed(base_seed, rank):
    """Seed of rank r's synthetic problem (rank 0 keeps the base seed)."""
    return base_seed + rank


def aggregate_rate(local_units, local_seconds, device=None):
    """(sum of units over ranks) / (max of seconds over ranks), and that max.

    Works on one process (no process group) and under any backend."""
    if not (dist.is_available() and dist.is_initialized()):
        return local_units / local_seconds, local_seconds
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())
