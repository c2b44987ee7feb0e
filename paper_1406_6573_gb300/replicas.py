"""Multi-GPU bookkeeping for independent replicas.

The operator path is run as independent replicas, one per GPU and process:
every rank applies the whole workload on its own device and no collective
touches the data path.  A job's time is the slowest rank's time and its
throughput counts the units of every rank.  These helpers are the only
collectives of a multi-rank run (two scalars per measurement).
"""
import torch
import torch.distributed as dist


def world_size():
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def max_over_ranks(value, device="cpu"):
    """The maximum of a per-rank scalar over all ranks (the value itself on one rank)."""
    if world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device="cpu"):
    if world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank, seconds_per_rank, device="cpu"):
    """Whole-job rate: units summed over ranks / the slowest rank's seconds."""
    return sum_over_ranks(units_per_rank, device) / max_over_ranks(seconds_per_rank, device)
