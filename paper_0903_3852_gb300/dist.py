"""Host-side logic of multi-GPU runs: one process per GPU, each integrating
its own copy of the workload with its own noise key (the ensemble method has no
exchange step, so no data-path collective), timing reduced by maximum.

Used by bench.py under torchrun (NCCL) and tested on CPU with gloo ranks.
"""
import os

RANK_SEED_STRIDE = 1000


def rank_info():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed, rank):
    """Noise key of a rank: distinct Philox keys give independent ensembles."""
    return seed + RANK_SEED_STRIDE * rank


def max_over_ranks(value, device="cpu"):
    """Maximum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max
