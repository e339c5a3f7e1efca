"""Host-side logic of multi-GPU runs: independent replicas (weak scaling).

Every rank evaluates its own batch of samples; samples are independent for
the local energy and O_k, so no collective touches the data path.  The only
communication is timing: a barrier on both sides of the timed region and
the maximum elapsed time over ranks.  The SR solve stays per rank (its S v
would need an all-reduce of an n-vector per CG step to pool the ranks'
samples; the library has no such exchange).
"""
from __future__ import annotations


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    import os
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def seed_offset(rank: int) -> int:
    """Input-stream offset of a rank, so replicas draw different samples."""
    return 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar (elapsed ms) over all ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(samples_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job samples/s: all ranks' samples over the slowest rank's time."""
    return world * samples_per_rank * steps / (max_ms / 1e3)
