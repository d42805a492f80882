"""Replica timing for runs on several GPUs of one node.

One product does not shard across GPUs (every level of the product needs the
neighbouring blocks of the previous one), so N GPUs run N independent replicas of the
same product.  The whole-job time of a step is the slowest replica's; the throughput is
the work of all replicas over that time.
"""
from __future__ import annotations


def slowest(ms: float, dist=None, device=None) -> float:
    """Largest per-step time over the ranks of the default process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(bytes_per_replica: float, world: int, ms: float) -> float:
    """GB/s of all replicas together for a step time of `ms` milliseconds."""
    return bytes_per_replica * world / (ms * 1e-3) / 1e9
