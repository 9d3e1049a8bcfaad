"""Replicas over disjoint event ranges: the multi-GPU form of the hot path.

Events are independent, so N GPUs each run the whole pipeline on their own
contiguous range of events with the weights replicated and no data exchange.
Only the measurement combines ranks: the job's time is the slowest rank's,
its work the sum over ranks (events and hits).
"""
from __future__ import annotations


def event_range(rank: int, world: int, per_rank: int) -> tuple[int, int]:
    """(first event, count) of `rank`: per_rank events each (weak scaling),
    rank r taking events [r * per_rank, (r + 1) * per_rank)."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError(f"rank {rank} of {world}, {per_rank} events per rank")
    return rank * per_rank, per_rank


def combine(dist, local_ms: float, local_events: int, local_hits: int, device=None):
    """Job totals: (max over ranks of local_ms, sum of events, sum of hits).
    `dist` is torch.distributed (or None for one process); `device` the
    device of the collective's tensors (a CUDA device for NCCL, CPU for gloo)."""
    if dist is None:
        return float(local_ms), int(local_events), int(local_hits)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(local_events), float(local_hits)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n[0].item())), int(round(n[1].item()))
