"""Replicas over disjoint event ranges: the multi-GPU form of the hot path.

Events are independent, so N GPUs each run the whole pipeline on their own
contiguous range of events with the weights replicated and no data exchange.
Only the measurement combines ranks: the job's time is the slowest rank's,
its work the sum over ranks (events and hits). `event_range` gives each rank
its own block of a fixed size (weak scaling, as the benchmark runs);
`balanced_ranges` splits one fixed set of events into contiguous ranges of
about equal hit counts (strong scaling).
"""
from __future__ import annotations


def event_range(rank: int, world: int, per_rank: int) -> tuple[int, int]:
    """(first event, count) of `rank`: per_rank events each (weak scaling),
    rank r taking events [r * per_rank, (r + 1) * per_rank)."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError(f"rank {rank} of {world}, {per_rank} events per rank")
    return rank * per_rank, per_rank


def balanced_ranges(hits_per_event, world: int) -> list[tuple[int, int]]:
    """Contiguous (first event, count) of each of `world` ranks over a fixed
    set of events, balanced by hit count (the work of an event grows with its
    hits): rank r takes the events whose cumulative hit count, taken at each
    event's midpoint, falls in [r, r + 1) x total / world. Every event goes to
    exactly one rank, in order; a rank may get none when events are fewer
    than ranks."""
    import numpy as np
    if world < 1:
        raise ValueError(f"world {world}")
    h = np.asarray(hits_per_event, dtype=np.float64)
    if np.any(h < 0):
        raise ValueError("negative hit count")
    total = float(h.sum())
    if total <= 0.0:
        mid = (np.arange(h.size) + 0.5) / max(h.size, 1)
    else:
        mid = (np.cumsum(h) - 0.5 * h) / total
    owner = np.minimum((mid * world).astype(np.int64), world - 1)
    out = []
    for r in range(world):
        idx = np.nonzero(owner == r)[0]
        out.append((int(idx[0]), int(idx.size)) if idx.size else (int(np.searchsorted(owner, r)), 0))
    return out


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
