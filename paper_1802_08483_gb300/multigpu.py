"""Frame sharding across GPUs (one process per GPU).

Frames are independent, so the decoder shards them: rank r decodes its own
frames and no collective touches the data path (weak scaling: every rank keeps
the same per-GPU work).  The only collectives combine the timing and the
decoded-bit count at the end of a measurement: the maximum step time over
ranks and the sum of bits.
"""
from __future__ import annotations


def frame_indices(rank: int, world: int, frames_per_rank: int):
    """Workload frame indices decoded by `rank` (its own seeded frames)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    start = rank * frames_per_rank
    return list(range(start, start + frames_per_rank))


def combine(ms_per_step: float, bits_per_step: float, dist=None, device="cpu"):
    """(max step time over ranks, total bits over ranks)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(ms_per_step), float(bits_per_step)
    import torch
    t = torch.tensor([float(ms_per_step)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([float(bits_per_step)], dtype=torch.float64, device=device)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())
