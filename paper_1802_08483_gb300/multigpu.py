"""Frame sharding across GPUs (one process per GPU).

Frames are independent, so the decoder shards them: rank r decodes its own
frames and no collective touches the data path.  The benchmark gives every
rank its own seeded frames (weak scaling: every rank keeps the same per-GPU
work) and combines only the timing and the decoded-bit count: the maximum step
time over ranks and the sum of bits.  For a fixed set of frames (strong
scaling) `lpt_partition` balances the ranks by estimated cost, `gather_results`
collects APPs and log-likelihoods on rank 0 in one gather, and a shared-channel
gradient needs one all-reduce of three sums (`allreduce_channel_grad`).
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


def frame_cost(fr) -> float:
    """Estimated work of one frame (the algorithmic flop count's dominant terms:
    lattice nodes plus the two q-contractions over the valid transitions)."""
    M = 2 * fr.xmax + 1
    MN = fr.n * (fr.I + 1) + 1
    cells = (fr.I + 1) * fr.n * (fr.n + 1) // 2 + fr.n
    lattice = (fr.rho + 1) * fr.q * cells * (2 * fr.I + 3)
    return float(2 * lattice + 4 * fr.q * fr.N * M * MN)


def lpt_partition(costs, world: int):
    """Longest-processing-time assignment of frames to `world` ranks: frames in
    decreasing cost, each to the currently least loaded rank (ties: lowest
    rank).  Returns one sorted index list per rank; deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    import heapq
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k))
    for k in order:
        load, r = heapq.heappop(heap)
        parts[r].append(k)
        heapq.heappush(heap, (load + float(costs[k]), r))
    return [sorted(p) for p in parts]


def allreduce_channel_grad(dchan_sum, dist=None):
    """Sum over ranks of the channel-parameter gradient (3 values: d/dPi, d/dPd,
    d/dPs summed over a rank's frames) for a channel shared by every frame: the
    one collective a data-parallel gradient step needs."""
    import torch
    t = torch.as_tensor(dchan_sum, dtype=torch.float64).reshape(3).clone()
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def gather_results(parts, app_per_rank, ll_per_rank, dist=None, world: int = 1):
    """Rank 0 view of every frame's APPs and log-likelihood after decoding the
    frames listed in `parts` (one list per rank): one object gather.  Returns
    (apps, lls) indexed by the global frame number on rank 0, None elsewhere."""
    mine = (list(app_per_rank), list(ll_per_rank))
    if dist is None or not dist.is_available() or not dist.is_initialized():
        gathered = [mine]
    else:
        gathered = [None] * world if dist.get_rank() == 0 else None
        dist.gather_object(mine, gathered, dst=0)
        if dist.get_rank() != 0:
            return None
    nframes = sum(len(p) for p in parts)
    apps, lls = [None] * nframes, [None] * nframes
    for r, (a, l) in enumerate(gathered):
        for k, f in enumerate(parts[r]):
            apps[f] = a[k]
            lls[f] = l[k]
    return apps, lls
