"""Frame sharding across ranks (one process per GPU).

Frames are independent, so a batch is split into contiguous frame-id ranges,
one per rank, with no exchange while decoding; each rank passes its range's
first id as the schedule's frame_base, so every frame draws the same
permutation events as in an unsplit run.  The only collective is a sum of
integer counters (frames, frame errors, bit errors, iterations) at the end.
"""
from __future__ import annotations


def shard_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) frame ids of `rank` when `total` frames are split over `world` ranks."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


COUNTERS = ("frames", "frame_errors", "bit_errors", "iterations")


def reduce_counters(counts: dict, group=None) -> dict:
    """Sum the integer counters over all ranks (torch.distributed all_reduce)."""
    import torch
    import torch.distributed as dist

    vec = torch.tensor([int(counts.get(k, 0)) for k in COUNTERS], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            vec = vec.cuda()
        dist.all_reduce(vec, op=dist.ReduceOp.SUM, group=group)
    return {k: int(v) for k, v in zip(COUNTERS, vec.cpu().tolist())}
