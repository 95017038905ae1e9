"""Host-side logic for running the path on several GPUs, one process each.

Registration pairs are independent, so they are split across ranks by a
balanced partition of their correspondence counts and registered with no
collective; only the tiny Sim(3) results travel to the rank that owns the pose
graph.  Fusion shards submaps: each rank compacts its own submaps and one
all-gather of a single int64 (its kept count) gives every rank its offset in
the global point buffer, so the global indices stay exact.  Timing takes the
maximum over ranks.  Works with any torch.distributed backend (gloo on CPU in
the tests, NCCL on GPUs).
"""
from __future__ import annotations

from typing import Sequence

import torch
import torch.distributed as dist


def partition_pairs(sizes: Sequence[int], world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [start, end) of pairs, one per rank, balancing the sum
    of ``sizes`` (correspondences per pair).  Deterministic; ranks may be empty."""
    n = len(sizes)
    total = float(sum(sizes))
    bounds = [0]
    acc = 0.0
    k = 0
    for r in range(1, world):
        target = total * r / world
        while k < n and acc + sizes[k] / 2.0 <= target:
            acc += sizes[k]
            k += 1
        bounds.append(k)
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def exclusive_offsets(local_count: int, group=None) -> tuple[int, int]:
    """(offset of this rank, total) for counts summed in rank order."""
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    t = torch.tensor([int(local_count)], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(out, t, group=group)
    counts = [int(x.item()) for x in out]
    return sum(counts[:rank]), sum(counts)


def gather_rows(local: torch.Tensor, ranges: list[tuple[int, int]], dst: int = 0,
                group=None) -> torch.Tensor | None:
    """Gather per-pair result rows ([n_local, C]) of every rank on rank ``dst``,
    in pair order; other ranks get None."""
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    width = local.shape[1]
    n_max = max(e - s for s, e in ranges)
    buf = torch.zeros((n_max, width), dtype=local.dtype, device=local.device)
    buf[:local.shape[0]] = local
    out = [torch.zeros_like(buf) for _ in range(ws)] if rank == dst else None
    dist.gather(buf, out, dst=dst, group=group)
    if rank != dst:
        return None
    return torch.cat([out[r][:e - s] for r, (s, e) in enumerate(ranges)])


def max_over_ranks(value: float, group=None) -> float:
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
