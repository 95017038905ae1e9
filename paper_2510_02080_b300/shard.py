"""One map's submap fusion on several GPUs, one process each.

Registration pairs are independent (Sec. III-C registers each submap pair on
its own), so they are split across ranks by a balanced partition of their
correspondence counts and registered with no collective; only the tiny Sim(3)
results travel to the rank that owns the pose graph (Sec. III-E), which
solves it and broadcasts the corrected poses.  Fusion shards submaps: each
rank compacts its own submaps under those poses, and one all-gather of a
single int64 (its kept count) gives every rank its offset in the global point
buffer, so the global indices stay exact.  Timing takes the maximum over
ranks.  Works with any torch.distributed backend (gloo on CPU in the tests,
NCCL on GPUs); without an initialised process group everything is one rank.

``map_step`` runs the whole step through a ``kernels`` object with three
calls (register, pose_graph, fuse); ``GpuKernels`` gives them the library's
CUDA path on one device.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import torch
import torch.distributed as dist


def _world(group=None) -> tuple[int, int]:
    if not dist.is_available() or not dist.is_initialized():
        return 1, 0
    return dist.get_world_size(group), dist.get_rank(group)


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
    ws, rank = _world(group)
    if ws == 1:
        return 0, int(local_count)
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
    ws, rank = _world(group)
    if ws == 1:
        return local
    width = local.shape[1]
    n_max = max(e - s for s, e in ranges)
    buf = torch.zeros((n_max, width), dtype=local.dtype, device=local.device)
    buf[:local.shape[0]] = local
    out = [torch.zeros_like(buf) for _ in range(ws)] if rank == dst else None
    dist.gather(buf, out, dst=dst, group=group)
    if rank != dst:
        return None
    return torch.cat([out[r][:e - s] for r, (s, e) in enumerate(ranges)])


def broadcast_rows(rows: torch.Tensor | None, n: int, width: int, src: int = 0, group=None,
                   device=None) -> torch.Tensor:
    """Rows [n, width] (float64) of rank ``src`` on every rank."""
    ws, rank = _world(group)
    if ws == 1:
        return rows
    if rank != src:
        rows = torch.empty((n, width), dtype=torch.float64, device=device)
    dist.broadcast(rows, src=src, group=group)
    return rows


def max_over_ranks(value: float, group=None) -> float:
    if _world(group)[0] == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def local_links(link_off, src, tgt, a: int, b: int):
    """The links of pairs [a, b) over a compact bank of just the frames they
    use: (link_off [b-a+1], src, tgt re-indexed, frames = the global frame of
    every local one, in first-use order).  Host int32 tensors in, out."""
    lo = [int(v) for v in link_off[a:b + 1].tolist()]
    s = [int(v) for v in src[lo[0]:lo[-1]].tolist()]
    t = [int(v) for v in tgt[lo[0]:lo[-1]].tolist()]
    where: dict[int, int] = {}
    for f in s + t:
        where.setdefault(f, len(where))
    i32 = dict(dtype=torch.int32)
    return (torch.tensor([v - lo[0] for v in lo], **i32),
            torch.tensor([where[f] for f in s], **i32),
            torch.tensor([where[f] for f in t], **i32),
            torch.tensor(list(where), dtype=torch.int64))


@dataclass
class ShardPlan:
    """This rank's share of one map (host data, made once per map)."""
    ranges: list           # pair range of every rank
    pairs: tuple           # this rank's pairs [a, b)
    link_off: torch.Tensor  # its links, over its local frames (int32)
    src: torch.Tensor
    tgt: torch.Tensor
    frames: torch.Tensor   # global frame of every local frame (int64)
    submaps: tuple         # the submaps it fuses [m0, m1)
    n_nodes: int


def plan_shard(link_off, src, tgt, sizes, n_nodes, group=None) -> ShardPlan:
    """Splits the pairs (balanced by their correspondence counts ``sizes``)
    and the submaps over the ranks of ``group``."""
    world, rank = _world(group)
    ranges = partition_pairs(sizes, world)
    a, b = ranges[rank]
    lo, ls, lt, frames = local_links(link_off, src, tgt, a, b)
    m = partition_pairs([1] * n_nodes, world)[rank]
    return ShardPlan(ranges, (a, b), lo, ls, lt, frames, m, n_nodes)


def map_step(kernels, plan: ShardPlan, xyz, conf, ei, ej, sub_xyz, sub_conf,
             pts_per_submap: int, pair_conf_min=None, pg_rank: int = 0, group=None) -> dict:
    """One map through registration, pose graph and fusion on every rank.

    xyz / conf: this rank's frames (the global frames plan.frames, in that
    order; [n, hw, 3] / [n, hw]); pair_conf_min: its pairs' thresholds or
    None.  Pair k of the map is the pose-graph edge (ei[k], ej[k]) (host
    arrays, every pair).  sub_xyz / sub_conf: its submaps plan.submaps ([m, n,
    3] / [m, n], n = pts_per_submap).  This rank registers its pairs; the
    Sim(3) rows meet on ``pg_rank``, which solves the pose graph and
    broadcasts the corrected poses; this rank fuses its submaps at its offset
    in the global point buffer (global flat indices m * n + i).

    Returns dict(rows = every pair's Sim(3) row on pg_rank, None elsewhere;
    poses [n_nodes, 13] on every rank; points, indices = this rank's fused
    points and their global indices; offset = their position in the global
    buffer, total = its length)."""
    world, rank = _world(group)
    rows = kernels.register(xyz, conf, plan.link_off, plan.src, plan.tgt, pair_conf_min)
    all_rows = gather_rows(rows, plan.ranges, dst=pg_rank, group=group)
    poses = kernels.pose_graph(plan.n_nodes, ei, ej, all_rows) if rank == pg_rank else None
    poses = broadcast_rows(poses, plan.n_nodes, 13, src=pg_rank, group=group,
                           device=rows.device)
    m0, m1 = plan.submaps
    pts, idx = kernels.fuse(sub_xyz, sub_conf, poses[m0:m1], m0 * pts_per_submap)
    off, total = exclusive_offsets(int(idx.shape[0]), group=group)
    return dict(rows=all_rows, poses=poses, points=pts, indices=idx, offset=off, total=total)


class GpuKernels:
    """map_step's calls on the library's CUDA path (one ec3r.Context on the
    device of the tensors it is given); every step runs in the library's
    kernels.  With ``adjoint``, the registration is followed by its backward
    call for the upstream gradient adjoint(n_pairs) -> (dL/dS [n,13],
    dL/dcost [n]), reusing the forward's checkpoints; the gradients are kept in
    ``self.grads``."""

    def __init__(self, ctx, delta=0.02, iters=10, pg_iters=10, adjoint=None):
        self.ctx, self.delta, self.iters, self.pg_iters = ctx, delta, iters, pg_iters
        self.adjoint = adjoint
        self.grads = None
        self._dev = {}

    def _on(self, t, dev):
        """Host index tensors moved to the device once."""
        key = (id(t), str(dev))
        if key not in self._dev:
            self._dev[key] = (t, t.to(dev))
        return self._dev[key][1]

    def register(self, xyz, conf, link_off, src, tgt, pair_conf_min):
        dev = xyz.device
        n = int(link_off.numel()) - 1
        if n == 0:                                     # no pair on this rank
            return torch.zeros((0, 13), dtype=torch.float64, device=dev)
        lo, s, t = self._on(link_off, dev), self._on(src, dev), self._on(tgt, dev)
        S, _, _ = self.ctx.align_submaps(xyz, conf, lo, s, t, pair_conf_min, delta=self.delta,
                                         iters=self.iters, want_cost=self.adjoint is not None)
        if self.adjoint is not None:
            gS, gc = self.adjoint(n)
            self.grads = self.ctx.align_submaps_backward(
                xyz, conf, lo, s, t, gS, gc, pair_conf_min, delta=self.delta, iters=self.iters,
                fwd_token=self.ctx.align_token())
        return S

    def pose_graph(self, n, ei, ej, rows):
        nodes = torch.zeros((n, 13), dtype=torch.float64, device=rows.device)
        nodes[:, 0] = 1.0
        nodes[:, [1, 5, 9]] = 1.0
        self.ctx.pose_graph_correct(nodes, ei, ej, rows.contiguous(), iters=self.pg_iters)
        return nodes

    def fuse(self, xyz, conf, poses, index_base):
        m = int(conf.shape[0])
        cap = max(int(conf.numel()), 1)
        dev = poses.device
        out_xyz = torch.empty((cap, 3), dtype=torch.float32, device=dev)
        out_idx = torch.empty((cap,), dtype=torch.int64, device=dev)
        cursor = torch.zeros((1,), dtype=torch.int64, device=dev)
        if m:
            self.ctx.fuse_points(xyz, conf, poses.contiguous(), out_xyz, out_idx, cursor,
                                 index_base=index_base)
        k = int(cursor.item())
        return out_xyz[:k], out_idx[:k]
