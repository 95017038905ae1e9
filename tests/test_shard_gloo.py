"""Gloo ranks on CPU (2, 3 and 7) run the sharded path's host logic: balanced pair
partition, registration of each shard (the FP64 oracle stands in for the
GPU, which this host lacks), gather of the Sim(3) rows on rank 0, fusion of
each rank's submaps with offsets from one all-gathered count, and the
max-over-ranks time.  The result must equal the single-process one."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_02080_b300 import shard


def test_partition_is_balanced_contiguous_and_complete():
    sizes = [5, 1, 1, 1, 9, 2, 2, 7, 3, 3]
    for world in (1, 2, 3, 4, 16):
        parts = shard.partition_pairs(sizes, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(sizes) and len(parts) == world
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
    loads = [sum(sizes[a:b]) for a, b in shard.partition_pairs(sizes, 2)]
    assert max(loads) - min(loads) <= max(sizes)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import fuse as ofuse
    from oracle import register as reg
    from paper_2510_02080_b300 import synth

    ch = synth.make_chain(synth.SEED_BASE + 21, M=6, F=2, H=20, W=28, device="cpu")
    ps = ch.pairs()
    sizes = [ps.hw] * ps.n_pairs
    ranges = shard.partition_pairs(sizes, world)
    a, b = ranges[rank]
    res = reg.align_pairs(ps, pairs=list(range(a, b)))
    rows = torch.tensor(np.stack([np.concatenate([[r["S"][0]], np.ravel(r["S"][1]), r["S"][2]])
                                  for r in res]) if res else np.zeros((0, 13)))
    allrows = shard.gather_rows(rows, ranges)
    # fusion: submaps split the same balanced way
    sub = shard.partition_pairs([1] * ch.M, world)[rank]
    xyz = ch.xyz.view(ch.M, -1, 3)[sub[0]:sub[1]].numpy()
    conf = ch.conf.view(ch.M, -1)[sub[0]:sub[1]].numpy()
    n = conf.shape[1] if conf.size else ch.xyz[0].numel() // 3
    poses = [(1.0, np.eye(3), np.zeros(3))] * (sub[1] - sub[0])
    ox, oi = ofuse.fuse_points(xyz, conf, poses, 1.0, index_base=sub[0] * n)
    off, total = shard.exclusive_offsets(len(oi))
    idx = [torch.zeros(total, dtype=torch.int64) for _ in range(world)]
    mine = torch.zeros(total, dtype=torch.int64)
    mine[off:off + len(oi)] = torch.from_numpy(oi)
    dist.all_reduce(mine)                       # each slot written by exactly one rank
    t = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        torch.save({"rows": allrows, "idx": mine, "t": t}, result_path)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 3, 7])
def test_gloo_ranks_match_single_process(tmp_path, world):
    """2 ranks: even shares; 3: uneven (5 pairs, 6 submaps); 7: more ranks than
    submaps, so one rank registers and fuses nothing."""
    from oracle import fuse as ofuse
    from oracle import register as reg
    from paper_2510_02080_b300 import synth

    path = str(tmp_path / "res.pt")
    mp.start_processes(_worker, args=(world, _free_port(), path), nprocs=world, join=True,
                       start_method="spawn")
    got = torch.load(path)
    ch = synth.make_chain(synth.SEED_BASE + 21, M=6, F=2, H=20, W=28, device="cpu")
    ps = ch.pairs()
    ref = reg.align_pairs(ps)
    ref_rows = np.stack([np.concatenate([[r["S"][0]], np.ravel(r["S"][1]), r["S"][2]]) for r in ref])
    assert np.array_equal(got["rows"].numpy(), ref_rows)
    _, ref_idx = ofuse.fuse_points(ch.xyz.view(ch.M, -1, 3).numpy(), ch.conf.view(ch.M, -1).numpy(),
                                   [(1.0, np.eye(3), np.zeros(3))] * ch.M, 1.0)
    assert np.array_equal(got["idx"].numpy(), ref_idx)
    assert got["t"] == float(world)


class OracleKernels:
    """map_step's three calls on the FP64 oracle (this host has no GPU; the
    oracle stands in for the library's kernels, nothing else)."""

    def __init__(self, H, W):
        self.H, self.W = H, W

    def register(self, xyz, conf, link_off, src, tgt, pcm):
        from oracle import register as reg
        from paper_2510_02080_b300 import synth
        if link_off.numel() == 1:
            return torch.zeros((0, 13), dtype=torch.float64)
        res = reg.align_pairs(synth.PairSet(xyz, conf, link_off, src, tgt, self.H, self.W,
                                            pair_conf_min=pcm))
        return torch.tensor(np.stack([np.concatenate([[r["S"][0]], np.ravel(r["S"][1]),
                                                      r["S"][2]]) for r in res]))

    def pose_graph(self, n, ei, ej, rows):
        from oracle import pose_graph as opg
        R = rows.numpy()
        Tij = [(float(r[0]), r[1:10].reshape(3, 3), r[10:13]) for r in R]
        init = opg.chain_init(n, ei, ej, Tij)
        nodes, _, _ = opg.gauss_newton(init, ei, ej, Tij, iters=2)
        return torch.tensor(np.stack([np.concatenate([[T[0]], np.ravel(T[1]), T[2]])
                                      for T in nodes]))

    def fuse(self, xyz, conf, poses, index_base):
        from oracle import fuse as ofuse
        P = poses.numpy()
        ox, oi = ofuse.fuse_points(xyz.numpy(), conf.numpy(),
                                   [(float(p[0]), p[1:10].reshape(3, 3), p[10:13]) for p in P],
                                   1.0, index_base=index_base)
        return torch.from_numpy(ox), torch.from_numpy(oi)


def _map(world=1, rank=0):
    """The test map (a 7-submap chain with one loop pair) and this rank's plan."""
    from paper_2510_02080_b300 import synth
    ch = synth.make_chain(synth.SEED_BASE + 22, M=7, F=2, H=20, W=28, device="cpu")
    ps = ch.pairs()
    # a loop pair: submap 6 (frame 12) registered onto submap 0 (frame 1)
    link_off = torch.cat([ps.link_off, torch.tensor([ps.n_pairs + 1], dtype=torch.int32)])
    src = torch.cat([ps.src, torch.tensor([12], dtype=torch.int32)])
    tgt = torch.cat([ps.tgt, torch.tensor([1], dtype=torch.int32)])
    ei = np.concatenate([np.arange(6), [0]]).astype(np.int32)
    ej = np.concatenate([np.arange(1, 7), [6]]).astype(np.int32)
    sizes = [ps.hw] * 7
    return ch, ps, link_off, src, tgt, ei, ej, sizes


def _map_worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ch, ps, link_off, src, tgt, ei, ej, sizes = _map()
    plan = shard.plan_shard(link_off, src, tgt, sizes, ch.M)
    m0, m1 = plan.submaps
    n = ch.F * ch.H * ch.W
    out = shard.map_step(OracleKernels(ch.H, ch.W), plan, ps.xyz[plan.frames],
                         ps.conf[plan.frames], ei, ej, ch.xyz.view(ch.M, -1, 3)[m0:m1],
                         ch.conf.view(ch.M, -1)[m0:m1], n)
    # assemble the global buffer: every slot is written by exactly one rank
    idx = torch.zeros(out["total"], dtype=torch.int64)
    pts = torch.zeros((out["total"], 3), dtype=torch.float64)
    o, k = out["offset"], out["indices"].shape[0]
    idx[o:o + k] = out["indices"]
    pts[o:o + k] = out["points"]
    dist.all_reduce(idx)
    dist.all_reduce(pts)
    poses = [torch.zeros_like(out["poses"]) for _ in range(world)]
    dist.all_gather(poses, out["poses"])
    if rank == 0:
        torch.save({"rows": out["rows"], "poses": poses, "idx": idx, "pts": pts,
                    "frames": [int(v) for v in plan.frames]}, result_path)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 3])
def test_map_step_on_gloo_ranks_equals_one_process(tmp_path, world):
    """One map split over 2 or 3 ranks: each registers its share of the pairs
    over only the frames they use, the rows meet on rank 0, which solves the
    pose graph (chain + one loop edge) and broadcasts the poses, and each rank
    fuses its submaps at its offset.  Rows, poses on every rank, fused indices
    and points equal those of one process, bit for bit."""
    path = str(tmp_path / "map.pt")
    mp.start_processes(_map_worker, args=(world, _free_port(), path), nprocs=world, join=True,
                       start_method="spawn")
    got = torch.load(path)
    ch, ps, link_off, src, tgt, ei, ej, sizes = _map()
    plan = shard.plan_shard(link_off, src, tgt, sizes, ch.M)
    assert plan.pairs == (0, 7) and plan.submaps == (0, 7)
    ref = shard.map_step(OracleKernels(ch.H, ch.W), plan, ps.xyz[plan.frames],
                         ps.conf[plan.frames], ei, ej, ch.xyz.view(ch.M, -1, 3),
                         ch.conf.view(ch.M, -1), ch.F * ch.H * ch.W)
    assert torch.equal(got["rows"], ref["rows"])
    for p in got["poses"]:
        assert torch.equal(p, ref["poses"])
    assert torch.equal(got["idx"], ref["indices"]) and torch.equal(got["pts"], ref["points"])
    # rank 0 held only the frames of its own pairs
    assert len(got["frames"]) < ps.xyz.shape[0]
