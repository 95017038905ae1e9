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
