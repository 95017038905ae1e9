"""GPU parity of ec3r_fuse_points (confidence-filtered global transform,
Sec. III-C Point Correction) against the FP64 oracle: indices bit-exact,
points within 1e-6 x scene extent."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import fuse as ofuse
from paper_2510_02080_b300 import ec3r, synth

pytestmark = pytest.mark.gpu
POINT_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def rand_poses(rng, M):
    s = rng.uniform(0.5, 2.0, M)
    R = Rotation.random(M, random_state=rng).as_matrix()
    t = rng.normal(size=(M, 3)) * 3
    rows = np.concatenate([s[:, None], R.reshape(M, 9), t], 1)
    return rows, [(s[m], R[m], t[m]) for m in range(M)]


def run_fuse(ctx, xyz, conf, rows, thr=1.0, index_base=0, capacity=None, cursor0=0):
    M = xyz.shape[0]
    xyz_d = torch.tensor(xyz, device="cuda").reshape(M, -1, 3).contiguous()
    conf_d = torch.tensor(conf, device="cuda").reshape(M, -1).contiguous()
    poses = torch.tensor(rows, dtype=torch.float64, device="cuda")
    cap = int(conf.size) if capacity is None else capacity
    out_xyz = torch.full((max(cap, 1), 3), -7.0, device="cuda")
    out_idx = torch.full((max(cap, 1),), -7, dtype=torch.int64, device="cuda")
    cursor = torch.tensor([cursor0], dtype=torch.int64, device="cuda")
    ctx._check(ctx._lib.ec3r_fuse_points(
        ctx._h, M, conf_d.shape[1], ec3r._ptr(xyz_d), ec3r._ptr(conf_d), ec3r._ptr(poses),
        float(thr), int(index_base), ec3r._ptr(out_xyz), ec3r._ptr(out_idx), cap,
        ec3r._ptr(cursor), ec3r._stream(None)))
    st = ctx.sync_status()
    return out_xyz.cpu().numpy(), out_idx.cpu().numpy(), int(cursor.item()), st


def extent(X):
    """Bounding-box diagonal of the fused points (at least their magnitude,
    so that a one-point map still has a scale)."""
    if len(X) == 0:
        return 1.0
    return max(float(np.linalg.norm(X.max(0) - X.min(0))), float(np.abs(X).max()))


@pytest.mark.parametrize("shape", [(3, 2, 33, 51), (2, 2, 64, 130), (1, 1, 1, 3)])
def test_fuse_matches_oracle(ctx, shape):
    M, F, H, W = shape
    rng = np.random.default_rng(sum(shape))
    xyz = (rng.normal(size=(M, F * H * W, 3)) * 4).astype(np.float32)
    conf = rng.lognormal(0, 0.5, size=(M, F * H * W)).astype(np.float32)
    conf.reshape(-1)[:: 97] = 1.0          # ties are dropped (strict >)
    conf.reshape(-1)[5:: 131] = np.nan
    rows, poses = rand_poses(rng, M)
    ox, oi = ofuse.fuse_points(xyz, conf, poses, 1.0, index_base=11)
    gx, gi, cur, st = run_fuse(ctx, xyz, conf, rows, 1.0, index_base=11)
    assert st == 0 and cur == len(oi)
    assert np.array_equal(gi[:cur], oi)
    assert (gi[cur:] == -7).all()
    assert np.abs(gx[:cur] - ox).max(initial=0.0) <= POINT_TOL * extent(ox)


def test_streaming_cursor_and_capacity(ctx):
    rng = np.random.default_rng(3)
    xyz = (rng.normal(size=(2, 9000, 3))).astype(np.float32)
    conf = rng.lognormal(0, 0.5, size=(2, 9000)).astype(np.float32)
    rows, poses = rand_poses(rng, 2)
    ox, oi = ofuse.fuse_points(xyz, conf, poses)
    K = len(oi)
    # capacity too small: nothing written past it, cursor still advances
    gx, gi, cur, st = run_fuse(ctx, xyz, conf, rows, capacity=K // 2)
    assert st == 4                       # EC3R_ERR_CAPACITY
    assert cur == K
    assert np.array_equal(gi[:K // 2], oi[:K // 2])
    # starting at a cursor offset
    gx, gi, cur, st = run_fuse(ctx, xyz, conf, rows, capacity=K + 100, cursor0=100)
    assert st == 0 and cur == K + 100
    assert np.array_equal(gi[100:], oi) and (gi[:100] == -7).all()


def test_all_dropped_and_all_kept(ctx):
    rng = np.random.default_rng(4)
    xyz = rng.normal(size=(2, 4100, 3)).astype(np.float32)
    rows, poses = rand_poses(rng, 2)
    _, gi, cur, st = run_fuse(ctx, xyz, np.zeros((2, 4100), np.float32), rows)
    assert cur == 0 and st == 0
    _, gi, cur, st = run_fuse(ctx, xyz, np.full((2, 4100), 5.0, np.float32), rows)
    assert cur == 8200 and np.array_equal(gi, np.arange(8200))


def test_full_size_chain_sampled_submaps(ctx):
    """All 200 x 5 x 294 x 518 points of the benchmark chain; the oracle
    recomputes sampled submaps and their offsets."""
    ch = synth.make_chain(synth.SEED_BASE + 2, M=200, F=5, H=294, W=518, device="cuda")
    M = ch.M
    n = ch.F * ch.H * ch.W
    rng = np.random.default_rng(5)
    rows, poses = rand_poses(rng, M)
    xyz = ch.xyz.reshape(M, n, 3)
    conf = ch.conf.reshape(M, n)
    keep = (conf > 1.0)
    K = int(keep.sum())
    out_xyz = torch.empty((K, 3), device="cuda")
    out_idx = torch.empty((K,), dtype=torch.int64, device="cuda")
    cursor = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.fuse_points(xyz, conf, torch.tensor(rows, device="cuda"), out_xyz, out_idx, cursor)
    assert ctx.sync_status() == 0 and int(cursor) == K
    before = torch.cumsum(keep.sum(1), 0).cpu().numpy()
    for m in (0, 77, 199):
        start = int(before[m - 1]) if m else 0
        ox, oi = ofuse.fuse_points(xyz[m:m + 1].cpu().numpy(), conf[m:m + 1].cpu().numpy(),
                                   [poses[m]], 1.0, index_base=m * n)
        gi = out_idx[start:start + len(oi)].cpu().numpy()
        gx = out_xyz[start:start + len(oi)].cpu().numpy()
        assert np.array_equal(gi, oi)
        assert np.abs(gx - ox).max() <= POINT_TOL * extent(ox)


@pytest.mark.parametrize("shape", [(3, 2, 33, 51), (2, 5, 294, 62)])
def test_count_then_scatter_equals_one_call(ctx, shape):
    """ec3r_fuse_count + ec3r_fuse_points_counted produce exactly what one
    ec3r_fuse_points call produces (points, indices, cursor), several tiles
    and a ragged last tile per submap, streaming after a non-zero cursor;
    and exactly the oracle's indices."""
    M, F, H, W = shape
    rng = np.random.default_rng(11)
    xyz = rng.normal(size=(M, F * H * W, 3)).astype(np.float32)
    conf = rng.lognormal(0.0, 0.5, size=(M, F * H * W)).astype(np.float32)
    conf[0, :5] = np.nan
    rows, Ts = rand_poses(rng, M)
    ref_xyz, ref_idx, ref_cur, st = run_fuse(ctx, xyz, conf, rows, index_base=3, cursor0=17)
    assert st == 0
    xyz_d = torch.tensor(xyz, device="cuda")
    conf_d = torch.tensor(conf, device="cuda")
    poses = torch.tensor(rows, dtype=torch.float64, device="cuda")
    out_xyz = torch.full((conf.size, 3), -7.0, device="cuda")
    out_idx = torch.full((conf.size,), -7, dtype=torch.int64, device="cuda")
    cursor = torch.tensor([17], dtype=torch.int64, device="cuda")
    counts, mask = ctx.fuse_count(conf_d)
    n = F * H * W
    tps = (n + 8191) // 8192
    assert counts.numel() == M * tps
    # the mask is the keep predicate, bit by bit, zero past each tile's end
    words = mask.cpu().numpy().view(np.uint32).reshape(M, tps, 256)
    bits = ((words[..., None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(M, tps * 8192)
    with np.errstate(invalid="ignore"):
        np.testing.assert_array_equal(bits[:, :n], (conf > 1.0).astype(np.uint32))
    assert not bits[:, n:].any()
    np.testing.assert_array_equal(counts.cpu().numpy().reshape(M, tps).sum(1),
                                  bits.sum(1))
    ctx.fuse_points_counted(xyz_d, counts, mask, poses, out_xyz, out_idx, cursor, index_base=3)
    assert ctx.sync_status() == 0
    assert int(cursor.item()) == ref_cur
    np.testing.assert_array_equal(out_idx.cpu().numpy(), ref_idx)
    np.testing.assert_array_equal(out_xyz.cpu().numpy(), ref_xyz)
    _, idx = ofuse.fuse_points(xyz.astype(np.float64), conf.astype(np.float64), Ts,
                               index_base=3)
    np.testing.assert_array_equal(out_idx.cpu().numpy()[17:ref_cur], idx)


def test_count_arguments(ctx):
    conf = torch.ones((2, 100), device="cuda")
    with pytest.raises(ValueError):
        ctx.fuse_count(conf, torch.empty((1,), dtype=torch.int32, device="cuda"))
    with pytest.raises(ec3r.Ec3rError):
        ctx.fuse_count(conf, threshold=float("nan"))
    counts = torch.empty((2,), dtype=torch.int32, device="cuda")
    st = ctx._lib.ec3r_fuse_count(ctx._h, 2, 100, ec3r._ptr(conf), 1.0, ec3r._ptr(counts), None,
                                  ec3r._stream(None))
    assert st == 1  # EC3R_ERR_INVALID_ARG: no mask buffer


@pytest.mark.timeout(1800)
def test_config5_map_fusion_sampled_submaps(ctx):
    """The large map: all 1000 x 5 x 392 x 518 = 1,015,280,000 points fused in
    one call under the submaps' true poses; the oracle recomputes sampled
    submaps, whose output offsets come from keep counts taken on the host."""
    ch = synth.make_chain(synth.SEED_BASE + 5, M=1000, F=5, H=392, W=518, device="cuda")
    M = ch.M
    n = ch.F * ch.H * ch.W
    s, R, t = (v.cpu().numpy() for v in (ch.T_gt.s, ch.T_gt.R, ch.T_gt.t))
    rows = np.concatenate([s[:, None], R.reshape(M, 9), t], 1)
    xyz = ch.xyz.reshape(M, n, 3)
    conf = ch.conf.reshape(M, n)
    counts = np.array([int((conf[m].cpu().numpy() > 1.0).sum()) for m in range(M)])
    K = int(counts.sum())
    out_xyz = torch.empty((K, 3), device="cuda")
    out_idx = torch.empty((K,), dtype=torch.int64, device="cuda")
    cursor = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.fuse_points(xyz, conf, torch.tensor(rows, device="cuda"), out_xyz, out_idx, cursor)
    assert ctx.sync_status() == 0 and int(cursor) == K
    before = np.concatenate([[0], np.cumsum(counts)])
    for m in (0, 437, 998, 999):
        start = int(before[m])
        ox, oi = ofuse.fuse_points(xyz[m:m + 1].cpu().numpy(), conf[m:m + 1].cpu().numpy(),
                                   [(s[m], R[m], t[m])], 1.0, index_base=m * n)
        assert len(oi) == counts[m]
        gi = out_idx[start:start + len(oi)].cpu().numpy()
        gx = out_xyz[start:start + len(oi)].cpu().numpy()
        assert np.array_equal(gi, oi)
        assert np.abs(gx - ox).max() <= POINT_TOL * extent(ox)
