"""GPU parity of ec3r_align_submaps_depth (Sec. III-C: submaps as the inverse
projection of predicted depths through predicted cameras, registered by the
weighted Umeyama solve in Huber IRLS) against the FP64 oracle: unprojection
(oracle.unproject) followed by the pointmap registration oracle.

Tolerances as for the pointmap path: rotation <= 1e-5 rad, scale <= 1e-6
relative, translation <= 1e-6 x scene extent; statuses equal; cost <= 1e-5
relative."""
import numpy as np
import pytest
import torch

from oracle import register as reg
from oracle import unproject as up
from paper_2510_02080_b300 import ec3r, synth
from parity import assert_sim3_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def oracle_pairset(dps, frames=None):
    """The oracle's pointmaps of (some) frames of a depth pair set."""
    n = dps.depth.shape[0]
    frames = range(n) if frames is None else frames
    xyz = np.full((n, dps.H * dps.W, 3), np.nan)
    idx = np.asarray(sorted(set(frames)))
    xyz[idx] = up.unproject(dps.depth[idx].numpy(), dps.cams[idx].numpy())
    return synth.PairSet(torch.from_numpy(xyz), dps.conf.view(n, -1), dps.link_off, dps.src,
                         dps.tgt, dps.H, dps.W)


def run(ctx, dps, pcm=None, **kw):
    S, st, cost = ctx.align_submaps_depth(dps.depth.cuda(), dps.conf.cuda(), dps.cams.cuda(),
                                          dps.link_off.cuda(), dps.src.cuda(), dps.tgt.cuda(),
                                          None if pcm is None else pcm.cuda(), **kw)
    torch.cuda.synchronize()
    return S.cpu().numpy(), st.cpu().numpy(), None if cost is None else cost.cpu().numpy()


def check(ps_or, S, st, cost, pairs=None, **kw):
    ref = reg.align_pairs(ps_or, pairs=pairs, **kw)
    for r in ref:
        k = r["pair"]
        assert int(st[k]) == r["status"], (k, int(st[k]), r["status"])
        if r["status"] == 0:
            assert_sim3_close(S[k], r["S"], r["extent"], f"pair {k}")
            Rg = S[k][1:10].reshape(3, 3)
            assert np.abs(Rg.T @ Rg - np.eye(3)).max() < 1e-14
            if cost is not None:
                assert abs(cost[k] - r["cost"]) <= 1e-5 * r["cost"] + 1e-12, (k, cost[k],
                                                                             r["cost"])
        else:
            assert S[k][0] == 1.0 and np.abs(S[k][10:]).max() == 0.0
    return ref


@pytest.mark.parametrize("overlap", [1, 2])
def test_depth_chain_matches_oracle(ctx, overlap):
    # 100 x 180 = 18000 pixels: two 8192-pixel tiles and a ragged tail per link;
    # overlap 2: two links per pair through different cameras
    ch = synth.make_depth_chain(synth.SEED_BASE + 40 + overlap, M=5, F=3, H=100, W=180,
                                overlap=overlap)
    dps = ch.pairs()
    S, st, cost = run(ctx, dps, want_cost=True)
    ref = check(oracle_pairset(dps), S, st, cost)
    assert all(r["status"] == 0 for r in ref)


def test_depth_matches_pointmap_path_and_truth(ctx):
    """The same pairs as pointmaps (the oracle's unprojection, stored as float32)
    through ec3r_align_submaps agree with the depth path, and both recover the
    ground truth up to the noise."""
    ch = synth.make_depth_chain(synth.SEED_BASE + 43, M=4, F=3, H=60, W=90, overlap=1,
                                sigma=0.002, outlier_frac=0.0)
    dps = ch.pairs()
    S, st, _ = run(ctx, dps)
    ps = oracle_pairset(dps)
    xyz = ps.xyz.to(torch.float32).cuda()
    S2, st2, _ = ctx.align_submaps(xyz, ps.conf.cuda(), ps.link_off.cuda(), ps.src.cuda(),
                                   ps.tgt.cuda())
    S2 = S2.cpu().numpy()
    assert (st == 0).all() and (st2.cpu().numpy() == 0).all()
    gt = synth.chain_pair_truth(ch)
    for k in range(dps.n_pairs):
        assert abs(S[k][0] / S2[k][0] - 1) < 1e-5
        assert np.abs(S[k][1:10] - S2[k][1:10]).max() < 1e-5
        assert abs(S[k][0] / float(gt.s[k]) - 1) < 1e-2


def test_invalid_depths_thresholds_and_degenerate_pairs(ctx):
    ch = synth.make_depth_chain(synth.SEED_BASE + 44, M=4, F=2, H=40, W=64, overlap=1)
    dps = ch.pairs()
    d = dps.depth.clone()
    rng = np.random.default_rng(3)
    flat = d.view(-1)
    for val in (0.0, -2.0, float("nan"), float("inf")):   # invalid depths
        flat[torch.from_numpy(rng.choice(flat.numel(), 300, replace=False))] = val
    d[dps.src[2]] = 0.0                                    # pair 2: no valid point at all
    dps2 = synth.DepthPairSet(d, dps.conf, dps.cams, dps.link_off, dps.src, dps.tgt, dps.H,
                              dps.W)
    pcm = torch.tensor([0.0, 1.2, 0.0], dtype=torch.float32)
    S, st, cost = run(ctx, dps2, pcm=pcm, want_cost=True)
    ps = oracle_pairset(dps2)
    ps.pair_conf_min = pcm
    ref = check(ps, S, st, cost)
    assert ref[2]["status"] == reg.DEG_FEW and int(st[2]) == reg.DEG_FEW


def test_unusable_camera_drops_its_link(ctx):
    """A frame whose camera has a NaN entry (or a zero focal length) yields no
    points: its link contributes nothing and the pair uses its other link."""
    ch = synth.make_depth_chain(synth.SEED_BASE + 47, M=3, F=3, H=50, W=64, overlap=2)
    dps = ch.pairs()
    cams = dps.cams.clone()
    cams[dps.src[0], 5] = float("nan")     # pair 0, link 0
    cams[dps.tgt[3], 0] = 0.0              # pair 1, link 1: fx = 0
    dps2 = synth.DepthPairSet(dps.depth, dps.conf, cams, dps.link_off, dps.src, dps.tgt, dps.H,
                              dps.W)
    S, st, cost = run(ctx, dps2, want_cost=True)
    ref = check(oracle_pairset(dps2), S, st, cost)
    assert all(r["status"] == 0 for r in ref)


def test_bad_links_and_arguments(ctx):
    ch = synth.make_depth_chain(synth.SEED_BASE + 45, M=3, F=2, H=20, W=24, overlap=1)
    dps = ch.pairs()
    tgt = dps.tgt.clone()
    tgt[1] = 99                                            # out-of-range frame
    bad = synth.DepthPairSet(dps.depth, dps.conf, dps.cams, dps.link_off, dps.src, tgt, dps.H,
                             dps.W)
    S, st, _ = run(ctx, bad)
    assert int(st[1]) == 16 and int(st[0]) == 0            # EC3R_PAIR_BAD_INPUT
    assert ctx.sync_status() == 1                          # EC3R_ERR_INVALID_ARG (bad index)
    # offsets that are no CSR array: with [0, 2, 1, 3] pairs 0 and 2 would both
    # claim link 1 and pair 1 runs backwards; every pair of the call is marked
    d4 = synth.make_depth_chain(synth.SEED_BASE + 45, M=4, F=2, H=20, W=24, overlap=1).pairs()
    overlap = synth.DepthPairSet(d4.depth, d4.conf, d4.cams,
                                 torch.tensor([0, 2, 1, 3], dtype=torch.int32), d4.src, d4.tgt,
                                 d4.H, d4.W)
    S, st, _ = run(ctx, overlap)
    assert st.tolist() == [16, 16, 16]
    assert ctx.sync_status() == 1
    S, st, _ = run(ctx, d4)
    assert st.tolist() == [0, 0, 0] and ctx.sync_status() == 0
    with pytest.raises(ValueError):
        ctx.align_submaps_depth(dps.depth.cuda(), dps.conf.cuda(), dps.cams[:1].cuda(),
                                dps.link_off.cuda(), dps.src.cuda(), dps.tgt.cuda())
    with pytest.raises(ec3r.Ec3rError):
        ctx.align_submaps_depth(dps.depth.cuda(), dps.conf.cuda(), dps.cams.cuda(),
                                dps.link_off.cuda(), dps.src.cuda(), dps.tgt.cuda(), delta=-1.0)


@pytest.mark.timeout(900)
def test_full_size_depth_chain_sampled_pairs(ctx):
    """200 submaps of 5 x 294 x 518 depth frames (the benchmark chain as depth):
    every pair through the depth path, six sampled pairs against the oracle."""
    ch = synth.make_depth_chain(synth.SEED_BASE + 46, M=200, F=5, H=294, W=518, device="cuda")
    dps = ch.pairs()
    S, st, cost = ctx.align_submaps_depth(dps.depth, dps.conf, dps.cams, dps.link_off, dps.src,
                                          dps.tgt, want_cost=True)
    torch.cuda.synchronize()
    S, st, cost = S.cpu().numpy(), st.cpu().numpy(), cost.cpu().numpy()
    assert (st == 0).all()
    pairs = [0, 41, 99, 100, 157, 198]
    frames = [int(f) for k in pairs for f in (dps.src[k], dps.tgt[k])]
    cpu = synth.DepthPairSet(dps.depth.cpu(), dps.conf.cpu(), dps.cams.cpu(), dps.link_off.cpu(),
                             dps.src.cpu(), dps.tgt.cpu(), dps.H, dps.W)
    check(oracle_pairset(cpu, frames), S, st, cost, pairs=pairs)


def _rand_pose_rows(rng, M):
    from scipy.spatial.transform import Rotation
    s = rng.uniform(0.5, 2.0, M)
    R = Rotation.random(M, random_state=rng).as_matrix()
    t = rng.normal(size=(M, 3)) * 3
    rows = np.concatenate([s[:, None], R.reshape(M, 9), t], 1)
    return rows, [(s[m], R[m], t[m]) for m in range(M)]


def test_depth_fusion_matches_oracle(ctx):
    """ec3r_fuse_points_depth against the oracle's unprojection + fusion: flat
    indices bit-exact, points within 1e-6 x extent; invalid depths and an
    unusable camera drop their pixels; two calls stream into one buffer and a
    short buffer reports the overflow."""
    from oracle import fuse as ofuse
    ch = synth.make_depth_chain(synth.SEED_BASE + 48, M=4, F=3, H=100, W=180, overlap=1)
    dps = ch.pairs()
    d = dps.depth.clone()
    rng = np.random.default_rng(5)
    flat = d.view(-1)
    for val in (0.0, -1.0, float("nan"), float("inf")):
        flat[torch.from_numpy(rng.choice(flat.numel(), 500, replace=False))] = val
    cams = dps.cams.clone()
    cams[4, 9] = float("nan")                        # frame 4 (submap 1): no points
    rows, poses = _rand_pose_rows(rng, ch.M)
    ref_x, ref_i = ofuse.fuse_points_depth(d.numpy(), dps.conf.numpy(), cams.numpy(), poses,
                                           frames=3, threshold=1.0, index_base=7)
    K = len(ref_i)
    out_x = torch.full((K + 5, 3), -3.0, device="cuda")
    out_i = torch.full((K + 5,), -3, dtype=torch.int64, device="cuda")
    cur = torch.zeros((1,), dtype=torch.int64, device="cuda")
    d_d, c_d, k_d = d.cuda(), dps.conf.cuda(), cams.cuda()
    P = torch.tensor(rows, dtype=torch.float64, device="cuda")
    ctx.fuse_points_depth(d_d[:6], c_d[:6], k_d[:6], P[:2], out_x, out_i, cur, frames=3,
                          index_base=7)
    ctx.fuse_points_depth(d_d[6:], c_d[6:], k_d[6:], P[2:], out_x, out_i, cur, frames=3,
                          index_base=7 + 6 * dps.H * dps.W)
    assert ctx.sync_status() == 0 and int(cur) == K
    gi = out_i[:K].cpu().numpy()
    gx = out_x[:K].cpu().numpy()
    np.testing.assert_array_equal(gi, ref_i)
    ext = float(np.linalg.norm(np.ptp(ref_x, axis=0)))
    assert np.abs(gx - ref_x).max() <= 1e-6 * ext
    assert not np.any((gi >= 7 + 4 * dps.H * dps.W) & (gi < 7 + 5 * dps.H * dps.W))
    # a buffer one point short: everything but the last point, then CAPACITY
    cur.zero_()
    short_x = torch.zeros((K - 1, 3), device="cuda")
    short_i = torch.zeros((K - 1,), dtype=torch.int64, device="cuda")
    ctx.fuse_points_depth(d_d, c_d, k_d, P, short_x, short_i, cur, frames=3, index_base=7)
    assert ctx.sync_status() == 4                     # EC3R_ERR_CAPACITY
    assert int(cur) == K
    np.testing.assert_array_equal(short_i.cpu().numpy(), ref_i[:K - 1])
