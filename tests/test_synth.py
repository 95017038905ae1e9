"""The seeded generator: deterministic, shaped as stated, and its ground truth
is what the oracle recovers from noise-free inputs."""
import numpy as np
import torch

from oracle import register as reg
from oracle import sim3
from paper_2510_02080_b300 import synth


def test_pair_deterministic_and_recoverable():
    a = synth.make_pair(1, H=24, W=40, sigma=0.0, outlier_frac=0.0)
    b = synth.make_pair(1, H=24, W=40, sigma=0.0, outlier_frac=0.0)
    assert torch.equal(a.xyz, b.xyz) and torch.equal(a.conf, b.conf)
    assert a.xyz.shape == (2, 24 * 40, 3) and a.xyz.dtype == torch.float32
    assert torch.isfinite(a.xyz).all() and (a.conf > 0).all()
    res = reg.align_pairs(a, delta=0.02, iters=3)[0]
    s, R, t = [v[0] for v in a.S_gt.numpy()]
    assert res["status"] == 0
    assert abs(res["S"][0] / s - 1) < 1e-5 and sim3.rotation_angle(res["S"][1], R) < 1e-5


def test_chain_pairs_share_a_keyframe():
    ch = synth.make_chain(2, M=4, F=5, H=16, W=20, sigma=0.0, outlier_frac=0.0)
    ps = ch.pairs()
    assert ps.n_pairs == 3 and ch.xyz.shape == (4, 5, 320, 3)
    truth = synth.chain_pair_truth(ch)
    for m in range(3):
        p = ps.xyz[int(ps.src[m])].double().numpy()
        q = ps.xyz[int(ps.tgt[m])].double().numpy()
        T = (float(truth.s[m]), truth.R[m].numpy(), truth.t[m].numpy())
        assert np.abs(sim3.act(T, p) - q).max() < 1e-4 * (1 + np.abs(q).max())


def test_loop_batch_valid_counts_follow_thresholds():
    ps = synth.make_loop_batch(3, n_pairs=6, H=32, W=48, min_valid=300, max_valid=4000)
    lo = ps.link_off.tolist()
    for k in range(6):
        f = lo[k + 1] - lo[k]
        assert 1 <= f <= 5
        cp = ps.conf[ps.src[lo[k]:lo[k + 1]].long()]
        cq = ps.conf[ps.tgt[lo[k]:lo[k + 1]].long()]
        thr = float(ps.pair_conf_min[k])
        n_valid = int(((cp > thr) & (cq > thr)).sum())
        expect = ps.meta["expected_valid"][k]
        assert abs(n_valid - expect) < 6 * np.sqrt(expect) + 20


def test_pose_graph_measurements_noise_free_are_consistent():
    g = synth.make_pose_graph(4, 12, 3, rot_noise=0, trans_noise=0, scale_noise=0)
    T = [(float(g.T_gt.s[v]), g.T_gt.R[v].numpy(), g.T_gt.t[v].numpy()) for v in range(12)]
    for k in range(len(g.ei)):
        i, j = int(g.ei[k]), int(g.ej[k])
        M = (float(g.T_meas.s[k]), g.T_meas.R[k].numpy(), g.T_meas.t[k].numpy())
        C = sim3.compose(T[i], M)
        assert abs(C[0] / T[j][0] - 1) < 1e-12 and np.abs(C[1] - T[j][1]).max() < 1e-12


def test_chain_follows_the_stated_recipe():
    """Confidences log-normal(0, 0.5); every frame's points replaced by uniform
    box points with probability 0.1, so a correspondence (two frames) is an
    outlier with probability 1 - 0.9^2 = 0.19 under the true transform; inlier
    residuals are the N(0, sigma^2) noise of both points (the source's scaled by
    s); submap scales in [0.5, 2]."""
    sigma = 0.01
    ch = synth.make_chain(5, M=4, F=5, H=40, W=60, sigma=sigma, outlier_frac=0.1)
    lc = torch.log(ch.conf.double()).reshape(-1)
    assert abs(float(lc.mean())) < 0.02 and abs(float(lc.std()) - 0.5) < 0.02
    lam = 1.0 / ch.T_gt.s.double()
    assert float(lam.min()) >= 0.5 and float(lam.max()) <= 2.0
    ps = ch.pairs()
    truth = synth.chain_pair_truth(ch)
    out, inl = [], []
    for m in range(ps.n_pairs):
        p = ps.xyz[int(ps.src[m])].double().numpy()
        q = ps.xyz[int(ps.tgt[m])].double().numpy()
        s = float(truth.s[m])
        r = sim3.act((s, truth.R[m].numpy(), truth.t[m].numpy()), p) - q
        d = np.linalg.norm(r, axis=1)
        far = d > 20 * sigma * (1 + s)
        out.append(far.mean())
        inl.append(r[~far] / (sigma * np.sqrt(1 + s * s)))    # unit normal per coordinate
    assert abs(float(np.mean(out)) - 0.19) < 0.02
    z = np.concatenate(inl).reshape(-1)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.03


def test_depth_chain_follows_the_stated_recipe():
    """Depth frames: pinhole intrinsics fx = fy, cx = W/2 - 1/2, cy = H/2 - 1/2
    and an orthonormal camera -> submap rotation; the shared keyframe,
    unprojected in both submaps, agrees under the true transform except where a
    depth was replaced by an outlier (probability 0.1 per frame, so about 0.19
    of the correspondences)."""
    from oracle import unproject as unp
    H, W, sigma = 30, 48, 0.01
    ch = synth.make_depth_chain(6, M=4, F=5, H=H, W=W, sigma=sigma, outlier_frac=0.1)
    cams = ch.cams.double().reshape(-1, 16).numpy()
    assert np.all(cams[:, 0] == cams[:, 1]) and np.all(cams[:, 0] > 0)
    assert np.all(cams[:, 2] == W / 2 - 0.5) and np.all(cams[:, 3] == H / 2 - 0.5)
    R = cams[:, 4:13].reshape(-1, 3, 3)
    assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-6
    dps = ch.pairs()
    truth = synth.chain_pair_truth(ch)
    far = []
    for m in range(dps.n_pairs):
        a, b = int(dps.src[m]), int(dps.tgt[m])
        p = unp.unproject(dps.depth[a:a + 1].numpy(), dps.cams[a:a + 1].numpy())[0]
        q = unp.unproject(dps.depth[b:b + 1].numpy(), dps.cams[b:b + 1].numpy())[0]
        s = float(truth.s[m])
        d = np.linalg.norm(sim3.act((s, truth.R[m].numpy(), truth.t[m].numpy()), p) - q, axis=1)
        far.append(np.mean(d > 0.2 * (1 + s)))
    assert abs(float(np.mean(far)) - 0.19) < 0.03


def test_keyframe_embeddings_follow_the_stated_kernel():
    """Random Fourier features average to the Gaussian kernel and the noise
    adds noise^2 to each squared norm, so keyframes j apart on the route
    (distance 0.1 j) have mean cosine exp(-(0.1 j)^2 / (2 x 0.35^2)) /
    (1 + 0.15^2); the second lap passes the first lap's places again."""
    n = 2048
    E = synth.make_keyframe_embeddings(9, n=n, d=1024).double()
    U = E / E.norm(dim=1, keepdim=True)
    for j in (1, 3, 6, 12):
        got = float((U[:-j] * U[j:]).sum(1).mean())
        want = np.exp(-(0.1 * j) ** 2 / (2 * 0.35 ** 2)) / (1 + 0.15 ** 2)
        assert abs(got - want) < 0.02, (j, got, want)
    same_place = (U[: n // 2] * U[n // 2:]).sum(1)           # lap 1 vs lap 2
    assert float(same_place.mean()) > 0.75
