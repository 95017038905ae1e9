"""Pins of the fusion oracle: compaction against numpy.flatnonzero and every
kept point against the homogeneous 4x4 transform of its source point."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import fuse


def test_fuse_matches_flatnonzero_and_homogeneous_transform():
    rng = np.random.default_rng(0)
    M, n = 4, 1037
    xyz = rng.normal(size=(M, n, 3)).astype(np.float32) * 5
    conf = rng.lognormal(0, 0.5, size=(M, n)).astype(np.float32)
    conf[0, :5] = 1.0                      # ties: strict '>' drops them
    conf[1, 7] = np.nan
    conf[2] = 0.5                          # a submap with nothing kept
    poses = [(float(rng.uniform(0.5, 2)), Rotation.random(random_state=rng).as_matrix(),
              rng.normal(size=3)) for _ in range(M)]
    out_xyz, out_idx = fuse.fuse_points(xyz, conf, poses, 1.0, index_base=1000)
    ref_idx = np.flatnonzero(conf.reshape(-1) > 1.0) + 1000
    assert np.array_equal(out_idx, ref_idx)
    for k, g in enumerate(out_idx - 1000):
        m, i = divmod(int(g), n)
        s, R, t = poses[m]
        H = np.eye(4)
        H[:3, :3] = s * R
        H[:3, 3] = t
        ref = (H @ np.append(xyz[m, i].astype(np.float64), 1.0))[:3]
        assert np.abs(out_xyz[k] - ref).max() < 1e-12


def test_fuse_empty():
    xyz = np.zeros((2, 3, 3), np.float32)
    conf = np.zeros((2, 3), np.float32)
    out_xyz, out_idx = fuse.fuse_points(xyz, conf, [(1.0, np.eye(3), np.zeros(3))] * 2)
    assert out_xyz.shape == (0, 3) and out_idx.shape == (0,)
    out_xyz, out_idx = fuse.fuse_points(np.zeros((0, 3, 3), np.float32),
                                        np.zeros((0, 3), np.float32), [], index_base=9)
    assert out_xyz.shape == (0, 3) and out_idx.shape == (0,)


def test_point_correction_closed_forms():
    """Point correction (Sec. III-C): identity pose copies the submap point;
    translation / scale poses add t / multiply by s; invalid or missing
    correspondences leave the sparse point unchanged."""
    rng = np.random.default_rng(7)
    M, n = 3, 50
    xyz = rng.normal(size=(M, n, 3)).astype(np.float32)
    conf = rng.uniform(0.5, 2.0, (M, n)).astype(np.float32)
    xyz[1, 4, 2] = np.nan
    conf[2, 9] = np.nan
    t = np.array([1.0, -2.0, 0.5])
    poses = [(1.0, np.eye(3), np.zeros(3)), (1.0, np.eye(3), t), (2.5, np.eye(3), np.zeros(3))]
    refs = np.array([-1, 3, n + 7, n + 4, 2 * n + 9, 2 * n + 11, 0])
    pts = rng.normal(size=(len(refs), 3))
    out, cnt = fuse.correct_points(pts, refs, xyz, conf, poses, threshold=1.0)
    for i, g in enumerate(refs):
        m, k = divmod(int(g), n) if g >= 0 else (None, None)
        valid = g >= 0 and conf[m, k] > 1.0 and np.all(np.isfinite(xyz[m, k]))
        if not valid:
            np.testing.assert_array_equal(out[i], pts[i])
        elif m == 0:
            np.testing.assert_array_equal(out[i], xyz[0, k].astype(np.float64))
        elif m == 1:
            np.testing.assert_allclose(out[i], xyz[1, k] + t, rtol=0, atol=1e-15)
        else:
            np.testing.assert_allclose(out[i], 2.5 * xyz[2, k].astype(np.float64), rtol=1e-15)
    assert cnt == sum(1 for g in refs if g >= 0 and conf.reshape(-1)[g] > 1.0 and
                      np.all(np.isfinite(xyz.reshape(-1, 3)[g])))


def test_point_correction_out_of_range_and_no_submaps():
    """A reference below -1 or past the last submap point leaves its point
    unchanged and is not counted; with no submap every reference is such."""
    rng = np.random.default_rng(8)
    M, n = 2, 10
    xyz = rng.normal(size=(M, n, 3)).astype(np.float32)
    conf = np.full((M, n), 2.0, np.float32)
    poses = [(1.0, np.eye(3), np.zeros(3))] * M
    refs = np.array([-5, M * n, M * n + 3, 7])
    pts = rng.normal(size=(4, 3))
    out, cnt = fuse.correct_points(pts, refs, xyz, conf, poses)
    np.testing.assert_array_equal(out[:3], pts[:3])
    np.testing.assert_array_equal(out[3], xyz[0, 7].astype(np.float64))
    assert cnt == 1
    out, cnt = fuse.correct_points(pts, refs, np.zeros((0, n, 3), np.float32),
                                   np.zeros((0, n), np.float32), [])
    np.testing.assert_array_equal(out, pts)
    assert cnt == 0
    ox, oi = fuse.fuse_points_depth(np.zeros((0, 2, 3)), np.zeros((0, 2, 3)), np.zeros((0, 16)),
                                    [], frames=1)
    assert ox.shape == (0, 3) and oi.shape == (0,)


def test_depth_fusion_closed_forms():
    """Fusion of depth frames: with identity camera and pose, a constant-depth
    plane fuses to the pinhole grid; a pixel without a point (depth <= 0, NaN,
    or a frame whose camera has a zero focal length) is dropped even when its
    confidence passes; a pose maps the kept points."""
    H, W, Z = 4, 6, 2.0
    cam = np.concatenate([[100.0, 80.0, 2.0, 1.0], np.eye(3).ravel(), np.zeros(3)])
    cams = np.stack([cam, cam.copy()])
    cams[1, 0] = 0.0                                     # frame 1: fx = 0, no points
    depth = np.full((2, H, W), Z)
    depth[0, 0, 0] = 0.0
    depth[0, 1, 2] = np.nan
    conf = np.full((2, H, W), 2.0)
    conf[0, 3, 5] = 0.5                                  # below the threshold
    s, t = 1.5, np.array([0.0, 1.0, -2.0])
    out, idx = fuse.fuse_points_depth(depth, conf, cams, [(s, np.eye(3), t)], frames=2,
                                      threshold=1.0, index_base=10)
    expect = [r * W + c for r in range(H) for c in range(W)
              if (r, c) not in ((0, 0), (1, 2), (3, 5))]
    np.testing.assert_array_equal(idx, np.asarray(expect) + 10)
    for k, g in enumerate(expect):
        r, c = divmod(g, W)
        x = np.array([(c - 2.0) / 100.0 * Z, (r - 1.0) / 80.0 * Z, Z])
        np.testing.assert_allclose(out[k], s * x + t, rtol=0, atol=1e-14)
