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
