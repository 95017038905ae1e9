"""GPU parity of ec3r_correct_points (Sec. III-C "Point Correction": sparse-map
points that correspond to submap pixels take their global coordinates)
against the FP64 oracle: corrected points within 1e-6 x scene extent, the
untouched ones bit-identical, the count exact; and every corrected point
bit-identical to the fused point of the same pixel."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import fuse as ofuse
from paper_2510_02080_b300 import ec3r

pytestmark = pytest.mark.gpu
POINT_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def scene(seed, M=4, n=3000):
    rng = np.random.default_rng(seed)
    xyz = (rng.normal(size=(M, n, 3)) * 4).astype(np.float32)
    conf = np.exp(0.5 * rng.normal(size=(M, n))).astype(np.float32)
    xyz[0, 5, 1] = np.nan
    conf[1, 17] = np.nan
    s = rng.uniform(0.5, 2.0, M)
    R = Rotation.random(M, random_state=rng).as_matrix()
    t = rng.normal(size=(M, 3)) * 3
    rows = np.concatenate([s[:, None], R.reshape(M, 9), t], 1)
    return rng, xyz, conf, rows, [(s[m], R[m], t[m]) for m in range(M)]


def test_correction_matches_oracle_and_fusion(ctx):
    rng, xyz, conf, rows, poses = scene(0)
    M, n = conf.shape
    n_sp = 20_000                                     # 79 CTAs of 256, ragged tail
    refs = rng.integers(-1, M * n, n_sp)
    refs[:4] = [5, n + 17, -1, M * n - 1]             # NaN point, NaN conf, none, last
    pts = rng.normal(size=(n_sp, 3)).astype(np.float32)
    d_pts = torch.tensor(pts, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    xyz_d = torch.tensor(xyz, device="cuda")
    conf_d = torch.tensor(conf, device="cuda")
    poses_d = torch.tensor(rows, dtype=torch.float64, device="cuda")
    ctx.correct_points(d_pts, torch.tensor(refs, device="cuda"), xyz_d, conf_d, poses_d,
                       threshold=1.0, n_corrected=cnt)
    assert ctx.sync_status() == 0
    got = d_pts.cpu().numpy()
    ref, ref_cnt = ofuse.correct_points(pts, refs, xyz, conf, poses, threshold=1.0)
    assert int(cnt) == ref_cnt
    changed = np.any(ref != pts.astype(np.float64), axis=1)
    ext = float(np.linalg.norm(np.ptp(ref[changed], axis=0)))
    assert np.array_equal(got[~changed], pts[~changed])
    assert np.abs(got[changed] - ref[changed]).max() <= POINT_TOL * ext
    # the fused point of the same pixel is the same float32 value
    kept = int((conf > 1.0).sum())
    ox = torch.empty((kept, 3), device="cuda")
    oi = torch.empty((kept,), dtype=torch.int64, device="cuda")
    cur = torch.zeros((1,), dtype=torch.int64, device="cuda")
    ctx.fuse_points(xyz_d, conf_d, poses_d, ox, oi, cur, threshold=1.0)
    fused = dict(zip(oi.cpu().numpy().tolist(), ox.cpu().numpy()))
    for i in np.nonzero(changed)[0][:2000]:
        assert np.array_equal(got[i], fused[int(refs[i])])


def test_bad_reference_is_reported(ctx):
    rng, xyz, conf, rows, poses = scene(1, M=2, n=100)
    refs = torch.tensor([3, -5, 150, 400], device="cuda")   # -5 and 400 are invalid
    pts = torch.zeros((4, 3), device="cuda")
    ctx.correct_points(pts, refs, torch.tensor(xyz, device="cuda"),
                       torch.tensor(conf, device="cuda"),
                       torch.tensor(rows, dtype=torch.float64, device="cuda"))
    assert ctx.sync_status() == 1                          # EC3R_ERR_INVALID_ARG
    got = pts.cpu().numpy()
    assert np.all(got[1] == 0) and np.all(got[3] == 0)
    assert ctx.sync_status() == 0
