"""Pins of the depth unprojection oracle (Sec. III-C, submaps from depth and
cameras): projection inverts it, a fronto-parallel plane maps to the pinhole
grid, invalid depths give no point, and the camera pose is a rigid motion."""
import numpy as np

from oracle import unproject as up


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _cam(rng, H, W):
    fx, fy = rng.uniform(100, 400, 2)
    cx, cy = W / 2 + rng.uniform(-3, 3), H / 2 + rng.uniform(-3, 3)
    return np.concatenate([[fx, fy, cx, cy], _rot(rng).ravel(), rng.normal(size=3)])


def test_projection_inverts_unprojection():
    rng = np.random.default_rng(0)
    H, W = 7, 11
    cams = np.stack([_cam(rng, H, W) for _ in range(3)])
    depth = rng.uniform(0.3, 20.0, (3, H, W))
    X = up.unproject(depth, cams)
    v, u = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for f in range(3):
        pu, pv, z = up.project(X[f], cams[f])
        np.testing.assert_allclose(pu, u.ravel(), atol=1e-9)
        np.testing.assert_allclose(pv, v.ravel(), atol=1e-9)
        np.testing.assert_allclose(z, depth[f].ravel(), rtol=1e-12)


def test_fronto_parallel_plane_is_the_pinhole_grid():
    H, W, Z, fx, fy, cx, cy = 5, 8, 3.0, 200.0, 250.0, 3.0, 2.0
    cam = np.concatenate([[fx, fy, cx, cy], np.eye(3).ravel(), np.zeros(3)])
    X = up.unproject(np.full((1, H, W), Z), cam[None])[0].reshape(H, W, 3)
    assert np.all(X[..., 2] == Z)
    np.testing.assert_allclose(np.diff(X[..., 0], axis=1), Z / fx, rtol=1e-14)
    np.testing.assert_allclose(np.diff(X[..., 1], axis=0), Z / fy, rtol=1e-14)
    np.testing.assert_array_equal(X[int(cy), int(cx)], [0.0, 0.0, Z])


def test_invalid_depths_have_no_point():
    rng = np.random.default_rng(1)
    H, W = 3, 4
    cam = _cam(rng, H, W)[None]
    d = rng.uniform(1, 2, (1, H, W))
    bad = [(0, 0, 0.0), (0, 1, -1.0), (1, 2, np.nan), (2, 3, np.inf)]
    for r, c, val in bad:
        d[0, r, c] = val
    X = up.unproject(d, cam)[0].reshape(H, W, 3)
    for r, c, _ in bad:
        assert np.all(np.isnan(X[r, c]))
    good = np.ones((H, W), bool)
    for r, c, _ in bad:
        good[r, c] = False
    assert np.all(np.isfinite(X[good]))


def test_camera_pose_is_a_rigid_motion():
    rng = np.random.default_rng(2)
    H, W = 6, 9
    cam = _cam(rng, H, W)
    ident = cam.copy()
    ident[4:13] = np.eye(3).ravel()
    ident[13:16] = 0.0
    d = rng.uniform(0.5, 5.0, (1, H, W))
    A = up.unproject(d, cam[None])[0]
    B = up.unproject(d, ident[None])[0]
    R, t = cam[4:13].reshape(3, 3), cam[13:16]
    np.testing.assert_allclose(A, B @ R.T + t, atol=1e-12)
    DA = np.linalg.norm(A[:, None] - A[None], axis=-1)
    DB = np.linalg.norm(B[:, None] - B[None], axis=-1)
    np.testing.assert_allclose(DA, DB, atol=1e-12)
