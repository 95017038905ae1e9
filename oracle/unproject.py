"""Inverse projection of depth maps through pinhole cameras: the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. III-C "Feed-Forward Inference": the current submap is obtained
by inverse-projecting the predicted depths D through the projection matrices
derived from the predicted cameras g (intrinsics and extrinsics); every
keyframe pixel gives one point, in the coordinates of the submap.

Readings where the paper is silent (each also listed in the design notes):

* pixel (row v, column u) has image coordinates (u, v), integers with no
  half-pixel offset, and its camera-frame point is
  d K^-1 [u, v, 1]^T = d ((u - cx) / fx, (v - cy) / fy, 1), with d the depth
  along the optical axis;
* a camera's pose is given camera -> submap: X = R x_cam + t;
* a pixel whose depth is not finite or not > 0 has no point (NaN), so the
  registration treats it as invalid.

Registration from depth is then the registration of these pointmaps
(``register.align_pairs`` on the unprojected frames).
"""
from __future__ import annotations

import numpy as np


def camera(cam):
    """(fx, fy, cx, cy, R [3,3], t [3]) of a 16-vector camera."""
    c = np.asarray(cam, dtype=np.float64)
    return c[0], c[1], c[2], c[3], c[4:13].reshape(3, 3), c[13:16]


def unproject(depth, cams):
    """depth [n, H, W], cams [n, 16] -> points [n, H*W, 3] (float64, submap frame)."""
    d = np.asarray(depth, dtype=np.float64)
    n, H, W = d.shape
    v, u = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                       indexing="ij")
    out = np.empty((n, H * W, 3))
    for f in range(n):
        fx, fy, cx, cy, R, t = camera(cams[f])
        df = d[f]
        with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
            x_cam = np.stack([(u - cx) / fx * df, (v - cy) / fy * df, df], -1).reshape(-1, 3)
            X = x_cam @ R.T + t
        ok = (np.isfinite(df) & (df > 0)).reshape(-1)
        X[~ok] = np.nan
        out[f] = X
    return out


def project(X, cam):
    """Pixel coordinates (u, v) and depth of submap points X [N, 3] (the inverse)."""
    fx, fy, cx, cy, R, t = camera(cam)
    x = (np.asarray(X, dtype=np.float64) - t) @ R      # R^T (X - t), row-wise
    z = x[:, 2]
    return fx * x[:, 0] / z + cx, fy * x[:, 1] / z + cy, z


def unproject_backward(gX, depth, cams):
    """Gradient with respect to the depths, given dL/dX of the unprojected points.

    X = R (d r) + t with the pixel's ray r = ((u - cx)/fx, (v - cy)/fy, 1), so
    dX/dd = R r and dL/dd = (R r) . dL/dX.  A pixel without a point (its depth
    not finite or not > 0) gets 0.  gX [n, H*W, 3], depth [n, H, W] ->
    [n, H, W] (float64).  This is the chain rule that carries the registration's
    adjoint (``oracle.adjoint``) from points back to depth maps.
    """
    d = np.asarray(depth, dtype=np.float64)
    n, H, W = d.shape
    g = np.asarray(gX, dtype=np.float64).reshape(n, H * W, 3)
    v, u = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                       indexing="ij")
    out = np.zeros((n, H, W))
    for f in range(n):
        fx, fy, cx, cy, R, t = camera(cams[f])
        r = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1).reshape(-1, 3)
        gd = ((r @ R.T) * g[f]).sum(1)
        ok = (np.isfinite(d[f]) & (d[f] > 0)).reshape(-1)
        out[f] = np.where(ok, gd, 0.0).reshape(H, W)
    return out
