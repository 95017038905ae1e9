"""Confidence-filtered fusion of submap points into the global map: the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper obtains "the global coordinates of all points in the current
submap" from the estimated transforms (Sec. III-C "Point Correction"); each
point of a submap carries a confidence (Sec. III-C "Feed-Forward Inference").
Readings:

* a point is kept when its confidence is strictly greater than the threshold
  (NaN confidences are dropped);
* kept points are emitted in ascending global flat index
  g = index_base + ((m*F + f)*H + row)*W + col (submap-major), which makes
  the compaction unique;
* the global point is T_m(x) = s_m R_m x + t_m evaluated in float64 from the
  float32 point and the float64 pose of submap m.

The compaction is written as its definition: an exclusive prefix sum of the
keep flags gives every kept point its output slot.
"""
from __future__ import annotations

import numpy as np


def fuse_points(xyz, conf, poses, threshold=1.0, index_base=0):
    """xyz [M, F*H*W, 3] (or [M,F,H,W,3]), conf [M, ...], poses = list of (s, R, t).

    Returns (out_xyz [K,3] float64, out_idx [K] int64).
    """
    xyz = np.asarray(xyz)
    conf = np.asarray(conf)
    M = xyz.shape[0]
    if M == 0:                                  # no submap: no point
        return np.empty((0, 3), dtype=np.float64), np.empty(0, dtype=np.int64)
    xyz = xyz.reshape(M, -1, 3)
    conf = conf.reshape(M, -1)
    n = conf.shape[1]
    with np.errstate(invalid="ignore"):
        keep = (conf > threshold).reshape(-1)
    slot = np.cumsum(keep, dtype=np.int64) - keep          # exclusive prefix sum
    K = int(keep.sum())
    out_idx = np.empty(K, dtype=np.int64)
    out_xyz = np.empty((K, 3), dtype=np.float64)
    g = np.arange(M * n, dtype=np.int64)
    out_idx[slot[keep]] = g[keep] + index_base
    for m in range(M):
        s, R, t = poses[m]
        km = keep[m * n:(m + 1) * n]
        X = xyz[m][km].astype(np.float64)
        out_xyz[slot[m * n:(m + 1) * n][km]] = s * (X @ np.asarray(R).T) + np.asarray(t)
    return out_xyz, out_idx


def correct_points(points, refs, xyz, conf, poses, threshold=1.0):
    """Point correction (Sec. III-C "Point Correction"): a sparse-map point
    that corresponds to a submap pixel takes that pixel's global coordinates.

    Readings: the correspondence is given as the flat submap point g of
    ``fuse_points`` (-1: none); the replacement happens only when the submap
    point is valid (confidence strictly above the threshold, finite
    coordinates), the other points keep their coordinates; the global point is
    T_m(x) in float64 as in ``fuse_points``.

    Returns (points [n, 3] float64, number corrected).
    """
    out = np.asarray(points, dtype=np.float64).copy()
    xyz = np.asarray(xyz)
    conf = np.asarray(conf)
    M = xyz.shape[0]
    n = conf.size // M if M else 0
    xyz = xyz.reshape(M, n, 3)
    conf = conf.reshape(M, n)
    count = 0
    for i, g in enumerate(np.asarray(refs, dtype=np.int64)):
        if g < 0 or g >= M * n:      # none (-1), or no such submap point: unchanged
            continue
        m, k = divmod(int(g), n)
        x = xyz[m, k].astype(np.float64)
        if not (conf[m, k] > threshold) or not np.all(np.isfinite(x)):
            continue
        s, R, t = poses[m]
        out[i] = s * (np.asarray(R) @ x) + np.asarray(t)
        count += 1
    return out, count


def fuse_points_depth(depth, conf, cams, poses, frames, threshold=1.0, index_base=0):
    """Fusion of depth frames (Sec. III-C: submaps are unprojected depths):
    ``unproject`` gives every pixel's submap point (none where the depth or the
    camera is invalid); a pixel is kept when it has a point and its confidence
    is strictly above the threshold; kept points go out in ascending flat
    index as in ``fuse_points``.  depth / conf [M*frames, H, W], cams
    [M*frames, 16], poses: list of M (s, R, t).

    Returns (out_xyz [K, 3] float64, out_idx [K] int64).
    """
    from . import unproject as up
    d = np.asarray(depth)
    nfr = d.shape[0]
    M = nfr // frames
    if M == 0:                                                # no submap: no point
        return np.empty((0, 3)), np.empty(0, dtype=np.int64)
    X = up.unproject(d, cams).reshape(M, -1, 3)              # [M, frames*H*W, 3]
    c = np.asarray(conf, dtype=np.float64).reshape(M, -1)
    with np.errstate(invalid="ignore"):
        keep = (c > threshold) & np.all(np.isfinite(X), axis=-1)
    flat_keep = keep.reshape(-1)
    n = c.shape[1]
    g = np.nonzero(flat_keep)[0].astype(np.int64)
    out = np.empty((len(g), 3))
    for m in range(M):
        sel = (g >= m * n) & (g < (m + 1) * n)
        s, R, t = poses[m]
        out[sel] = s * (X[m][g[sel] - m * n] @ np.asarray(R).T) + np.asarray(t)
    return out, g + index_base
