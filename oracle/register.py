"""Weighted Sim(3) registration of submap pairs: the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. III-C "Sim3 Point Cloud Registration" of the paper:

* the current submap holds points P = {p_i} from old keyframes; the same
  keyframes reconstructed in another submap give the counterparts Q = {q_i},
  so a correspondence is the same pixel of the same shared keyframe in the
  two submaps (no nearest-neighbour search);
* the confidences are "normalized into weights" w_i;
* S = {s, R, t} minimises sum_i w_i ||s R p_i + t - q_i||^2 (Eq. (sim3)),
  solved by the weighted extension of Umeyama's closed form.

Readings where the paper is silent (each also listed in the design notes):

* weight of a correspondence = c_p * c_q (``rule="product"``) or c_p
  (``rule="src"``), then divided by its sum ("normalized"); the solution is
  invariant to that division;
* a correspondence is valid when p, q, c_p, c_q are finite and
  c_p > conf_min and c_q > conf_min (strict);
* robustness: Huber IRLS with threshold delta on the Euclidean residual
  r_i = ||s R p_i + t - q_i||; weight h_i = 1 if r_i <= delta else delta/r_i;
  the first solve uses h = 1; ``iters`` solves in total, the result is the
  last one;
* degeneracy: fewer than 3 valid points, total weight <= 0 or non-finite,
  source variance <= 0, or second singular value of the cross-covariance
  <= 1e-4 times the first (far above FP32 rounding of the moments, far
  below any real scene), or a non-finite result: the pair is flagged and
  reported as the identity.
"""
from __future__ import annotations

import numpy as np

from . import sim3

DEG_FEW = 1
DEG_WEIGHT = 2
DEG_RANK = 4
DEG_NONFINITE = 8
RANK_REL_TOL = 1e-4


def pair_correspondences(xyz, conf, link_off, src, tgt, k, conf_min=0.0, rule="product",
                         mask=None):
    """Correspondences of pair ``k`` (all of its shared frames, concatenated).

    Returns P, Q [N,3] float64, c_p, c_q [N] float64 and a bool ``valid`` [N]
    over every pixel of every shared frame, in link order.
    """
    xyz = np.asarray(xyz)
    conf = np.asarray(conf)
    a, b = int(link_off[k]), int(link_off[k + 1])
    P = np.concatenate([xyz[int(src[l])] for l in range(a, b)]).astype(np.float64) if b > a \
        else np.zeros((0, 3))
    Q = np.concatenate([xyz[int(tgt[l])] for l in range(a, b)]).astype(np.float64) if b > a \
        else np.zeros((0, 3))
    cp = np.concatenate([conf[int(src[l])] for l in range(a, b)]).astype(np.float64) if b > a \
        else np.zeros(0)
    cq = np.concatenate([conf[int(tgt[l])] for l in range(a, b)]).astype(np.float64) if b > a \
        else np.zeros(0)
    with np.errstate(invalid="ignore"):
        valid = (np.isfinite(P).all(1) & np.isfinite(Q).all(1) & np.isfinite(cp) & np.isfinite(cq)
                 & (cp > conf_min) & (cq > conf_min))
    if mask is not None:
        valid &= np.concatenate([np.asarray(mask[int(src[l])]) for l in range(a, b)]).astype(bool)
    return P, Q, cp, cq, valid


def base_weights(cp, cq, rule="product"):
    if rule == "product":
        return cp * cq
    if rule == "src":
        return cp.copy()
    raise ValueError(rule)


def weighted_umeyama(P, Q, w):
    """Closed-form minimiser of sum w_i ||s R p_i + t - q_i||^2.

    Umeyama (1991) with weights: centroids and covariances are weighted means.
    Returns ((s, R, t), status).
    """
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    if P.shape[0] < 3:
        return sim3.identity(), DEG_FEW
    W = w.sum()
    if not np.isfinite(W) or W <= 0:
        return sim3.identity(), DEG_WEIGHT
    mu_p = (w[:, None] * P).sum(0) / W
    mu_q = (w[:, None] * Q).sum(0) / W
    Pc = P - mu_p
    Qc = Q - mu_q
    Sigma = (Qc * w[:, None]).T @ Pc / W          # (1/W) sum w (q-mu_q)(p-mu_p)^T
    var_p = float((w * (Pc * Pc).sum(1)).sum() / W)
    if not np.isfinite(var_p) or not np.all(np.isfinite(Sigma)):
        return sim3.identity(), DEG_NONFINITE
    U, D, Vt = np.linalg.svd(Sigma)
    if var_p <= 0 or D[0] <= 0 or D[1] <= RANK_REL_TOL * D[0]:
        return sim3.identity(), DEG_RANK
    E = np.eye(3)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        E[2, 2] = -1.0
    R = U @ E @ Vt
    s = float(np.trace(np.diag(D) @ E) / var_p)
    t = mu_q - s * (R @ mu_p)
    if not (np.isfinite(s) and np.all(np.isfinite(R)) and np.all(np.isfinite(t))):
        return sim3.identity(), DEG_NONFINITE
    return (s, R, t), 0


def huber_weights(r, delta):
    return np.where(r <= delta, 1.0, delta / np.where(r > 0, r, 1.0))


def residuals(T, P, Q):
    return np.linalg.norm(sim3.act(T, P) - Q, axis=1)


def irls(P, Q, w, delta, iters):
    """Huber-IRLS around weighted Umeyama.

    Returns dict(S=(s,R,t), status, cost, history=[S_1..S_K]).  ``cost`` is
    sum_i omega_i r_i(S_K)^2 / sum_i omega_i with the last solve's weights
    omega_i = w_i h_i.
    """
    w = np.asarray(w, dtype=np.float64)
    Wsum = w.sum()
    w = w / Wsum if (np.isfinite(Wsum) and Wsum > 0) else w   # "normalized into weights"
    S = None
    hist = []
    omega = w
    for k in range(1, iters + 1):
        if k == 1:
            h = np.ones_like(w)
        else:
            h = huber_weights(residuals(S, P, Q), delta)
        omega = w * h
        S, status = weighted_umeyama(P, Q, omega)
        if status:
            return dict(S=sim3.identity(), status=status, cost=0.0, history=hist, iters_done=k)
        hist.append(S)
    r = residuals(S, P, Q)
    cost = float((omega * r * r).sum() / omega.sum()) if iters > 0 else 0.0
    return dict(S=S, status=0, cost=cost, history=hist, iters_done=iters)


def align_pairs(ps, delta=0.02, iters=10, conf_min=0.0, rule="product", pairs=None):
    """Register every pair (or the listed ones) of a ``synth.PairSet``-like set."""
    xyz = ps.xyz.cpu().numpy() if hasattr(ps.xyz, "cpu") else np.asarray(ps.xyz)
    conf = ps.conf.cpu().numpy() if hasattr(ps.conf, "cpu") else np.asarray(ps.conf)
    lo = np.asarray(ps.link_off.cpu() if hasattr(ps.link_off, "cpu") else ps.link_off)
    src = np.asarray(ps.src.cpu() if hasattr(ps.src, "cpu") else ps.src)
    tgt = np.asarray(ps.tgt.cpu() if hasattr(ps.tgt, "cpu") else ps.tgt)
    pcm = None
    if getattr(ps, "pair_conf_min", None) is not None:
        pcm = np.asarray(ps.pair_conf_min.cpu())
    out = []
    for k in (range(len(lo) - 1) if pairs is None else pairs):
        # thresholds are float32, like the confidences they are compared with
        cmin = float(np.float32(pcm[k] if pcm is not None else conf_min))
        P, Q, cp, cq, valid = pair_correspondences(xyz, conf, lo, src, tgt, k, cmin, rule)
        w = base_weights(cp[valid], cq[valid], rule)
        res = irls(P[valid], Q[valid], w, delta, iters)
        Qv = Q[valid]
        ext = float(np.linalg.norm(Qv.max(0) - Qv.min(0))) if Qv.shape[0] else 0.0
        res.update(n_valid=int(valid.sum()), extent=ext, pair=k)
        out.append(res)
    return out
