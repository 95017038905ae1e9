"""Reverse-mode derivative of the Huber-IRLS Umeyama registration: the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper has no gradient; this is the adjoint of the forward computation in
``oracle.register`` (Sec. III-C, Eq. (sim3) solved by weighted Umeyama and
wrapped in Huber IRLS), unrolled through every iteration (the Huber weights
of iteration k depend on S_{k-1}, hence on the inputs).  Upstream gradients
are dL/ds, dL/dR (3x3, ambient), dL/dt of the final S = S_K and dL/dcost,
with cost = sum omega_i r_i(S_K)^2 / sum omega_i (omega = last weights).

Each step is written in the forward's own variables:

* moments A = sum omega q p^T, b_p = sum omega p, b_q = sum omega q,
  W = sum omega, C = sum omega |p|^2; mu = b / W;
  Sigma = A/W - mu_q mu_p^T; v = C/W - |mu_p|^2;
* R = U' V^T with Sigma = U' D' V^T a signed SVD (U' = U E, D' = D E);
  with G' = U'^T (dL/dR) V: dL/dSigma = U' K V^T, K_ij = (G'_ij - G'_ji) /
  (d'_i + d'_j) for i != j (the polar-factor form, no 1/(d_i^2 - d_j^2));
* s = tr(D')/v with d tr(D') / dSigma = R;  t = mu_q - s R mu_p;
* omega = w h, h = 1 (r <= delta) or delta / r, r = |s R p + t - q|.

The base weight is w = c_p c_q (or c_p); the normalisation by sum w drops
out because the result is invariant to a global scale of w.
"""
from __future__ import annotations

import numpy as np

from . import sim3
from .register import RANK_REL_TOL


def _solve_fwd(P, Q, om):
    W = om.sum()
    bp = om @ P
    bq = om @ Q
    A = (Q * om[:, None]).T @ P
    C = float(om @ (P * P).sum(1))
    mup, muq = bp / W, bq / W
    Sig = A / W - np.outer(muq, mup)
    v = C / W - float(mup @ mup)
    U, D, Vt = np.linalg.svd(Sig)
    E = np.ones(3)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        E[2] = -1.0
    Up = U * E[None, :]
    dp = D * E
    R = Up @ Vt
    tau = float(dp.sum())
    s = tau / v
    t = muq - s * (R @ mup)
    ok = P.shape[0] >= 3 and W > 0 and v > 0 and D[0] > 0 and D[1] > RANK_REL_TOL * D[0]
    return dict(W=W, bp=bp, bq=bq, A=A, C=C, mup=mup, muq=muq, Sig=Sig, v=v, Up=Up, dp=dp,
                V=Vt.T, R=R, tau=tau, s=s, t=t, ok=ok)


def _solve_bwd(f, P, Q, om, gs, gR, gt):
    """Back through one weighted-Umeyama solve: returns (g_omega, gP, gQ)."""
    s, R, mup, muq, W, v = f["s"], f["R"], f["mup"], f["muq"], f["W"], f["v"]
    # t = mu_q - s R mu_p
    gmuq = gt.copy()
    gs_tot = gs - float(gt @ (R @ mup))
    gR_tot = gR - s * np.outer(gt, mup)
    gmup = -s * (R.T @ gt)
    # s = tau / v
    gtau = gs_tot / v
    gv = -gs_tot * f["tau"] / (v * v)
    gSig = gtau * R
    # R = U' V^T
    Up, V, dp = f["Up"], f["V"], f["dp"]
    G = Up.T @ gR_tot @ V
    K = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            if i != j:
                K[i, j] = (G[i, j] - G[j, i]) / (dp[i] + dp[j])
    gSig = gSig + Up @ K @ V.T
    # Sigma = A/W - mu_q mu_p^T ; v = C/W - |mu_p|^2
    gA = gSig / W
    gmuq = gmuq - gSig @ mup
    gmup = gmup - gSig.T @ muq
    gC = gv / W
    gmup = gmup - 2.0 * gv * mup
    gW = -float((gSig * f["A"]).sum()) / (W * W) - gv * f["C"] / (W * W)
    gbp = gmup / W
    gbq = gmuq / W
    gW += -float(gmup @ f["bp"]) / (W * W) - float(gmuq @ f["bq"]) / (W * W)
    # per point
    g_om = gW + P @ gbp + Q @ gbq + gC * (P * P).sum(1) + np.einsum("ni,ij,nj->n", Q, gA, P)
    gP = om[:, None] * (gbp[None, :] + 2.0 * gC * P + Q @ gA)
    gQ = om[:, None] * (gbq[None, :] + P @ gA.T)
    return g_om, gP, gQ


def _residual(S, P, Q, estimate_dtype):
    """e = s R p + t - q; with estimate_dtype, the estimate as a path that
    holds it in that type uses it: A = s R and b = t + A m_p - m_q around the
    means m of P and Q, rounded to estimate_dtype, e = A (p - m_p) + b - (q - m_q)
    (everything else in FP64)."""
    if estimate_dtype is None:
        return sim3.act(S, P) - Q
    s, R, t = S
    mp, mq = P.mean(0), Q.mean(0)
    A = s * R
    b = t + A @ mp - mq
    A = A.astype(estimate_dtype).astype(np.float64)
    b = b.astype(estimate_dtype).astype(np.float64)
    return (P - mp) @ A.T + b - (Q - mq)


def irls_forward(P, Q, w, delta, iters, estimate_dtype=None):
    """Forward pass keeping what the reverse pass needs.  estimate_dtype
    (default None: FP64 throughout) rounds the estimate that weights the next
    iteration, as ``_residual`` describes: a model of a path that keeps it in
    FP32, used to size that rounding's effect on the gradients."""
    P = np.asarray(P, np.float64)
    Q = np.asarray(Q, np.float64)
    w = np.asarray(w, np.float64)
    tape = []
    S = None
    for k in range(1, iters + 1):
        e = None
        if k == 1:
            r = None
            h = np.ones_like(w)
        else:
            e = _residual(S, P, Q, estimate_dtype)
            r = np.linalg.norm(e, axis=1)
            h = np.where(r <= delta, 1.0, delta / np.where(r > 0, r, 1.0))
        om = w * h
        f = _solve_fwd(P, Q, om)
        tape.append(dict(f=f, r=r, h=h, om=om, S_prev=S, e=e))
        if not f["ok"]:
            return None, tape, 0.0
        S = (f["s"], f["R"], f["t"])
    om = tape[-1]["om"]
    eK = sim3.act(S, P) - Q
    cost = float((om * (eK * eK).sum(1)).sum() / om.sum())
    return S, tape, cost


def irls_backward(P, Q, w, delta, tape, S, gs, gR, gt, gcost):
    """Returns (gP [N,3], gQ [N,3], gw [N])."""
    P = np.asarray(P, np.float64)
    Q = np.asarray(Q, np.float64)
    w = np.asarray(w, np.float64)
    gP = np.zeros_like(P)
    gQ = np.zeros_like(Q)
    gw = np.zeros_like(w)
    if S is None:
        return gP, gQ, gw
    gs, gR, gt = float(gs), np.array(gR, np.float64).reshape(3, 3), np.array(gt, np.float64)
    # cost = sum om r^2 / sum om, evaluated at S_K with the last weights
    last = tape[-1]
    om = last["om"]
    s, R, t = S
    e = sim3.act(S, P) - Q
    r2 = (e * e).sum(1)
    Om, J = om.sum(), float(om @ r2)
    gJ = gcost / Om
    gOm = -gcost * J / (Om * Om)
    g_om_extra = gJ * r2 + gOm
    ge = 2.0 * gJ * om[:, None] * e
    gP += s * (ge @ R)
    gQ -= ge
    gs += float((ge * (P @ R.T)).sum())
    gR = gR + s * ge.T @ P
    gt = gt + ge.sum(0)
    g_om_next = g_om_extra
    for k in range(len(tape), 0, -1):
        rec = tape[k - 1]
        g_om, dP, dQ = _solve_bwd(rec["f"], P, Q, rec["om"], gs, gR, gt)
        g_om = g_om + g_om_next
        gP += dP
        gQ += dQ
        gw += g_om * rec["h"]
        if k == 1:
            break
        gh = g_om * w
        r = rec["r"]
        gr = np.where(r > delta, -gh * delta / np.where(r > 0, r * r, 1.0), 0.0)
        sp, Rp, tp = rec["S_prev"]
        e = rec["e"]
        ge = (gr / np.where(r > 0, r, 1.0))[:, None] * e
        gP += sp * (ge @ Rp)
        gQ -= ge
        gs = float((ge * (P @ Rp.T)).sum())
        gR = sp * ge.T @ P
        gt = ge.sum(0)
        g_om_next = 0.0
    return gP, gQ, gw


def weight_grads(gw, cp, cq, rule="product"):
    if rule == "product":
        return gw * cq, gw * cp
    return gw.copy(), np.zeros_like(cq)


def geodesic_loss_grad(S_hat, S_gt, h=1e-6):
    """L = ||log(S_gt^-1 S_hat)||^2 and its gradient as (gs, gR, gt).

    The tangent gradient g (right perturbation S_hat Exp(delta)) is taken by
    central differences; it maps to the ambient (s, R, t) gradient through
    dt = s R drho, dR = R dphi^, ds = s dsigma.
    """
    L = sim3.geodesic_sq(S_gt, S_hat)
    g = np.zeros(7)
    for a in range(7):
        d = np.zeros(7)
        d[a] = h
        g[a] = (sim3.geodesic_sq(S_gt, sim3.compose(S_hat, sim3.exp(d)))
                - sim3.geodesic_sq(S_gt, sim3.compose(S_hat, sim3.exp(-d)))) / (2 * h)
    s, R, t = S_hat
    gt = R @ g[0:3] / s
    gR = R @ sim3.hat(g[3:6] / 2.0)
    gs = g[6] / s
    return L, gs, gR, gt
