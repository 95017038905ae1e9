"""Pins of the adjoint oracle: FP64 central finite differences (h = 1e-6) of
the forward registration loss, skipping points whose residual sits within
1e-4 of the Huber kink (where the loss is not differentiable)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import adjoint as adj
from oracle import register as reg
from oracle import sim3


def problem(seed, n=60, outliers=6):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, 3)) * np.array([2.0, 1.5, 1.0]) + 1.0
    S = (float(rng.uniform(0.6, 1.8)), Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3))
    Q = sim3.act(S, P) + 0.02 * rng.normal(size=(n, 3))
    Q[:outliers] += rng.normal(size=(outliers, 3))
    cp = rng.lognormal(0, 0.5, n)
    cq = rng.lognormal(0, 0.5, n)
    return P, Q, cp, cq, S


def loss(P, Q, cp, cq, S_gt, delta, iters, lam):
    S, tape, cost = adj.irls_forward(P, Q, cp * cq, delta, iters)
    return sim3.geodesic_sq(S_gt, S) + lam * cost


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_matches_finite_differences(seed):
    P, Q, cp, cq, S_gt = problem(seed)
    delta, iters, lam = 0.05, 10, 1.0
    w = cp * cq
    S, tape, cost = adj.irls_forward(P, Q, w, delta, iters)
    # forward agrees with the plain oracle
    ref = reg.irls(P, Q, w, delta, iters)
    assert abs(S[0] - ref["S"][0]) < 1e-12 and np.abs(S[1] - ref["S"][1]).max() < 1e-12
    assert abs(cost - ref["cost"]) < 1e-12 * max(cost, 1e-30) + 1e-18
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S_gt)
    gP, gQ, gw = adj.irls_backward(P, Q, w, delta, tape, S, gs, gR, gt, lam)
    gcp, gcq = adj.weight_grads(gw, cp, cq)
    # points near the Huber kink at any iteration are not differentiable
    near = np.zeros(len(w), bool)
    for rec in tape[1:]:
        near |= np.abs(rec["r"] - delta) < 1e-4
    h = 1e-6
    rng = np.random.default_rng(seed)
    idx = [i for i in rng.permutation(len(w)) if not near[i]][:12]
    assert len(idx) >= 8
    for i in idx:
        for a in range(3):
            for X, G in ((P, gP), (Q, gQ)):
                Xp, Xm = X.copy(), X.copy()
                Xp[i, a] += h
                Xm[i, a] -= h
                args_p = (Xp, Q) if X is P else (P, Xp)
                args_m = (Xm, Q) if X is P else (P, Xm)
                fd = (loss(*args_p, cp, cq, S_gt, delta, iters, lam)
                      - loss(*args_m, cp, cq, S_gt, delta, iters, lam)) / (2 * h)
                assert abs(fd - G[i, a]) <= 1e-6 * max(1.0, abs(fd)), (i, a, fd, G[i, a])
        for c, G in ((cp, gcp), (cq, gcq)):
            cpp, cmm = c.copy(), c.copy()
            cpp[i] += h
            cmm[i] -= h
            a1 = (cpp, cq) if c is cp else (cp, cpp)
            a2 = (cmm, cq) if c is cp else (cp, cmm)
            fd = (loss(P, Q, *a1, S_gt, delta, iters, lam) - loss(P, Q, *a2, S_gt, delta, iters, lam)) / (2 * h)
            assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, G[i])


def test_weight_gradient_orthogonal_to_weights():
    """The loss is invariant to a global scale of w, so sum_i w_i dL/dw_i = 0."""
    P, Q, cp, cq, S_gt = problem(11)
    w = cp * cq
    S, tape, cost = adj.irls_forward(P, Q, w, 0.05, 10)
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S_gt)
    _, _, gw = adj.irls_backward(P, Q, w, 0.05, tape, S, gs, gR, gt, 1.0)
    assert abs(float(gw @ w)) < 1e-9 * float(np.abs(gw * w).sum())


def test_source_weight_rule_matches_finite_differences():
    """With the source-confidence rule (w = c_p) the gradient reaches c_p only:
    dL/dc_p matches central differences and dL/dc_q is zero."""
    P, Q, cp, cq, S_gt = problem(21)
    delta, iters, lam = 0.05, 10, 1.0
    S, tape, cost = adj.irls_forward(P, Q, cp, delta, iters)
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S_gt)
    _, _, gw = adj.irls_backward(P, Q, cp, delta, tape, S, gs, gR, gt, lam)
    gcp, gcq = adj.weight_grads(gw, cp, cq, rule="src")
    assert np.all(gcq == 0.0)

    def loss_src(c):
        S_, _, cost_ = adj.irls_forward(P, Q, c, delta, iters)
        return sim3.geodesic_sq(S_gt, S_) + lam * cost_

    near = np.zeros(len(cp), bool)
    for rec in tape[1:]:
        near |= np.abs(rec["r"] - delta) < 1e-4
    h = 1e-6
    idx = [i for i in range(len(cp)) if not near[i]][:10]
    assert len(idx) >= 8
    for i in idx:
        cpp, cmm = cp.copy(), cp.copy()
        cpp[i] += h
        cmm[i] -= h
        fd = (loss_src(cpp) - loss_src(cmm)) / (2 * h)
        assert abs(fd - gcp[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gcp[i])


def depth_problem(seed, H=6, W=10):
    """Two depth frames of one surface seen from two camera poses (same
    intrinsics), 1 % depth noise and a few outlier depths."""
    from oracle import unproject as unp
    rng = np.random.default_rng(seed)
    fx, cx, cy = 8.0, (W - 1) / 2.0, (H - 1) / 2.0

    def cam(R, t):
        return np.concatenate([[fx, fx, cx, cy], R.ravel(), t])[None]

    Rp, Rq = (Rotation.random(random_state=rng).as_matrix() for _ in range(2))
    tp, tq = rng.normal(size=3), rng.normal(size=3)
    dp = rng.uniform(1.5, 3.0, (1, H, W))
    dq = dp * (1 + 0.01 * rng.normal(size=dp.shape))
    dq[0, 0, :4] *= 1.5
    cp, cq = rng.lognormal(0, 0.5, H * W), rng.lognormal(0, 0.5, H * W)
    R_gt = Rq @ Rp.T
    S_gt = (1.0, R_gt, tq - R_gt @ tp)                  # q = R_gt (p - t_p) + t_q
    return unp, dp, dq, cam(Rp, tp), cam(Rq, tq), cp, cq, S_gt


def test_depth_gradient_matches_finite_differences():
    """The registration's adjoint carried to the depth maps (dL/dd = (R r) .
    dL/dX) matches FP64 central differences of the whole chain: unprojection
    of both frames, Huber-IRLS registration, geodesic loss plus cost."""
    unp, dp, dq, camp, camq, cp, cq, S_gt = depth_problem(31)
    delta, iters, lam = 0.05, 10, 1.0
    w = cp * cq

    def loss_depth(a, b):
        P, Q = unp.unproject(a, camp)[0], unp.unproject(b, camq)[0]
        S_, _, cost_ = adj.irls_forward(P, Q, w, delta, iters)
        return sim3.geodesic_sq(S_gt, S_) + lam * cost_

    P, Q = unp.unproject(dp, camp)[0], unp.unproject(dq, camq)[0]
    S, tape, cost = adj.irls_forward(P, Q, w, delta, iters)
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S_gt)
    gP, gQ, _ = adj.irls_backward(P, Q, w, delta, tape, S, gs, gR, gt, lam)
    gdp = unp.unproject_backward(gP[None], dp, camp)
    gdq = unp.unproject_backward(gQ[None], dq, camq)
    assert np.abs(gdp).max() > 1e-3 and np.abs(gdq).max() > 1e-3
    near = np.zeros(len(w), bool)
    for rec in tape[1:]:
        near |= np.abs(rec["r"] - delta) < 1e-4
    assert (np.abs(tape[-1]["r"]) > delta).sum() >= 2          # both Huber branches taken
    h = 1e-6
    W_ = dp.shape[2]
    idx = [i for i in range(len(w)) if not near[i]][::4]
    assert len(idx) >= 10
    for i in idx:
        v, u = divmod(i, W_)
        for which, G in (("p", gdp), ("q", gdq)):
            a_p, a_m = dp.copy(), dp.copy()
            b_p, b_m = dq.copy(), dq.copy()
            if which == "p":
                a_p[0, v, u] += h
                a_m[0, v, u] -= h
            else:
                b_p[0, v, u] += h
                b_m[0, v, u] -= h
            fd = (loss_depth(a_p, b_p) - loss_depth(a_m, b_m)) / (2 * h)
            assert abs(fd - G[0, v, u]) <= 1e-6 * max(1.0, abs(fd)), (which, v, u, fd, G[0, v, u])


def test_depth_gradient_is_zero_where_a_pixel_has_no_point():
    unp, dp, dq, camp, camq, cp, cq, S_gt = depth_problem(32)
    d = dp.copy()
    d[0, 1, 2], d[0, 3, 4], d[0, 5, 9] = 0.0, -1.0, np.nan
    g = unp.unproject_backward(np.ones((1, d[0].size, 3)), d, camp)
    assert g[0, 1, 2] == 0.0 and g[0, 3, 4] == 0.0 and g[0, 5, 9] == 0.0
    assert np.count_nonzero(g) == d[0].size - 3


def test_estimate_dtype_float64_is_the_plain_forward():
    """The pivot-relative residual of the estimate_dtype model, without
    rounding (float64), is algebraically the plain residual: same estimates,
    costs and gradients to rounding."""
    P, Q, cp, cq, S_gt = problem(5, n=200, outliers=20)
    w = cp * cq
    S, tape, cost = adj.irls_forward(P, Q, w, 0.05, 10)
    S2, tape2, cost2 = adj.irls_forward(P, Q, w, 0.05, 10, estimate_dtype=np.float64)
    assert abs(S2[0] - S[0]) < 1e-12 and np.abs(S2[1] - S[1]).max() < 1e-12
    assert np.abs(S2[2] - S[2]).max() < 1e-11 and abs(cost2 - cost) < 1e-12 * cost
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S_gt)
    g = adj.irls_backward(P, Q, w, 0.05, tape, S, gs, gR, gt, 1.0)
    g2 = adj.irls_backward(P, Q, w, 0.05, tape2, S2, gs, gR, gt, 1.0)
    for a, b in zip(g, g2):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()


def test_gradient_is_far_more_sensitive_to_the_weighting_estimate_than_the_result():
    """Rounding the estimate that weights the next iteration to FP32 (relative
    change <= 2^-24 per element) moves the registration's result by about that
    much, but its gradient by three to four orders of magnitude more (relative
    to the largest gradient element): the curvature of the Huber weight at
    r ~ delta amplifies point offsets of O(1) by O(1 / delta).  This is the
    effect the GPU parity tests allow for on top of their rounding bound."""
    rng = np.random.default_rng(11)
    n = 20000
    P = rng.normal(size=(n, 3)) * np.array([2.0, 1.5, 1.0]) + np.array([3.0, -1.0, 6.0])
    S0 = (1.3, Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3))
    Q = sim3.act(S0, P) + 0.01 * rng.normal(size=(n, 3))
    Q[:2000] += 0.2 * rng.normal(size=(2000, 3))
    w = rng.lognormal(0, 0.3, n)
    delta = 0.02
    S, tape, _ = adj.irls_forward(P, Q, w, delta, 10)
    S32, tape32, _ = adj.irls_forward(P, Q, w, delta, 10, estimate_dtype=np.float32)
    ds = max(abs(S32[0] - S[0]) / S[0], np.abs(S32[1] - S[1]).max())
    L, gs, gR, gt = adj.geodesic_loss_grad(S, S0)
    gP = adj.irls_backward(P, Q, w, delta, tape, S, gs, gR, gt, 1.0)[0]
    gP32 = adj.irls_backward(P, Q, w, delta, tape32, S32, gs, gR, gt, 1.0)[0]
    dg = np.abs(gP32 - gP).max() / np.abs(gP).max()
    assert ds < 2.0 ** -23
    assert 0.0 < dg < 1e-3
    assert dg > 1e3 * ds
