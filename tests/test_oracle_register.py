"""Pins of the registration oracle (Sec. III-C, Eq. (sim3) and weighted Umeyama).

Each test checks the oracle against something other than itself: exact
recovery of a known transform, group properties, Horn's independent
quaternion solution, brute-force nonlinear least squares, a brute-force Huber
minimiser, and invariances that any correct solver has.
"""
import numpy as np
import pytest
from scipy.optimize import least_squares, minimize
from scipy.spatial.transform import Rotation

from oracle import register as reg
from oracle import sim3


def rand_sim3(rng):
    q = rng.normal(size=4)
    R = Rotation.from_quat(q / np.linalg.norm(q)).as_matrix()
    return (float(rng.uniform(0.5, 2.0)), R, rng.normal(size=3))


def cloud(rng, n, spread=(3.0, 2.0, 1.0)):
    return rng.normal(size=(n, 3)) * np.asarray(spread) + rng.uniform(-5, 5, size=3)


@pytest.mark.parametrize("seed", range(5))
def test_noise_free_exact_recovery(seed):
    rng = np.random.default_rng(seed)
    P = cloud(rng, 60)
    S = rand_sim3(rng)
    Q = sim3.act(S, P)
    w = rng.uniform(0.1, 3.0, size=60)
    (s, R, t), st = reg.weighted_umeyama(P, Q, w)
    assert st == 0
    assert abs(s / S[0] - 1) < 1e-12
    assert np.abs(R - S[1]).max() < 1e-12
    assert np.abs(t - S[2]).max() < 1e-11


@pytest.mark.parametrize("seed", range(6))
def test_proper_rotation_even_for_reflections(seed):
    rng = np.random.default_rng(seed)
    P = cloud(rng, 40)
    Q = P * np.array([1, 1, -1]) + rng.normal(size=(40, 3)) * 0.3   # mirror image: det < 0 case
    if seed % 2:
        Q = sim3.act(rand_sim3(rng), P) + rng.normal(size=(40, 3))
    (s, R, t), st = reg.weighted_umeyama(P, Q, rng.uniform(0.1, 1, size=40))
    assert st == 0
    assert abs(np.linalg.det(R) - 1) < 1e-14
    assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
    assert s > 0


def horn_rotation(Pc, Qc, w):
    """Horn (1987): the rotation is the top eigenvector of a 4x4 symmetric matrix."""
    M = (Pc * w[:, None]).T @ Qc          # sum w p q^T
    Sxx, Sxy, Sxz = M[0]
    Syx, Syy, Syz = M[1]
    Szx, Szy, Szz = M[2]
    N = np.array([
        [Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
        [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
        [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
        [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    vals, vecs = np.linalg.eigh(N)
    q0, qx, qy, qz = vecs[:, -1]
    return Rotation.from_quat([qx, qy, qz, q0]).as_matrix()


@pytest.mark.parametrize("seed", range(5))
def test_rotation_matches_horn(seed):
    rng = np.random.default_rng(100 + seed)
    P = cloud(rng, 200)
    S = rand_sim3(rng)
    Q = sim3.act(S, P) + 0.2 * rng.normal(size=(200, 3))
    w = rng.uniform(0.2, 2.0, size=200)
    (s, R, t), st = reg.weighted_umeyama(P, Q, w)
    mp = (w[:, None] * P).sum(0) / w.sum()
    mq = (w[:, None] * Q).sum(0) / w.sum()
    Rh = horn_rotation(P - mp, Q - mq, w)
    assert np.abs(R - Rh).max() < 1e-10
    # Horn's scale (asymmetric form): sum w q'.(R p') / sum w |p'|^2
    sh = float((w * ((Q - mq) * ((P - mp) @ Rh.T)).sum(1)).sum() / (w * ((P - mp) ** 2).sum(1)).sum())
    assert abs(s - sh) < 1e-12 * abs(sh) + 1e-14


def _params_to_sim3(x):
    return (float(np.exp(x[0])), Rotation.from_rotvec(x[1:4]).as_matrix(), x[4:7])


@pytest.mark.parametrize("seed", range(3))
def test_brute_force_least_squares_10_points(seed):
    rng = np.random.default_rng(200 + seed)
    P = cloud(rng, 10)
    S = rand_sim3(rng)
    Q = sim3.act(S, P) + 0.05 * rng.normal(size=(10, 3))
    w = rng.uniform(0.2, 2.0, size=10)
    (s, R, t), st = reg.weighted_umeyama(P, Q, w)
    cost_o = float((w * ((sim3.act((s, R, t), P) - Q) ** 2).sum(1)).sum())

    def resid(x):
        return (np.sqrt(w)[:, None] * (sim3.act(_params_to_sim3(x), P) - Q)).ravel()

    best = None
    for _ in range(100):
        x0 = np.concatenate([[rng.uniform(-1, 1)], Rotation.random(random_state=rng).as_rotvec(),
                             rng.normal(size=3) * 3])
        sol = least_squares(resid, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15)
        if best is None or sol.cost < best.cost:
            best = sol
    Sb = _params_to_sim3(best.x)
    assert 2 * best.cost >= cost_o * (1 - 1e-12)
    assert abs(2 * best.cost - cost_o) <= 1e-9 * cost_o
    assert abs(Sb[0] / s - 1) < 1e-6
    assert sim3.rotation_angle(Sb[1], R) < 1e-6
    assert np.abs(Sb[2] - t).max() < 1e-5


def test_weight_scale_invariance_and_equivariance():
    rng = np.random.default_rng(7)
    P = cloud(rng, 300)
    Q = sim3.act(rand_sim3(rng), P) + 0.3 * rng.normal(size=(300, 3))
    w = rng.uniform(0.1, 3, size=300)
    S1, _ = reg.weighted_umeyama(P, Q, w)
    S2, _ = reg.weighted_umeyama(P, Q, 1e3 * w)
    assert abs(S1[0] - S2[0]) < 1e-12 and np.abs(S1[1] - S2[1]).max() < 1e-12
    assert np.abs(S1[2] - S2[2]).max() < 1e-11
    Sp = rand_sim3(rng)
    S3, _ = reg.weighted_umeyama(P, sim3.act(Sp, Q), w)
    C = sim3.compose(Sp, S1)
    assert abs(S3[0] / C[0] - 1) < 1e-12 and np.abs(S3[1] - C[1]).max() < 1e-12
    assert np.abs(S3[2] - C[2]).max() < 1e-10


def test_degenerate_cases():
    rng = np.random.default_rng(3)
    P = cloud(rng, 2)
    assert reg.weighted_umeyama(P, P, np.ones(2))[1] == reg.DEG_FEW
    P = cloud(rng, 10)
    assert reg.weighted_umeyama(P, P, np.zeros(10))[1] == reg.DEG_WEIGHT
    L = np.zeros((10, 3))
    L[:, 0] = np.arange(10.0)                       # collinear: rank 1
    assert reg.weighted_umeyama(L, L + 1.0, np.ones(10))[1] == reg.DEG_RANK
    Pl = cloud(rng, 50)
    Pl[:, 2] = 0.0                                   # planar: rank 2 is allowed
    S = rand_sim3(rng)
    (s, R, t), st = reg.weighted_umeyama(Pl, sim3.act(S, Pl), np.ones(50))
    assert st == 0 and abs(s / S[0] - 1) < 1e-12 and np.abs(R - S[1]).max() < 1e-11
    res = reg.irls(L, L, np.ones(10), 0.02, 10)
    assert res["status"] == reg.DEG_RANK and res["S"][0] == 1.0


@pytest.mark.parametrize("seed", range(3))
def test_irls_noise_free_every_iteration_exact(seed):
    rng = np.random.default_rng(300 + seed)
    P = cloud(rng, 100)
    S = rand_sim3(rng)
    res = reg.irls(P, sim3.act(S, P), rng.uniform(0.1, 2, 100), 0.02, 10)
    assert res["status"] == 0 and len(res["history"]) == 10
    for Sk in res["history"]:
        assert abs(Sk[0] / S[0] - 1) < 1e-12 and np.abs(Sk[1] - S[1]).max() < 1e-11
        assert np.abs(Sk[2] - S[2]).max() < 1e-10
    assert res["cost"] < 1e-20


def test_irls_large_delta_is_umeyama():
    rng = np.random.default_rng(11)
    P = cloud(rng, 80)
    Q = sim3.act(rand_sim3(rng), P) + 0.5 * rng.normal(size=(80, 3))
    w = rng.uniform(0.1, 2, 80)
    res = reg.irls(P, Q, w, 1e9, 7)
    S, _ = reg.weighted_umeyama(P, Q, w)
    assert abs(res["S"][0] - S[0]) < 1e-13 and np.abs(res["S"][1] - S[1]).max() < 1e-13


def umeyama_min_error(P, Q, w):
    """Umeyama (1991): the minimum over (s, R, t) of (1/W) sum w |s R p + t - q|^2
    is sigma_q^2 - (d1 + d2 + e d3)^2 / sigma_p^2, with d1 >= d2 >= d3 the
    singular values of the weighted cross-covariance and e the sign of its
    determinant.  No residual is evaluated; the singular values come from the
    eigenvalues of C^T C."""
    W = w.sum()
    mp, mq = (w[:, None] * P).sum(0) / W, (w[:, None] * Q).sum(0) / W
    Pc, Qc = P - mp, Q - mq
    vp = (w * (Pc * Pc).sum(1)).sum() / W
    vq = (w * (Qc * Qc).sum(1)).sum() / W
    C = (w[:, None] * Qc).T @ Pc / W
    d = np.sqrt(np.clip(np.linalg.eigvalsh(C.T @ C), 0.0, None))[::-1]
    e = 1.0 if np.linalg.det(C) >= 0 else -1.0
    return vq - (d[0] + d[1] + e * d[2]) ** 2 / vp


@pytest.mark.parametrize("iters", [1, 4])
def test_cost_is_umeyamas_minimum_error_for_the_last_weights(iters):
    """The reported cost is sum omega r(S_K)^2 / sum omega with the weights of
    the last solve, omega = w min(1, delta / r(S_{K-1})); S_K minimises that
    weighted error, so the cost is Umeyama's closed-form minimum for omega."""
    rng = np.random.default_rng(500 + iters)
    n, delta = 400, 0.05
    P = cloud(rng, n)
    Q = sim3.act(rand_sim3(rng), P) + 0.01 * rng.normal(size=(n, 3))
    out = rng.random(n) < 0.2
    Q[out] += rng.normal(size=(int(out.sum()), 3))          # outliers far past delta
    w = rng.uniform(0.1, 2.0, n)
    res = reg.irls(P, Q, w, delta, iters)
    assert res["status"] == 0 and len(res["history"]) == iters
    om = w
    if iters > 1:
        s, R, t = res["history"][-2]
        r = np.linalg.norm(P @ (s * R).T + t - Q, axis=1)
        assert (r > delta).sum() > 50                        # the Huber branch is taken
        om = w * np.minimum(1.0, delta / r)
    ref = umeyama_min_error(P, Q, om)
    assert ref > 0
    assert abs(res["cost"] - ref) <= 1e-10 * ref


def huber_rho(r, d):
    return np.where(r <= d, 0.5 * r * r, d * r - 0.5 * d * d)


@pytest.mark.parametrize("seed", range(3))
def test_irls_converges_to_brute_force_huber_minimiser(seed):
    """IRLS for Huber is a descent method for sum w rho_delta(r) (rho: Huber)."""
    rng = np.random.default_rng(400 + seed)
    n = 30
    P = cloud(rng, n, (1.0, 0.8, 0.6))
    S = rand_sim3(rng)
    Q = sim3.act(S, P) + 0.01 * rng.normal(size=(n, 3))
    Q[:4] += rng.normal(size=(4, 3)) * 2.0           # outliers
    w = rng.uniform(0.3, 2.0, n)
    delta = 0.03
    res = reg.irls(P, Q, w, delta, 500)
    So = res["S"]

    def energy(x):
        T = _params_to_sim3(x)
        return float((w * huber_rho(np.linalg.norm(sim3.act(T, P) - Q, axis=1), delta)).sum())

    x_o = np.concatenate([[np.log(So[0])], Rotation.from_matrix(So[1]).as_rotvec(), So[2]])
    best = None
    for _ in range(6):
        x0 = x_o + rng.normal(size=7) * 0.05
        sol = minimize(energy, x0, method="Nelder-Mead",
                       options=dict(xatol=1e-10, fatol=1e-14, maxiter=6000, maxfev=6000))
        sol = minimize(energy, sol.x, method="BFGS", options=dict(gtol=1e-12))
        if best is None or sol.fun < best.fun:
            best = sol
    assert energy(x_o) <= best.fun * (1 + 1e-9) + 1e-15
    Sb = _params_to_sim3(best.x)
    assert abs(Sb[0] / So[0] - 1) < 1e-5
    assert sim3.rotation_angle(Sb[1], So[1]) < 1e-5


def test_correspondence_validity_bruteforce():
    rng = np.random.default_rng(5)
    nf, hw = 4, 37
    xyz = rng.normal(size=(nf, hw, 3)).astype(np.float32)
    conf = rng.lognormal(0, 0.5, size=(nf, hw)).astype(np.float32)
    xyz[1, 3, 1] = np.nan
    xyz[2, 5, 0] = np.inf
    conf[0, 7] = np.nan
    conf[3, 9] = 0.0
    link_off = np.array([0, 2, 3])
    src = np.array([0, 1, 2])
    tgt = np.array([2, 3, 0])
    for k in range(2):
        P, Q, cp, cq, valid = reg.pair_correspondences(xyz, conf, link_off, src, tgt, k, 0.5)
        rows = []
        for l in range(link_off[k], link_off[k + 1]):
            for i in range(hw):
                p, q = xyz[src[l], i], xyz[tgt[l], i]
                a, b = conf[src[l], i], conf[tgt[l], i]
                ok = all(np.isfinite(v) for v in list(p) + list(q) + [a, b]) and a > 0.5 and b > 0.5
                rows.append(ok)
        assert valid.tolist() == rows
        assert P.shape == (hw * (link_off[k + 1] - link_off[k]), 3)
