"""Pins of the Sim(3) algebra and pose-graph oracle (Sec. III-E).

Closed forms (Rodrigues, pure-scale exponential), group identities, a
consistent graph with zero energy, convergence back to the truth, a tree
that keeps its chained poses, and the first-order optimality of the
Gauss-Newton result on a noisy loop (numerical gradient of chi^2).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import pose_graph as pg
from oracle import sim3


def rand_sim3(rng, scale=1.0):
    return (float(np.exp(0.3 * rng.normal())), Rotation.random(random_state=rng).as_matrix(),
            scale * rng.normal(size=3))


def close(A, B, tol):
    return abs(A[0] - B[0]) <= tol * abs(B[0]) and np.abs(A[1] - B[1]).max() <= tol \
        and np.abs(A[2] - B[2]).max() <= tol * (1 + np.abs(B[2]).max())


def test_exp_closed_forms():
    rng = np.random.default_rng(1)
    for _ in range(5):
        phi = rng.normal(size=3)
        th = np.linalg.norm(phi)
        K = sim3.hat(phi / th)
        Rrod = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K      # Rodrigues
        s, R, t = sim3.exp(np.concatenate([np.zeros(3), phi, [0.0]]))
        assert abs(s - 1) < 1e-14 and np.abs(R - Rrod).max() < 1e-13 and np.abs(t).max() == 0
        sig = rng.normal()
        rho = rng.normal(size=3)
        s, R, t = sim3.exp(np.concatenate([rho, np.zeros(3), [sig]]))
        assert abs(s - np.exp(sig)) < 1e-13 * np.exp(sig)
        assert np.abs(t - (np.exp(sig) - 1) / sig * rho).max() < 1e-13 * (1 + np.abs(t).max())
        # pure translation: Exp(rho, 0, 0) = (1, I, rho)
        s, R, t = sim3.exp(np.concatenate([rho, np.zeros(4)]))
        assert np.abs(t - rho).max() < 1e-14 and np.abs(R - np.eye(3)).max() < 1e-15


def test_exp_log_round_trip_and_group_laws():
    rng = np.random.default_rng(2)
    for _ in range(20):
        xi = rng.normal(size=7) * np.array([2, 2, 2, 0.8, 0.8, 0.8, 0.5])
        xi2 = sim3.log(sim3.exp(xi))
        assert np.abs(xi2 - xi).max() < 1e-12
        T = rand_sim3(rng, 3.0)
        assert close(sim3.exp(sim3.log(T)), T, 1e-12)
        A, B, C = rand_sim3(rng), rand_sim3(rng), rand_sim3(rng)
        assert close(sim3.compose(sim3.compose(A, B), C), sim3.compose(A, sim3.compose(B, C)), 1e-13)
        assert close(sim3.compose(A, sim3.inverse(A)), sim3.identity(), 1e-13)
        X = rng.normal(size=(5, 3))
        assert np.abs(sim3.act(sim3.compose(A, B), X) - sim3.act(A, sim3.act(B, X))).max() < 1e-12
    # Exp(xi) Exp(-xi) = I and exp of a scaled generator commutes
    xi = rng.normal(size=7)
    assert close(sim3.compose(sim3.exp(xi), sim3.exp(-xi)), sim3.identity(), 1e-12)
    assert close(sim3.compose(sim3.exp(0.3 * xi), sim3.exp(0.7 * xi)), sim3.exp(xi), 1e-12)


@pytest.mark.parametrize("angle", [1e-9, 1e-4, 1.0, 3.0, np.pi - 1e-6])
@pytest.mark.parametrize("sigma", [0.0, 1e-9, 0.7, -1.2])
def test_exp_log_round_trip_at_extreme_angles_and_scales(angle, sigma):
    """Log(Exp(xi)) = xi from a vanishing rotation to one just short of pi, and
    from unit scale (sigma = 0, where the translation series degenerates) to
    strong shrinking and growth."""
    rng = np.random.default_rng(int(angle * 1e3) + int(sigma * 10) + 50)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    xi = np.concatenate([2.0 * rng.normal(size=3), angle * axis, [sigma]])
    assert np.abs(sim3.log(sim3.exp(xi)) - xi).max() < 1e-12


def random_graph(rng, n, loops, noise=0.0):
    T = [sim3.identity()] + [rand_sim3(rng, 2.0) for _ in range(n - 1)]
    ei = list(range(n - 1))
    ej = list(range(1, n))
    while len(ei) < n - 1 + loops:
        i, j = sorted(rng.choice(n, 2, replace=False))
        if j - i >= 2:
            ei.append(int(i))
            ej.append(int(j))
    Tij = []
    for i, j in zip(ei, ej):
        M = sim3.compose(sim3.inverse(T[i]), T[j])
        if noise:
            M = sim3.compose(M, sim3.exp(noise * rng.normal(size=7)))
        Tij.append(M)
    return T, ei, ej, Tij


def test_consistent_graph_zero_energy_and_no_step():
    rng = np.random.default_rng(3)
    T, ei, ej, Tij = random_graph(rng, 8, 4)
    assert pg.chi2(T, ei, ej, Tij) < 1e-24
    nodes, hist, steps = pg.gauss_newton(T, ei, ej, Tij, iters=2)
    assert max(steps) < 1e-9
    for a, b in zip(nodes, T):
        assert close(a, b, 1e-10)


def test_perturbed_consistent_graph_returns_to_truth():
    rng = np.random.default_rng(4)
    T, ei, ej, Tij = random_graph(rng, 7, 3)
    start = [T[0]] + [sim3.compose(t, sim3.exp(0.05 * rng.normal(size=7))) for t in T[1:]]
    nodes, hist, steps = pg.gauss_newton(start, ei, ej, Tij, iters=10)
    assert hist[-1] < 1e-20 and hist[0] > 1e-4
    for a, b in zip(nodes, T):
        assert close(a, b, 1e-8)


def test_tree_keeps_chained_poses():
    rng = np.random.default_rng(5)
    T, ei, ej, Tij = random_graph(rng, 9, 0, noise=0.05)
    init = pg.chain_init(9, ei, ej, Tij)
    assert pg.chi2(init, ei, ej, Tij) < 1e-22
    nodes, hist, steps = pg.gauss_newton(init, ei, ej, Tij, iters=3)
    for a, b in zip(nodes, init):
        assert close(a, b, 1e-9)


def test_chain_init_follows_edge_direction():
    rng = np.random.default_rng(6)
    T, _, _, _ = random_graph(rng, 5, 0)
    ei, ej = [1, 1, 3, 3], [0, 2, 2, 4]          # mixed directions
    Tij = [sim3.compose(sim3.inverse(T[i]), T[j]) for i, j in zip(ei, ej)]
    init = pg.chain_init(5, ei, ej, Tij, root=0, T_root=T[0])
    for a, b in zip(init, T):
        assert close(a, b, 1e-11)


def test_noisy_loop_first_order_optimality():
    rng = np.random.default_rng(7)
    T, ei, ej, Tij = random_graph(rng, 6, 2, noise=0.02)
    init = pg.chain_init(6, ei, ej, Tij)
    # GN converges linearly on a problem with non-zero residuals
    nodes, hist, steps = pg.gauss_newton(init, ei, ej, Tij, iters=30)
    assert hist[-1] < hist[0] and steps[-1] < 1e-11
    # numerical gradient of chi^2 w.r.t. right perturbations of every free node
    h = 1e-6
    for v in range(1, 6):
        for a in range(7):
            d = np.zeros(7)
            d[a] = h
            up = list(nodes)
            dn = list(nodes)
            up[v] = sim3.compose(nodes[v], sim3.exp(d))
            dn[v] = sim3.compose(nodes[v], sim3.exp(-d))
            g = (pg.chi2(up, ei, ej, Tij) - pg.chi2(dn, ei, ej, Tij)) / (2 * h)
            assert abs(g) < 1e-7, (v, a, g)


def test_fixed_node_only_chooses_the_gauge():
    """The edge error is left-invariant (T_v -> G T_v for every node leaves it
    unchanged), so holding a different node changes only the gauge: chi^2 and
    every relative pose T_i^-1 T_j of the optimum agree, and the held node
    keeps its initial pose."""
    rng = np.random.default_rng(9)
    T, ei, ej, Tij = random_graph(rng, 6, 2, noise=0.02)
    a, ha, sa = pg.gauss_newton(pg.chain_init(6, ei, ej, Tij), ei, ej, Tij, iters=30, fixed=0)
    start = pg.chain_init(6, ei, ej, Tij, root=3, T_root=rand_sim3(rng))
    b, hb, sb = pg.gauss_newton(start, ei, ej, Tij, iters=30, fixed=3)
    assert sa[-1] < 1e-11 and sb[-1] < 1e-11
    assert hb[-1] < hb[0] and abs(ha[-1] - hb[-1]) <= 1e-10 * ha[-1]
    assert b[3][0] == start[3][0] and np.array_equal(b[3][1], start[3][1]) \
        and np.array_equal(b[3][2], start[3][2])
    for i in range(6):
        for j in range(6):
            ra = sim3.compose(sim3.inverse(a[i]), a[j])
            rb = sim3.compose(sim3.inverse(b[i]), b[j])
            assert close(rb, ra, 1e-9), (i, j)


def test_information_matrix_scales_energy():
    rng = np.random.default_rng(8)
    T, ei, ej, Tij = random_graph(rng, 5, 1, noise=0.03)
    info = [np.diag(rng.uniform(0.5, 2, 7)).ravel() for _ in ei]
    e = [pg.edge_error(T[i], T[j], M) for i, j, M in zip(ei, ej, Tij)]
    ref = sum(float(x @ np.asarray(I).reshape(7, 7) @ x) for x, I in zip(e, info))
    assert abs(pg.chi2(T, ei, ej, Tij, info) - ref) < 1e-14 * max(ref, 1)


def test_lm_is_monotone_and_reaches_the_truth():
    """Levenberg-Marquardt (Sec. III-E): chi^2 never increases along the kept
    steps and a consistent graph is recovered from a far start."""
    rng = np.random.default_rng(11)
    T, ei, ej, Tij = random_graph(rng, 7, 3)
    start = [T[0]] + [sim3.compose(t, sim3.exp(0.4 * rng.normal(size=7))) for t in T[1:]]
    nodes, hist, lams = pg.levenberg_marquardt(start, ei, ej, Tij, iters=40, lambda0=1e-2)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 1e-18
    for a, b in zip(nodes, T):
        assert close(a, b, 1e-8)


def test_lm_rejects_a_step_that_raises_the_energy():
    """From the identity, an undamped step overshoots: LM discards it, raises
    lambda tenfold and keeps the poses; a later, damped step is kept."""
    rng = np.random.default_rng(32)
    T, ei, ej, Tij = random_graph(rng, 6, 4, noise=0.6)   # strongly inconsistent loops
    start = [sim3.identity()] * 6
    _, gn_hist, _ = pg.gauss_newton(start, ei, ej, Tij, iters=1)
    assert gn_hist[1] > gn_hist[0]                   # the plain step raises chi^2
    nodes, hist, lams = pg.levenberg_marquardt(start, ei, ej, Tij, iters=12, lambda0=1e-6)
    assert hist[1] == hist[0] and lams[1] == lams[0] * 10.0
    assert hist[-1] < hist[0]
    assert all(b <= a for a, b in zip(hist, hist[1:]))


def test_lm_fixed_point_is_stationary():
    rng = np.random.default_rng(13)
    T, ei, ej, Tij = random_graph(rng, 6, 2, noise=0.02)
    init = pg.chain_init(6, ei, ej, Tij)
    nodes, hist, lams = pg.levenberg_marquardt(init, ei, ej, Tij, iters=40, lambda0=1e-3)
    h = 1e-6
    for v in range(1, 6):
        for a in range(7):
            d = np.zeros(7)
            d[a] = h
            up, dn = list(nodes), list(nodes)
            up[v] = sim3.compose(nodes[v], sim3.exp(d))
            dn[v] = sim3.compose(nodes[v], sim3.exp(-d))
            g = (pg.chi2(up, ei, ej, Tij) - pg.chi2(dn, ei, ej, Tij)) / (2 * h)
            assert abs(g) < 1e-7, (v, a, g)
