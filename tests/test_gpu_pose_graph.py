"""GPU parity of ec3r_pose_graph_correct (Sec. III-E: e = log(T_ij^-1 T_i^-1 T_j),
chi^2, chaining initialisation, Gauss-Newton) against the FP64 oracle, both
in FP64: poses and chi^2 within 1e-9 relative (translations relative to the
extent of the trajectory)."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import pose_graph as opg
from oracle import sim3
from paper_2510_02080_b300 import ec3r, synth

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def rows(Ts):
    return torch.tensor(np.stack([np.concatenate([[T[0]], np.asarray(T[1]).ravel(), T[2]])
                                  for T in Ts]), dtype=torch.float64, device="cuda")


def tuples(t):
    return [ec3r.sim3_row(r) for r in t.cpu().numpy()]


def assert_poses_close(got, ref, tol=TOL):
    ext = max(float(np.linalg.norm(np.ptp(np.stack([T[2] for T in ref]), axis=0))), 1.0)
    for v, (a, b) in enumerate(zip(got, ref)):
        assert abs(a[0] / b[0] - 1) <= tol, (v, a[0], b[0])
        assert np.abs(a[1] - b[1]).max() <= tol, v
        assert np.linalg.norm(a[2] - b[2]) <= tol * ext, (v, np.linalg.norm(a[2] - b[2]), ext)


def graph_from_synth(g):
    Tij = [(float(g.T_meas.s[k]), g.T_meas.R[k].numpy(), g.T_meas.t[k].numpy())
           for k in range(len(g.ei))]
    return g.ei.numpy(), g.ej.numpy(), Tij


def run_both(ctx, n, ei, ej, Tij, iters, info=None, fixed=0, lm=0.0, start=None):
    start = start if start is not None else [sim3.identity()] * n
    nodes = rows(start)
    info_d = None if info is None else torch.tensor(np.stack(info), dtype=torch.float64,
                                                    device="cuda")
    chi2 = ctx.pose_graph_correct(nodes, ei, ej, rows(Tij), info_d, iters=iters, fixed=fixed,
                                  lm_lambda=lm)
    assert ctx.sync_status() == 0
    init = opg.chain_init(n, ei, ej, Tij, root=fixed, T_root=start[fixed])
    ref, hist, steps = opg.gauss_newton(init, ei, ej, Tij, info=info, iters=iters, fixed=fixed,
                                        lm_lambda=lm)
    return tuples(nodes), chi2.cpu().numpy(), ref, np.array(hist), init


def test_chaining_only_matches_oracle(ctx):
    g = synth.make_pose_graph(synth.SEED_BASE + 3, 60, 10)
    ei, ej, Tij = graph_from_synth(g)
    got, chi2, ref, hist, init = run_both(ctx, 60, ei, ej, Tij, iters=0)
    assert_poses_close(got, init, 1e-12)
    assert abs(chi2[0] - hist[0]) <= TOL * hist[0]


@pytest.mark.parametrize("n,loops,seed", [(30, 8, 1), (200, 40, 3)])
def test_gauss_newton_matches_oracle(ctx, n, loops, seed):
    g = synth.make_pose_graph(synth.SEED_BASE + seed, n, loops)
    ei, ej, Tij = graph_from_synth(g)
    got, chi2, ref, hist, _ = run_both(ctx, n, ei, ej, Tij, iters=10)
    assert hist[-1] < hist[0]
    np.testing.assert_allclose(chi2, hist, rtol=TOL)
    assert_poses_close(got, ref)


def test_information_matrices_fixed_node_and_damping(ctx):
    g = synth.make_pose_graph(synth.SEED_BASE + 7, 25, 6)
    ei, ej, Tij = graph_from_synth(g)
    rng = np.random.default_rng(0)
    info = []
    for _ in ei:
        A = rng.normal(size=(7, 7)) * 0.2
        info.append((A @ A.T + np.diag(rng.uniform(0.5, 2.0, 7))).ravel())
    got, chi2, ref, hist, _ = run_both(ctx, 25, ei, ej, Tij, iters=6, info=info, fixed=4, lm=0.5)
    np.testing.assert_allclose(chi2, hist, rtol=TOL)
    assert_poses_close(got, ref)


def test_chain_is_consistent_after_chaining(ctx):
    """A tree (odometry only): chaining satisfies every edge; GN keeps it."""
    g = synth.make_pose_graph(synth.SEED_BASE + 2, 200, 0)
    ei, ej, Tij = graph_from_synth(g)
    got, chi2, ref, hist, init = run_both(ctx, 200, ei, ej, Tij, iters=10)
    assert chi2.max() < 1e-18
    assert_poses_close(got, ref)


def test_disconnected_node_and_no_edge_block(ctx):
    """Node 5 has no edge: chaining leaves it the identity and its normal block is
    zero, so the factorisation reports a non-positive pivot and skips updates."""
    g = synth.make_pose_graph(synth.SEED_BASE + 9, 5, 0)
    ei, ej, Tij = graph_from_synth(g)
    nodes = rows([sim3.identity()] * 6)
    ctx.pose_graph_correct(nodes, ei, ej, rows(Tij), iters=2)
    assert ctx.sync_status() == 5              # EC3R_ERR_NOT_SPD
    init = opg.chain_init(6, ei, ej, Tij)
    assert_poses_close(tuples(nodes), init, 1e-12)


def test_invalid_edges_rejected(ctx):
    nodes = rows([sim3.identity()] * 3)
    T = rows([sim3.identity()])
    with pytest.raises(ec3r.Ec3rError):
        ctx.pose_graph_correct(nodes, [1], [1], T)
    with pytest.raises(ec3r.Ec3rError):
        ctx.pose_graph_correct(nodes, [0], [3], T)


@pytest.mark.timeout(1800)
def test_large_loop_graph_converges_to_the_oracle(ctx):
    """The large map's graph: 1000 nodes, 999 odometry and 300 random loop
    edges (minimum-degree ordering, a dense trailing supernode in the factor),
    all 10 Gauss-Newton iterations, against the oracle's dense FP64 solves:
    the chi^2 history iterate by iterate, and the poses at convergence (the
    oracle's last step is below 1e-8)."""
    n = 1000
    g = synth.make_pose_graph(synth.SEED_BASE + 5, n, 300)
    ei, ej, Tij = graph_from_synth(g)
    init = opg.chain_init(n, ei, ej, Tij)
    ref, hist, steps = opg.gauss_newton(init, ei, ej, Tij, iters=10)
    assert steps[-1] < 1e-8 and hist[-1] < hist[0]
    nodes = rows([sim3.identity()] * n)
    chi2 = ctx.pose_graph_correct(nodes, ei, ej, rows(Tij), iters=10)
    assert ctx.sync_status() == 0
    np.testing.assert_allclose(chi2.cpu().numpy(), np.array(hist), rtol=TOL)
    assert_poses_close(tuples(nodes), ref)


@pytest.mark.parametrize("n,loops,seed", [(30, 8, 1), (200, 40, 3)])
def test_levenberg_marquardt_matches_oracle(ctx, n, loops, seed):
    """Adaptive LM (the paper's optimiser) from the chained start: the chi^2
    history (kept and discarded steps alike) and the final poses."""
    g = synth.make_pose_graph(synth.SEED_BASE + seed, n, loops)
    ei, ej, Tij = graph_from_synth(g)
    nodes = rows([sim3.identity()] * n)
    chi2 = ctx.pose_graph_correct(nodes, ei, ej, rows(Tij), iters=10, lm_lambda=1e-3,
                                  lm_adaptive=True)
    assert ctx.sync_status() == 0
    init = opg.chain_init(n, ei, ej, Tij)
    ref, hist, lams = opg.levenberg_marquardt(init, ei, ej, Tij, iters=10, lambda0=1e-3)
    np.testing.assert_allclose(chi2.cpu().numpy(), np.array(hist), rtol=TOL)
    assert_poses_close(tuples(nodes), ref)


def test_levenberg_marquardt_discards_an_overshooting_step(ctx):
    """Strongly inconsistent loops from the identity: the first undamped step
    raises chi^2, is discarded (poses restored, no error) and later damped
    steps are kept, as in the oracle."""
    from test_oracle_pose_graph import random_graph
    rng = np.random.default_rng(32)
    T, ei, ej, Tij = random_graph(rng, 6, 4, noise=0.6)
    nodes = rows([sim3.identity()] * 6)
    chi2 = ctx.pose_graph_correct(nodes, np.array(ei), np.array(ej), rows(Tij), iters=12,
                                  init=False, lm_lambda=1e-6, lm_adaptive=True)
    assert ctx.sync_status() == 0
    ref, hist, _ = opg.levenberg_marquardt([sim3.identity()] * 6, ei, ej, Tij, iters=12,
                                           lambda0=1e-6)
    got = chi2.cpu().numpy()
    assert got[1] == got[0] and got[-1] < got[0]
    np.testing.assert_allclose(got, np.array(hist), rtol=TOL)
    assert_poses_close(tuples(nodes), ref)
