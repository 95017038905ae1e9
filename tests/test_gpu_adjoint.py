"""GPU parity of ec3r_align_submaps_backward (the adjoint of the Huber-IRLS
registration) against the FP64 oracle's reverse mode, which is itself pinned to
finite differences (tests/test_oracle_adjoint.py), and directly against FP64
central finite differences (h = 1e-6) of the oracle's forward on a 2k-point
pair.  Loss: Sim(3) geodesic error to the ground truth plus the weighted
residual (lambda = 1).  Points within 1e-4 of the Huber kink at any iteration
are excluded (the loss is not differentiable there).

Tolerance: per gradient array, max |GPU - oracle| <= 2e-3 x max |oracle|
(FP32 per-point arithmetic against FP64)."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import register as reg
from oracle import sim3
from paper_2510_02080_b300 import ec3r, synth

pytestmark = pytest.mark.gpu
DELTA, ITERS = 0.02, 10
RTOL = 2e-3


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def cuda_set(ps):
    return synth.PairSet(ps.xyz.cuda(), ps.conf.cuda(), ps.link_off.cuda(), ps.src.cuda(),
                         ps.tgt.cuda(), ps.H, ps.W, ps.S_gt,
                         None if ps.pair_conf_min is None else ps.pair_conf_min.cuda())


def oracle_grads(ps, S_gt_list, delta=DELTA, iters=ITERS, lam=1.0):
    """Upstream gradient of the geodesic loss at the oracle's estimate, and the
    oracle's FP64 input gradients mapped to the frame bank."""
    xyz = ps.xyz.double().numpy()
    conf = ps.conf.double().numpy()
    lo, src, tgt = ps.link_off.numpy(), ps.src.numpy(), ps.tgt.numpy()
    hw = xyz.shape[1]
    gx = np.zeros_like(xyz)
    gc = np.zeros_like(conf)
    gS = np.zeros((len(lo) - 1, 13))
    kink = np.zeros(xyz.shape[:2], bool)
    for k in range(len(lo) - 1):
        P, Q, cp, cq, valid = reg.pair_correspondences(xyz, conf, lo, src, tgt, k, 0.0)
        w = cp[valid] * cq[valid]
        S, tape, cost = oadj.irls_forward(P[valid], Q[valid], w, delta, iters)
        L, gs, gR, gt = oadj.geodesic_loss_grad(S, S_gt_list[k])
        gS[k] = np.concatenate([[gs], np.asarray(gR).ravel(), gt])
        gP, gQ, gw = oadj.irls_backward(P[valid], Q[valid], w, delta, tape, S, gs, gR, gt, lam)
        gcp, gcq = oadj.weight_grads(gw, cp[valid], cq[valid])
        near = np.zeros(valid.sum(), bool)
        for rec in tape[1:]:
            near |= np.abs(rec["r"] - delta) < 1e-4
        fullP = np.zeros((valid.size, 3)); fullP[valid] = gP
        fullQ = np.zeros((valid.size, 3)); fullQ[valid] = gQ
        fcp = np.zeros(valid.size); fcp[valid] = gcp
        fcq = np.zeros(valid.size); fcq[valid] = gcq
        fnear = np.zeros(valid.size, bool); fnear[valid] = near
        for j, l in enumerate(range(lo[k], lo[k + 1])):
            sl = slice(j * hw, (j + 1) * hw)
            gx[src[l]] += fullP[sl]
            gx[tgt[l]] += fullQ[sl]
            gc[src[l]] += fcp[sl]
            gc[tgt[l]] += fcq[sl]
            kink[src[l]] |= fnear[sl]
            kink[tgt[l]] |= fnear[sl]
    return gS, gx, gc, kink


def compare(g_gpu, g_or, keep, what):
    a = g_gpu[keep]
    b = g_or[keep]
    scale = np.abs(b).max()
    err = np.abs(a - b).max()
    assert err <= RTOL * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e}"
    return err / scale


def truth_list(ps):
    s, R, t = ps.S_gt.numpy()
    return [(float(s[k]), R[k], t[k]) for k in range(len(s))]


@pytest.mark.parametrize("H,W", [(64, 96), (294, 518)])
def test_adjoint_matches_oracle_reverse_mode(ctx, H, W):
    ps = synth.make_pair(synth.SEED_BASE + 4, H=H, W=W, sigma=0.005)
    gS, gx_or, gc_or, kink = oracle_grads(ps, truth_list(ps))
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(1, dtype=torch.float64, device="cuda"))
    gx, gc = gx.cpu().double().numpy(), gc.cpu().double().numpy()
    keep = ~kink
    compare(gx, gx_or, keep, "dL/dxyz")
    compare(gc, gc_or, keep, "dL/dconf")


def test_adjoint_shared_frames_accumulate(ctx):
    """Frame 0 is the source of two pairs: its gradient is the sum of both."""
    a = synth.make_pair(synth.SEED_BASE + 6, H=40, W=60, sigma=0.005)
    b = synth.make_pair(synth.SEED_BASE + 6, H=40, W=60, sigma=0.005, outlier_frac=0.2)
    xyz = torch.stack([a.xyz[0], a.xyz[1], b.xyz[1]])
    conf = torch.stack([a.conf[0], a.conf[1], b.conf[1]])
    i32 = torch.int32
    ps = synth.PairSet(xyz, conf, torch.tensor([0, 1, 2], dtype=i32),
                       torch.tensor([0, 0], dtype=i32), torch.tensor([1, 2], dtype=i32), 40, 60)
    truths = truth_list(a) + truth_list(a)
    gS, gx_or, gc_or, kink = oracle_grads(ps, truths)
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(2, dtype=torch.float64, device="cuda"))
    compare(gx.cpu().double().numpy(), gx_or, ~kink, "dL/dxyz")
    compare(gc.cpu().double().numpy(), gc_or, ~kink, "dL/dconf")


def test_adjoint_against_fp64_finite_differences_2k_subset(ctx):
    """2048-point pair; FP64 central differences of the oracle forward loss."""
    ps = synth.make_pair(synth.SEED_BASE + 8, H=32, W=64, sigma=0.005)
    S_gt = truth_list(ps)[0]
    gS, _, _, kink = oracle_grads(ps, [S_gt])
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(1, dtype=torch.float64, device="cuda"))
    gx, gc = gx.cpu().double().numpy(), gc.cpu().double().numpy()
    xyz = ps.xyz.double().numpy()
    conf = ps.conf.double().numpy()

    def loss(X, Cf):
        S, tape, cost = oadj.irls_forward(X[0], X[1], Cf[0] * Cf[1], DELTA, ITERS)
        return sim3.geodesic_sq(S_gt, S) + cost

    h = 1e-6
    rng = np.random.default_rng(0)
    cand = [i for i in rng.permutation(xyz.shape[1]) if not kink[0, i] and not kink[1, i]]
    scale_x = np.abs(gx).max()
    scale_c = np.abs(gc).max()
    checked = 0
    for i in cand[:8]:
        for f in (0, 1):
            for a in range(3):
                Xp, Xm = xyz.copy(), xyz.copy()
                Xp[f, i, a] += h
                Xm[f, i, a] -= h
                fd = (loss(Xp, conf) - loss(Xm, conf)) / (2 * h)
                assert abs(fd - gx[f, i, a]) <= RTOL * scale_x, (f, i, a, fd, gx[f, i, a])
            Cp, Cm = conf.copy(), conf.copy()
            Cp[f, i] += h
            Cm[f, i] -= h
            fd = (loss(xyz, Cp) - loss(xyz, Cm)) / (2 * h)
            assert abs(fd - gc[f, i]) <= RTOL * scale_c, (f, i, fd, gc[f, i])
            checked += 1
    assert checked >= 12


def test_autograd_function_matches_direct_call(ctx):
    ps = cuda_set(synth.make_pair(synth.SEED_BASE + 9, H=48, W=64, sigma=0.005))
    xyz = ps.xyz.clone().requires_grad_(True)
    conf = ps.conf.clone().requires_grad_(True)
    S, cost, status = ec3r.EC3RAlign.apply(ctx, xyz, conf, ps.link_off, ps.src, ps.tgt)
    w = torch.linspace(-1, 1, 13, dtype=torch.float64, device="cuda")
    loss = (S * w).sum() + 0.5 * cost.sum()
    loss.backward()
    gx, gc = ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt,
                                        w.expand(1, 13).contiguous(),
                                        torch.full((1,), 0.5, dtype=torch.float64, device="cuda"))
    assert torch.equal(xyz.grad, gx) and torch.equal(conf.grad, gc)
    assert int(status[0]) == 0
