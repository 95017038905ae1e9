"""GPU parity of ec3r_align_submaps_backward (the adjoint of the Huber-IRLS
registration) against the FP64 oracle's reverse mode, which is itself pinned to
finite differences (tests/test_oracle_adjoint.py), and directly against FP64
central finite differences (h = 1e-6) of the oracle's forward on a 2k-point
pair.  Loss: Sim(3) geodesic error to the ground truth plus the weighted
residual (lambda = 1), or a fixed upstream gradient.  Points within 1e-4 of the
Huber kink at any iteration are excluded (the loss is not differentiable
there, and the FP32 and FP64 residuals may take different branches).

Tolerance, element by element: |GPU - oracle| <= A_REL |oracle| + B_ABS
max|oracle| + F32_EST per gradient array.  The GPU evaluates every per-point
gradient in FP32 from the FP32 estimates of the forward (FP32 moments, so S_k
differs from the oracle's by up to ~1e-6 relative) and from moment adjoints
rounded to FP32; each element is a short sum of products whose terms carry
relative errors of a few FP32 roundings (u = 2^-24) amplified by the
conditioning of the 3x3 solves, which A_REL covers; where the terms cancel (a
small gradient of a point whose terms are large), the error is a few roundings
of the terms' scale, which B_ABS covers.

F32_EST: the registration weights iteration k by residuals under S_{k-1} held
in FP32 (the FP32-residual design), and the gradient is far more sensitive to
that estimate than the result is: through the Huber weight's curvature
(d^2 h / dr^2 = 2 delta / r^3 at r ~ delta, against point offsets of metres)
a relative change eps of S_{K-1} moves the gradient by some 10^2 - 10^3 eps
of its largest element (measured on the oracle; the last estimate and the
earlier ones matter far less).  So rounding the estimate to FP32 alone moves
the exact FP64 gradient by up to a few 1e-5 of max|oracle| on the 294x518
pair: the oracle measures this itself, as the difference between its
gradient and that of the same forward with the weighting estimate rounded to
FP32 (oracle.adjoint.irls_forward(estimate_dtype=float32)), and F32_EST is
twice that difference's largest element (the GPU's rounding pattern is not
the model's; the factor covers a different pattern of the same size)."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import register as reg
from oracle import sim3
from paper_2510_02080_b300 import ec3r, synth
from parity import sub_pairset

pytestmark = pytest.mark.gpu
DELTA, ITERS = 0.02, 10
A_REL, B_ABS = 2e-3, 1e-5
F32_FACTOR = 2.0        # F32_EST = F32_FACTOR x the oracle's own FP32-estimate effect
FD_RTOL = 2e-3          # finite differences: h = 1e-6 central differences of FP64


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def cuda_set(ps):
    return synth.PairSet(ps.xyz.cuda(), ps.conf.cuda(), ps.link_off.cuda(), ps.src.cuda(),
                         ps.tgt.cuda(), ps.H, ps.W, ps.S_gt,
                         None if ps.pair_conf_min is None else ps.pair_conf_min.cuda())


def oracle_grads(ps, S_gt_list=None, gS_rows=None, delta=DELTA, iters=ITERS, lam=1.0):
    """The oracle's FP64 input gradients mapped to the frame bank, for the
    upstream gradient of the geodesic loss at the oracle's estimate (S_gt_list)
    or a given one (gS_rows [n_pairs, 13]); dL/dcost = lam.  Also returns the
    upstream rows, the mask of pixels near the Huber kink, and F32_EST per
    array (dict x, c: absolute)."""
    xyz = ps.xyz.double().numpy()
    conf = ps.conf.double().numpy()
    lo, src, tgt = ps.link_off.numpy(), ps.src.numpy(), ps.tgt.numpy()
    hw = xyz.shape[1]
    gx = np.zeros_like(xyz)
    gc = np.zeros_like(conf)
    gx32 = np.zeros_like(xyz)
    gc32 = np.zeros_like(conf)
    gS = np.zeros((len(lo) - 1, 13))
    kink = np.zeros(xyz.shape[:2], bool)
    for k in range(len(lo) - 1):
        P, Q, cp, cq, valid = reg.pair_correspondences(xyz, conf, lo, src, tgt, k, 0.0)
        w = cp[valid] * cq[valid]
        S, tape, cost = oadj.irls_forward(P[valid], Q[valid], w, delta, iters)
        if gS_rows is None:
            L, gs, gR, gt = oadj.geodesic_loss_grad(S, S_gt_list[k])
            gS[k] = np.concatenate([[gs], np.asarray(gR).ravel(), gt])
        else:
            gS[k] = gS_rows[k]
        gs, gR, gt = gS[k][0], gS[k][1:10].reshape(3, 3), gS[k][10:13]
        gP, gQ, gw = oadj.irls_backward(P[valid], Q[valid], w, delta, tape, S, gs, gR, gt, lam)
        gcp, gcq = oadj.weight_grads(gw, cp[valid], cq[valid])
        S32, tape32, _ = oadj.irls_forward(P[valid], Q[valid], w, delta, iters,
                                           estimate_dtype=np.float32)
        gP32, gQ32, gw32 = oadj.irls_backward(P[valid], Q[valid], w, delta, tape32, S32, gs, gR,
                                              gt, lam)
        gcp32, gcq32 = oadj.weight_grads(gw32, cp[valid], cq[valid])
        near = np.zeros(valid.sum(), bool)
        for rec in tape[1:]:
            near |= np.abs(rec["r"] - delta) < 1e-4
        fullP = np.zeros((valid.size, 3)); fullP[valid] = gP
        fullQ = np.zeros((valid.size, 3)); fullQ[valid] = gQ
        fcp = np.zeros(valid.size); fcp[valid] = gcp
        fcq = np.zeros(valid.size); fcq[valid] = gcq
        fnear = np.zeros(valid.size, bool); fnear[valid] = near
        f32 = [np.zeros((valid.size, 3)), np.zeros((valid.size, 3)), np.zeros(valid.size),
               np.zeros(valid.size)]
        for a, v in zip(f32, (gP32, gQ32, gcp32, gcq32)):
            a[valid] = v
        for j, l in enumerate(range(lo[k], lo[k + 1])):
            sl = slice(j * hw, (j + 1) * hw)
            gx[src[l]] += fullP[sl]
            gx[tgt[l]] += fullQ[sl]
            gc[src[l]] += fcp[sl]
            gc[tgt[l]] += fcq[sl]
            gx32[src[l]] += f32[0][sl]
            gx32[tgt[l]] += f32[1][sl]
            gc32[src[l]] += f32[2][sl]
            gc32[tgt[l]] += f32[3][sl]
            kink[src[l]] |= fnear[sl]
            kink[tgt[l]] |= fnear[sl]
    allow = {"x": F32_FACTOR * float(np.abs(gx32 - gx)[~kink].max(initial=0.0)),
             "c": F32_FACTOR * float(np.abs(gc32 - gc)[~kink].max(initial=0.0))}
    return gS, gx, gc, kink, allow


def compare(g_gpu, g_or, keep, what, f32_est):
    """Element-by-element bound; returns the largest error / bound ratio."""
    a = np.asarray(g_gpu)[keep]
    b = np.asarray(g_or)[keep]
    scale = np.abs(b).max()
    err = np.abs(a - b)
    bound = A_REL * np.abs(b) + B_ABS * scale + f32_est
    worst = float((err / bound).max())
    i = int((err / bound).argmax())
    assert worst <= 1.0, (f"{what}: element {i}: |GPU - oracle| {err.ravel()[i]:.3e}, "
                          f"oracle {b.ravel()[i]:.3e}, max|oracle| {scale:.3e}")
    return worst


def truth_list(ps):
    s, R, t = ps.S_gt.numpy()
    return [(float(s[k]), R[k], t[k]) for k in range(len(s))]


@pytest.mark.parametrize("H,W", [(64, 96), (294, 518)])
def test_adjoint_matches_oracle_reverse_mode(ctx, H, W):
    ps = synth.make_pair(synth.SEED_BASE + 4, H=H, W=W, sigma=0.005)
    gS, gx_or, gc_or, kink, allow = oracle_grads(ps, truth_list(ps))
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(1, dtype=torch.float64, device="cuda"))
    gx, gc = gx.cpu().double().numpy(), gc.cpu().double().numpy()
    keep = ~kink
    compare(gx, gx_or, keep, "dL/dxyz", allow["x"])
    compare(gc, gc_or, keep, "dL/dconf", allow["c"])


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
    gS, gx_or, gc_or, kink, allow = oracle_grads(ps, truths)
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(2, dtype=torch.float64, device="cuda"))
    compare(gx.cpu().double().numpy(), gx_or, ~kink, "dL/dxyz", allow["x"])
    compare(gc.cpu().double().numpy(), gc_or, ~kink, "dL/dconf", allow["c"])


def test_adjoint_scalar_path_with_invalid_pixels(ctx):
    """hw = 31 x 39 = 1209, not a multiple of 4: the scalar load paths of the
    forward sweeps and of the backward's reduction sweeps.  Invalid pixels (NaN
    and infinite coordinates, zero and negative confidences) carry the stored
    weight NaN; their gradients are zero and the rest match the oracle's."""
    ps = synth.make_pair(synth.SEED_BASE + 9, H=31, W=39, sigma=0.005)
    xyz, conf = ps.xyz.clone(), ps.conf.clone()
    xyz[0, 7, 1] = float("nan")
    xyz[0, 300, 0] = float("inf")
    xyz[1, 512, 2] = -float("inf")
    conf[0, 40] = 0.0
    conf[1, 41] = -1.0
    conf[1, 1208] = float("nan")
    ps = synth.PairSet(xyz, conf, ps.link_off, ps.src, ps.tgt, ps.H, ps.W, ps.S_gt)
    gS, gx_or, gc_or, kink, allow = oracle_grads(ps, truth_list(ps))
    d = cuda_set(ps)
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(1, dtype=torch.float64, device="cuda"))
    gx, gc = gx.cpu().double().numpy(), gc.cpu().double().numpy()
    for f, i in ((0, 7), (0, 300), (1, 512), (0, 40), (1, 41), (1, 1208)):
        assert np.all(gx[f, i] == 0.0) and gc[f, i] == 0.0, (f, i)
    compare(gx, gx_or, ~kink, "dL/dxyz", allow["x"])
    compare(gc, gc_or, ~kink, "dL/dconf", allow["c"])


@pytest.mark.parametrize("variant", [0, 9, 12])
def test_backward_after_each_forward_schedule(ctx, request, variant):
    """The backward's reduction sweeps read the pixel weights that the forward's
    first sweep stored: by the persistent launch (variants 0 and 9) or by the
    separate-grid schedule (variant 12).  Each forward followed by the backward
    on its token matches the oracle."""
    ps = synth.make_pair(synth.SEED_BASE + 4, H=64, W=96, sigma=0.005)
    gS, gx_or, gc_or, kink, allow = oracle_grads(ps, truth_list(ps))
    d = cuda_set(ps)
    ctx.set_align_variant(variant)
    request.addfinalizer(lambda: ctx.set_align_variant(-1))
    ctx.align_submaps(d.xyz, d.conf, d.link_off, d.src, d.tgt, want_cost=True)
    assert ctx.last_align_variant()[0] == variant
    gx, gc = ctx.align_submaps_backward(d.xyz, d.conf, d.link_off, d.src, d.tgt,
                                        torch.tensor(gS, device="cuda"),
                                        torch.ones(1, dtype=torch.float64, device="cuda"),
                                        fwd_token=ctx.align_token())
    assert ctx.sync_status() == 0
    compare(gx.cpu().double().numpy(), gx_or, ~kink, "dL/dxyz", allow["x"])
    compare(gc.cpu().double().numpy(), gc_or, ~kink, "dL/dconf", allow["c"])


def test_adjoint_against_fp64_finite_differences_2k_subset(ctx):
    """2048-point pair; FP64 central differences of the oracle forward loss."""
    ps = synth.make_pair(synth.SEED_BASE + 8, H=32, W=64, sigma=0.005)
    S_gt = truth_list(ps)[0]
    gS, _, _, kink, _ = oracle_grads(ps, [S_gt])
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
                assert abs(fd - gx[f, i, a]) <= FD_RTOL * scale_x, (f, i, a, fd, gx[f, i, a])
            Cp, Cm = conf.copy(), conf.copy()
            Cp[f, i] += h
            Cm[f, i] -= h
            fd = (loss(xyz, Cp) - loss(xyz, Cm)) / (2 * h)
            assert abs(fd - gc[f, i]) <= FD_RTOL * scale_c, (f, i, fd, gc[f, i])
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


def test_autograd_backward_never_reads_the_forward_outputs(ctx):
    """The status and cost tensors that EC3RAlign.forward returns belong to the
    caller: with both dropped and their memory handed out again and filled
    with junk before backward, the gradients equal those of a direct call."""
    ps = cuda_set(synth.make_pair(synth.SEED_BASE + 9, H=48, W=64, sigma=0.005))
    xyz = ps.xyz.clone().requires_grad_(True)
    conf = ps.conf.clone().requires_grad_(True)
    S, cost, status = ec3r.EC3RAlign.apply(ctx, xyz, conf, ps.link_off, ps.src, ps.tgt)
    w = torch.linspace(-1, 1, 13, dtype=torch.float64, device="cuda")
    loss = (S * w).sum() + 0.5 * cost.sum()
    del S, cost, status
    junk = [torch.full((1,), 7, dtype=torch.int32, device="cuda") for _ in range(16)]
    junk += [torch.full((1,), 1e30, dtype=torch.float64, device="cuda") for _ in range(16)]
    loss.backward()
    gx, gc = ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt,
                                        w.expand(1, 13).contiguous(),
                                        torch.full((1,), 0.5, dtype=torch.float64, device="cuda"))
    assert torch.equal(xyz.grad, gx) and torch.equal(conf.grad, gc)
    assert float(gx.abs().max()) > 0 and len(junk) == 32


def test_autograd_rejects_inputs_modified_in_place(ctx):
    """Inputs rewritten in place between forward and backward: autograd's
    saved-tensor version check refuses the backward."""
    ps = cuda_set(synth.make_pair(synth.SEED_BASE + 9, H=48, W=64, sigma=0.005))
    base = ps.xyz.clone().requires_grad_(True)
    xyz = base * 1.0
    S, cost, status = ec3r.EC3RAlign.apply(ctx, xyz, ps.conf, ps.link_off, ps.src, ps.tgt)
    loss = S.sum()
    with torch.no_grad():
        xyz.mul_(1.01)
    with pytest.raises(RuntimeError, match="modified by an inplace operation"):
        loss.backward()


def test_backward_token_rules(ctx, request):
    """fwd_token = 0 recomputes the checkpoints, so the gradients follow frames
    rewritten in place at the same address; the token of the last forward call
    reuses its checkpoints (bitwise the same gradients); a stale token, or the
    token of a call with other options, is refused before anything runs; a
    forward without the cost sweep serves a backward without a cost gradient.
    Both contexts use one sweep variant (each context's autotuner chooses by
    its own timing, and variants differ at FP32 rounding level)."""
    a = cuda_set(synth.make_pair(synth.SEED_BASE + 9, H=48, W=64, sigma=0.005))
    b = cuda_set(synth.make_pair(synth.SEED_BASE + 10, H=48, W=64, sigma=0.01))
    gS = torch.linspace(-1, 1, 13, dtype=torch.float64, device="cuda").reshape(1, 13)
    gc = torch.ones(1, dtype=torch.float64, device="cuda")
    ctx.set_align_variant(0)
    request.addfinalizer(lambda: ctx.set_align_variant(-1))
    fresh = ec3r.Context()
    fresh.set_align_variant(0)
    gx_b, gc_b = fresh.align_submaps_backward(b.xyz, b.conf, b.link_off, b.src, b.tgt, gS, gc)
    gx_bn, gc_bn = fresh.align_submaps_backward(b.xyz, b.conf, b.link_off, b.src, b.tgt, gS)
    fresh.close()
    xyz, conf = a.xyz.clone(), a.conf.clone()
    links = (a.link_off, a.src, a.tgt)

    def bwd(grad_cost, token):
        return ctx.align_submaps_backward(xyz, conf, *links, gS, grad_cost, fwd_token=token)

    ctx.align_submaps(xyz, conf, *links, want_cost=True)
    assert ctx.align_token() != 0
    xyz.copy_(b.xyz)                      # rewritten in place: same addresses
    conf.copy_(b.conf)
    gx, gcf = bwd(gc, 0)
    assert torch.equal(gx, gx_b) and torch.equal(gcf, gc_b)
    ctx.align_submaps(xyz, conf, *links, want_cost=True)
    tok = ctx.align_token()
    gx, gcf = bwd(gc, tok)
    assert torch.equal(gx, gx_b) and torch.equal(gcf, gc_b)
    ctx.align_submaps(xyz, conf, *links, want_cost=True)
    with pytest.raises(ec3r.Ec3rError):
        bwd(gc, tok)                      # stale: another registration ran since
    ctx.align_submaps(xyz, conf, *links, delta=0.05, want_cost=True)
    with pytest.raises(ec3r.Ec3rError):
        bwd(gc, ctx.align_token())        # that call had another delta
    ctx.align_submaps(xyz, conf, *links)
    with pytest.raises(ec3r.Ec3rError):
        bwd(gc, ctx.align_token())        # no cost sweep, but a cost gradient
    gx, gcf = bwd(None, ctx.align_token())
    assert torch.equal(gx, gx_bn) and torch.equal(gcf, gc_bn)


@pytest.mark.timeout(1800)
def test_chain_adjoint_full_size_sampled_pairs(ctx):
    """The adjoint that is benchmarked: the 200-submap chain at 294 x 518 (199
    pairs, 30 M link pixels) with a fixed upstream gradient for every pair, in
    one backward call; the oracle's reverse mode recomputes sampled pairs.  In
    the chain every frame belongs to one link, so a pair's frame gradients are
    its own."""
    ch = synth.make_chain(synth.SEED_BASE + 2, M=200, F=5, H=294, W=518, device="cuda")
    ps = ch.pairs()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    gS = torch.randn((ps.n_pairs, 13), generator=gen, dtype=torch.float64, device="cuda")
    gcost = torch.ones((ps.n_pairs,), dtype=torch.float64, device="cuda")
    S, st, _ = ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, want_cost=True)
    # the gradient buffers come from the caching allocator: hand it blocks full
    # of NaN first, so that a frame the call fails to write would show
    junk = [torch.full_like(ps.xyz, float("nan")), torch.full_like(ps.conf, float("nan"))]
    del junk
    gx, gc = ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, gS, gcost,
                                        fwd_token=ctx.align_token())
    assert ctx.sync_status() == 0 and int((st != 0).sum()) == 0
    # frames that no link references (three of every five) get exact zeros
    ref = torch.zeros(gc.shape[0], dtype=torch.bool, device="cuda")
    ref[ps.src.long()] = True
    ref[ps.tgt.long()] = True
    assert int((~ref).sum()) > 0
    assert bool((gx[~ref] == 0).all()) and bool((gc[~ref] == 0).all())
    gS_h = gS.cpu().numpy()
    for k in (0, 99, 198):
        fa, fb = int(ps.src[k]), int(ps.tgt[k])
        sub = sub_pairset(ps, k)
        _, gx_or, gc_or, kink, allow = oracle_grads(sub, gS_rows=gS_h[k:k + 1])
        g_x = torch.stack([gx[fa], gx[fb]]).cpu().double().numpy()
        g_c = torch.stack([gc[fa], gc[fb]]).cpu().double().numpy()
        compare(g_x, gx_or, ~kink, f"pair {k} dL/dxyz", allow["x"])
        compare(g_c, gc_or, ~kink, f"pair {k} dL/dconf", allow["c"])


def test_reduction_share_of_sms_bit_identical(ctx, request):
    """ec3r_align_backward_set_ctas_per_sm: the reduction sweeps as 1 or 3 CTAs
    per SM striding over the tiles (a 40-submap chain at 294 x 518: 741 tiles,
    more than either grid) give the same gradients, bit for bit, as one CTA per
    tile; values outside 0..4 are rejected."""
    ch = synth.make_chain(synth.SEED_BASE + 2, M=40, F=5, H=294, W=518, device="cuda")
    ps = ch.pairs()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    gS = torch.randn((ps.n_pairs, 13), generator=gen, dtype=torch.float64, device="cuda")
    gcost = torch.ones((ps.n_pairs,), dtype=torch.float64, device="cuda")
    _, st, _ = ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, want_cost=True)
    tok = ctx.align_token()
    request.addfinalizer(lambda: ctx.set_backward_ctas_per_sm(0))
    out = {}
    for c in (0, 1, 3):
        ctx.set_backward_ctas_per_sm(c)
        gx, gc = ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, gS,
                                            gcost, fwd_token=tok)
        assert ctx.sync_status() == 0
        out[c] = (gx.clone(), gc.clone())
    assert int((st != 0).sum()) == 0
    assert bool(out[0][0].abs().sum() > 0)
    for c in (1, 3):
        assert torch.equal(out[c][0], out[0][0]) and torch.equal(out[c][1], out[0][1])
    lib = ec3r.lib()
    for bad in (-1, 5):
        assert lib.ec3r_align_backward_set_ctas_per_sm(ctx._h, bad) == 1  # EC3R_ERR_INVALID_ARG
