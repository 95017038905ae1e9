"""GPU parity of ec3r_align_submaps (Sec. III-C, Eq. (sim3), weighted Umeyama
in Huber IRLS) against the FP64 oracle, through the C ABI.

Tolerances: rotation <= 1e-5 rad, scale <= 1e-6 relative, translation <=
1e-6 x scene extent; status codes equal; cost <= 1e-5 relative."""
import numpy as np
import pytest
import torch

from oracle import register as reg
from paper_2510_02080_b300 import ec3r, synth
from parity import assert_sim3_close, sub_pairset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def to_cuda(ps):
    out = synth.PairSet(ps.xyz.cuda(), ps.conf.cuda(), ps.link_off.cuda(), ps.src.cuda(),
                        ps.tgt.cuda(), ps.H, ps.W, ps.S_gt,
                        None if ps.pair_conf_min is None else ps.pair_conf_min.cuda(), meta=ps.meta)
    return out


def run(ctx, ps, **kw):
    S, st, cost = ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt,
                                    ps.pair_conf_min, **kw)
    torch.cuda.synchronize()
    return S.cpu().numpy(), st.cpu().numpy(), None if cost is None else cost.cpu().numpy()


def check_against_oracle(ps_cpu, S, st, cost, delta=0.02, iters=10, conf_min=0.0, rule="product"):
    ref = reg.align_pairs(ps_cpu, delta=delta, iters=iters, conf_min=conf_min, rule=rule)
    for k, r in enumerate(ref):
        assert int(st[k]) == r["status"], (k, int(st[k]), r["status"])
        if r["status"] == 0:
            assert_sim3_close(S[k], r["S"], r["extent"], f"pair {k}")
            Rg = S[k][1:10].reshape(3, 3)
            assert np.abs(Rg.T @ Rg - np.eye(3)).max() < 1e-14 and abs(np.linalg.det(Rg) - 1) < 1e-14
            if cost is not None:
                assert abs(cost[k] - r["cost"]) <= 1e-5 * r["cost"] + 1e-12, (k, cost[k], r["cost"])
        else:
            assert S[k][0] == 1.0 and np.abs(S[k][10:]).max() == 0.0
    return ref


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("seed", [0, 1])
def test_single_pair_matches_oracle(ctx, precision, seed):
    # 100 x 180 = 18000 pixels: two full 8192-pixel tiles and a ragged tail
    ps = synth.make_pair(synth.SEED_BASE + 1 + seed, H=100, W=180, sigma=0.005)
    S, st, cost = run(ctx, to_cuda(ps), precision=precision, want_cost=True)
    ref = check_against_oracle(ps, S, st, cost)
    assert ref[0]["status"] == 0


@pytest.mark.parametrize("iters", [1, 3])
def test_iteration_counts_and_delta(ctx, iters):
    ps = synth.make_pair(synth.SEED_BASE + 11, H=64, W=96, sigma=0.01)
    S, st, cost = run(ctx, to_cuda(ps), iters=iters, delta=0.05, want_cost=True)
    check_against_oracle(ps, S, st, cost, delta=0.05, iters=iters)


def test_loop_batch_uneven_links_and_thresholds(ctx):
    ps = synth.make_loop_batch(synth.SEED_BASE + 3, n_pairs=9, H=60, W=100, min_valid=500,
                               max_valid=25000)
    S, st, cost = run(ctx, to_cuda(ps), want_cost=True)
    check_against_oracle(ps, S, st, cost)


def test_chain_pairs_and_src_weight_rule(ctx):
    ch = synth.make_chain(synth.SEED_BASE + 2, M=5, F=3, H=90, W=120)
    ps = ch.pairs()
    S, st, _ = run(ctx, to_cuda(ps), rule="src")
    check_against_oracle(ps, S, st, None, rule="src")


def _custom_set():
    """Edge cases, one pair each: empty, zero confidence, two points, collinear,
    NaN/Inf sprinkled, all outliers, plus a good pair."""
    rng = np.random.default_rng(7)
    hw = 37 * 29           # not a multiple of 4: scalar path
    frames = []
    conf = []

    def add(p, q, cp, cq):
        frames.extend([p, q])
        conf.extend([cp, cq])
        return len(frames) - 2, len(frames) - 1

    base = rng.normal(size=(hw, 3)) * np.array([2.0, 1.5, 1.0]) + 3.0
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    R *= np.sign(np.linalg.det(R))
    good_q = 1.3 * base @ R.T + np.array([0.5, -1.0, 2.0]) + 0.005 * rng.normal(size=(hw, 3))
    ones = rng.lognormal(0, 0.5, hw)
    links = []
    links.append([])                                                   # 0: no link
    links.append([add(base, good_q, np.zeros(hw), ones)])              # 1: zero confidence
    c2 = np.zeros(hw)
    c2[[5, 9]] = 1.0
    links.append([add(base, good_q, c2, ones)])                        # 2: two valid points
    line = np.zeros((hw, 3))
    line[:, 0] = np.arange(hw) * 0.01
    links.append([add(line, line + 1.0, ones, ones)])                  # 3: collinear
    pn = base.copy()
    pn[3, 1] = np.nan
    pn[17, 0] = np.inf
    qn = good_q.copy()
    qn[40, 2] = -np.inf
    cn = ones.copy()
    cn[50] = np.nan
    links.append([add(pn, qn, cn, ones)])                              # 4: NaN / Inf
    links.append([add(base, rng.uniform(-5, 5, (hw, 3)), ones, ones)])  # 5: all outliers
    links.append([add(base, good_q, ones, ones), add(base, good_q, ones, ones)])  # 6: two links
    off = [0]
    src, tgt = [], []
    for L in links:
        for a, b in L:
            src.append(a)
            tgt.append(b)
        off.append(len(src))
    i32 = torch.int32
    return synth.PairSet(torch.tensor(np.stack(frames), dtype=torch.float32),
                         torch.tensor(np.stack(conf), dtype=torch.float32),
                         torch.tensor(off, dtype=i32), torch.tensor(src, dtype=i32),
                         torch.tensor(tgt, dtype=i32), 37, 29)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_edge_cases(ctx, precision):
    ps = _custom_set()
    S, st, cost = run(ctx, to_cuda(ps), precision=precision, want_cost=True)
    ref = check_against_oracle(ps, S, st, cost)
    assert [r["status"] for r in ref] == [reg.DEG_FEW, reg.DEG_FEW, reg.DEG_FEW, reg.DEG_RANK,
                                          0, 0, 0]
    assert ctx.sync_status() == 0


def test_bad_frame_index_is_flagged_not_read(ctx):
    ps = to_cuda(synth.make_pair(synth.SEED_BASE + 5, H=16, W=16))
    bad_tgt = torch.tensor([7], dtype=torch.int32, device="cuda")    # only 2 frames exist
    S, st, _ = ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, bad_tgt)
    assert ctx.sync_status() == 1          # EC3R_ERR_INVALID_ARG
    assert int(st[0]) == ec3r.PAIR_BAD_INPUT
    assert float(S[0, 0]) == 1.0


def test_bad_index_raises_at_sync(ctx):
    ps = to_cuda(synth.make_pair(synth.SEED_BASE + 5, H=16, W=16))
    bad_off = torch.tensor([0, 3], dtype=torch.int32, device="cuda")  # 3 > n_links
    ctx.align_submaps(ps.xyz, ps.conf, bad_off, ps.src, ps.tgt)
    assert ctx.sync_status() == 1
    assert ctx.sync_status() == 0        # the flag was cleared


def test_invalid_arguments_rejected_before_launch(ctx):
    ps = to_cuda(synth.make_pair(synth.SEED_BASE + 5, H=16, W=16))
    with pytest.raises(ec3r.Ec3rError):
        ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, iters=0)
    with pytest.raises(ec3r.Ec3rError):
        ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, delta=-1.0)


def test_deterministic_bitwise(ctx):
    ps = to_cuda(synth.make_loop_batch(synth.SEED_BASE + 4, n_pairs=5, H=50, W=80,
                                       min_valid=300, max_valid=15000))
    a = run(ctx, ps)[0]
    b = run(ctx, ps)[0]
    assert np.array_equal(a, b)


def test_full_size_chain_sampled_pairs(ctx):
    """The 200-submap chain at 294x518 in the benchmark's launch configuration;
    the oracle recomputes a sample of the 199 pairs one by one."""
    ch = synth.make_chain(synth.SEED_BASE + 2, M=200, F=5, H=294, W=518, device="cuda")
    ps = ch.pairs()
    S, st, _ = run(ctx, ps)
    assert (st == 0).all()
    sample = [0, 57, 123, 198]
    for k in sample:
        a, b = int(ps.src[k]), int(ps.tgt[k])
        sub = synth.PairSet(torch.stack([ps.xyz[a], ps.xyz[b]]).cpu(),
                            torch.stack([ps.conf[a], ps.conf[b]]).cpu(),
                            torch.tensor([0, 1], dtype=torch.int32),
                            torch.tensor([0], dtype=torch.int32),
                            torch.tensor([1], dtype=torch.int32), ps.H, ps.W)
        r = reg.align_pairs(sub)[0]
        assert r["status"] == 0
        assert_sim3_close(S[k], r["S"], r["extent"], f"chain pair {k}")


def test_malformed_offsets_mark_every_pair(ctx):
    """Offsets [0, 3, 2, 5] are no CSR array: pairs 0 and 2 would both claim
    link 2 and pair 1 runs backwards.  Every pair of the call is marked (no
    pair is solved from a link that another pair claims), the error is raised
    at sync, and a well-formed call right after is unaffected.  Offsets whose
    last value is not the link count are refused the same way."""
    ps = to_cuda(synth.make_pair(synth.SEED_BASE + 5, H=40, W=60))
    i32 = dict(dtype=torch.int32, device="cuda")
    src, tgt = torch.zeros(5, **i32), torch.ones(5, **i32)
    for off in ([0, 3, 2, 5],          # pairs 0 and 2 share link 2
                [0, 2, 4]):            # the last offset is not the link count (5)
        S, st, _ = ctx.align_submaps(ps.xyz, ps.conf, torch.tensor(off, **i32), src, tgt)
        assert ctx.sync_status() == 1, off
        assert st.tolist() == [ec3r.PAIR_BAD_INPUT] * (len(off) - 1), off
        assert (S[:, 0] == 1.0).all() and (S[:, 10:] == 0.0).all()
    S, st, _ = ctx.align_submaps(ps.xyz, ps.conf, torch.tensor([0, 2, 3, 5], **i32), src, tgt)
    assert ctx.sync_status() == 0 and st.tolist() == [0, 0, 0]


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_config1_pair_at_full_size(ctx, precision):
    """The single-pair configuration at its stated size: one shared 294 x 518
    frame (152,292 points), sigma 0.005, 10 % outliers, delta 0.02, 10
    iterations, in both accumulation modes."""
    ps = synth.make_pair(synth.SEED_BASE + 1, H=294, W=518, sigma=0.005)
    S, st, cost = run(ctx, to_cuda(ps), precision=precision, want_cost=True)
    ref = check_against_oracle(ps, S, st, cost)
    assert ref[0]["status"] == 0


def check_sampled(S, st, cost, ps, sample, what):
    for k in sample:
        r = reg.align_pairs(sub_pairset(ps, k))[0]
        assert int(st[k]) == r["status"], (what, k)
        if r["status"] == 0:
            assert_sim3_close(S[k], r["S"], r["extent"], f"{what} pair {k}")
            if cost is not None:
                assert abs(cost[k] - r["cost"]) <= 1e-5 * r["cost"] + 1e-12, (k, cost[k])


@pytest.mark.timeout(1200)
def test_config3_loop_batch_full_size_sampled_pairs(ctx):
    """512 loop candidates with 1-5 shared 294 x 518 frames each and per-pair
    thresholds for U[20k, 760k] valid points, registered in one call (the
    launch that is benchmarked); the oracle recomputes 12 sampled pairs: the
    first and last, the ones with the most and fewest links, and 8 at random."""
    ps = synth.make_loop_batch(synth.SEED_BASE + 3, n_pairs=512, H=294, W=518, device="cuda")
    S, st, cost = run(ctx, ps, want_cost=True)
    assert ctx.sync_status() == 0 and (st == 0).all()
    frames = np.asarray(ps.meta["frames"])
    rng = np.random.default_rng(3)
    sample = sorted({0, 511, int(frames.argmax()), int(frames.argmin())} |
                    {int(k) for k in rng.choice(512, 8, replace=False)})
    check_sampled(S, st, cost, ps, sample, "loop batch")


@pytest.mark.timeout(1800)
def test_config5_map_registration_sampled_pairs(ctx):
    """The large map at 392 x 518: 1000 submaps of 5 frames, 999 chain pairs
    plus 300 loop pairs (1-5 shared frames) in one call; the oracle recomputes
    sampled chain and loop pairs."""
    M = 1000
    ch = synth.make_chain(synth.SEED_BASE + 5, M=M, F=5, H=392, W=518, device="cuda")
    lb = synth.make_loop_batch(synth.SEED_BASE + 55, n_pairs=300, H=392, W=518,
                               max_valid=760_000, device="cuda")
    cp = ch.pairs()
    del ch
    nf = cp.xyz.shape[0]
    dev = cp.xyz.device
    bank = synth.PairSet(torch.cat([cp.xyz, lb.xyz]), torch.cat([cp.conf, lb.conf]),
                         torch.cat([cp.link_off[:-1], lb.link_off + int(cp.link_off[-1])]),
                         torch.cat([cp.src, lb.src + nf]), torch.cat([cp.tgt, lb.tgt + nf]),
                         392, 518,
                         pair_conf_min=torch.cat([torch.zeros(cp.n_pairs, device=dev),
                                                  lb.pair_conf_min]))
    del cp, lb
    S, st, cost = run(ctx, bank, want_cost=True)
    assert ctx.sync_status() == 0 and (st == 0).all()
    check_sampled(S, st, cost, bank, [0, 500, 998], "map chain")
    rng = np.random.default_rng(55)
    check_sampled(S, st, cost, bank, [999 + int(k) for k in rng.choice(300, 4, replace=False)],
                  "map loop")


def test_persistent_wait_runs_out_and_the_context_recovers(cuda_lib):
    """The persistent registration's waits on a pair's solve are bounded.  With
    the test injection no solve publishes its epoch, so the second sweep's
    waits run out: EC3R_ERR_TIMEOUT at sync, every CTA stops, no fault.  The
    same context then registers the batch correctly."""
    c = ec3r.Context()
    ps = synth.make_loop_batch(synth.SEED_BASE + 4, n_pairs=4, H=50, W=80, min_valid=300,
                               max_valid=15000)
    d = to_cuda(ps)
    c.set_wait_limit(0.005)
    c.inject(ec3r.INJECT_ALIGN_NO_EPOCH)
    run(c, d)
    assert c.sync_status() == 6                      # EC3R_ERR_TIMEOUT
    c.inject(0)
    c.set_wait_limit(0)
    S, st, cost = run(c, d, want_cost=True)
    assert c.sync_status() == 0
    check_against_oracle(ps, S, st, cost)
    c.close()


N_VARIANTS = 13   # ec3r_align_variant_count(): 12 persistent, then separate grids


@pytest.mark.parametrize("v", range(N_VARIANTS))
def test_every_sweep_variant_matches_oracle_and_is_deterministic(ctx, v):
    """Every registration variant (the persistent launch's pixels per tile x
    CTAs per SM, and one grid per sweep and per solve) against the oracle, on a
    batch of 1-5 shared 150 x 240 frames per pair (36,000 pixels: ragged tiles
    of 4096, 8192, 16384 and 32768 pixels) with a degenerate pair; a rerun is
    bitwise identical."""
    assert ec3r.align_variant_count() == N_VARIANTS
    ps = synth.make_loop_batch(synth.SEED_BASE + 4, n_pairs=6, H=150, W=240, min_valid=2000,
                               max_valid=100000)
    xyz = ps.xyz.clone()
    xyz[ps.src[ps.link_off[2]:ps.link_off[3]].long(), :, 1:] = 0.0   # pair 2: collinear
    ps = synth.PairSet(xyz, ps.conf, ps.link_off, ps.src, ps.tgt, ps.H, ps.W, ps.S_gt,
                       ps.pair_conf_min)
    d = to_cuda(ps)
    ctx.set_align_variant(v)
    try:
        S, st, cost = run(ctx, d, want_cost=True)
        S2, st2, cost2 = run(ctx, d, want_cost=True)
        assert ctx.last_align_variant()[0] == v
    finally:
        ctx.set_align_variant(-1)
    assert np.array_equal(S, S2) and np.array_equal(st, st2) and np.array_equal(cost, cost2)
    assert ctx.sync_status() == 0
    ref = check_against_oracle(ps, S, st, cost)
    assert ref[2]["status"] == reg.DEG_RANK and sum(r["status"] == 0 for r in ref) == 5


def test_autotuner_times_each_variant_once_per_size_bucket(cuda_lib):
    """The first call of a size bucket times every variant and keeps the
    fastest; later calls of the bucket reuse it without timing again."""
    c = ec3r.Context()
    d = to_cuda(synth.make_loop_batch(synth.SEED_BASE + 4, n_pairs=5, H=50, W=80,
                                      min_valid=300, max_valid=15000))
    run(c, d)
    v, ms = c.last_align_variant()
    assert sorted(ms) == list(range(ec3r.align_variant_count()))
    assert all(t > 0 for t in ms.values()) and v == min(ms, key=ms.get)
    S1 = run(c, d)[0]
    v2, ms2 = c.last_align_variant()
    assert v2 == v and ms2 == ms
    assert np.array_equal(S1, run(c, d)[0])
    c.close()


def test_zero_sized_calls(ctx):
    """No pair, no submap: the registration writes nothing and succeeds; the
    backward call zeroes the gradients of every frame (each point's gradient is
    zero when no pair uses it); fusion of no submap keeps nothing."""
    xyz = torch.randn((2, 16, 3), device="cuda")
    conf = torch.ones((2, 16), device="cuda")
    lo = torch.zeros(1, dtype=torch.int32, device="cuda")
    none = torch.zeros(0, dtype=torch.int32, device="cuda")
    S, st, cost = ctx.align_submaps(xyz, conf, lo, none, none, want_cost=True)
    assert S.shape == (0, 13) and st.shape == (0,) and cost.shape == (0,)
    gx, gc = ctx.align_submaps_backward(xyz, conf, lo, none, none,
                                        torch.zeros((0, 13), dtype=torch.float64,
                                                    device="cuda"))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert torch.count_nonzero(gx) == 0 and torch.count_nonzero(gc) == 0
    out_xyz = torch.full((4, 3), float("nan"), device="cuda")
    out_idx = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    cursor = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.fuse_points(torch.zeros((0, 16, 3), device="cuda"), torch.zeros((0, 16), device="cuda"),
                    torch.zeros((0, 13), dtype=torch.float64, device="cuda"), out_xyz,
                    out_idx, cursor)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert int(cursor) == 0 and int((out_idx == -7).sum()) == 4
