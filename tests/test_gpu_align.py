"""GPU parity of ec3r_align_submaps (Sec. III-C, Eq. (sim3), weighted Umeyama
in Huber IRLS) against the FP64 oracle, through the C ABI.

Tolerances: rotation <= 1e-5 rad, scale <= 1e-6 relative, translation <=
1e-6 x scene extent; status codes equal; cost <= 1e-5 relative."""
import numpy as np
import pytest
import torch

from oracle import register as reg
from paper_2510_02080_b300 import ec3r, synth
from parity import assert_sim3_close

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
