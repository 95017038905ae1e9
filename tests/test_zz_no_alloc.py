"""ec3r_align_submaps_noalloc: registration for callers that may not allocate.

Some callers cannot call cudaMalloc (they run inside a memory arena they do
not own, in a real-time loop where an allocation's implicit synchronisation is
not allowed, or under another framework's allocator).  The no-allocation entry
point keeps its scratch in a fixed device array inside the library.  This test
calls it through the C ABI and checks it against the regular entry point,
ec3r_align_submaps, on two different batches in a row (so a stale scratch
would show), and checks that sizes beyond the fixed scratch are refused.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_02080_b300 import ec3r, synth
from parity import assert_sim3_close

pytestmark = pytest.mark.gpu

MAX_PAIRS = 1024          # EC3R_NOALLOC_MAX_PAIRS


def noalloc_fn():
    l = ec3r.lib()
    f = l.ec3r_align_submaps_noalloc
    P, I64 = C.c_void_p, C.c_int64
    f.argtypes = [P, P, I64, I64, C.c_int, I64, P, P, P, P, C.POINTER(ec3r.AlignOpts), P, P, P,
                  P]
    f.restype = C.c_int
    return f


def call_noalloc(ps, n_pairs=None, **kw):
    f = noalloc_fn()
    n_frames, hw = ps.conf.shape
    n_pairs = ps.n_pairs if n_pairs is None else n_pairs
    out = torch.full((max(n_pairs, 1), 13), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((max(n_pairs, 1),), -1, dtype=torch.int32, device="cuda")
    cost = torch.full((max(n_pairs, 1),), np.nan, dtype=torch.float64, device="cuda")
    o = ec3r.AlignOpts(kw.get("delta", 0.02), kw.get("iters", 10), 0.0, 0,
                       ec3r.PREC[kw.get("precision", "fp32c")], 1)
    pcm = ps.pair_conf_min
    rc = f(ec3r._ptr(ps.xyz), ec3r._ptr(ps.conf), n_frames, hw, n_pairs, int(ps.src.numel()),
           ec3r._ptr(ps.link_off), ec3r._ptr(ps.src), ec3r._ptr(ps.tgt),
           None if pcm is None else ec3r._ptr(pcm), C.byref(o), ec3r._ptr(out), ec3r._ptr(st),
           ec3r._ptr(cost), ec3r._stream(None))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), st.cpu().numpy(), cost.cpu().numpy()


def cuda_set(ps):
    return synth.PairSet(ps.xyz.cuda(), ps.conf.cuda(), ps.link_off.cuda(), ps.src.cuda(),
                         ps.tgt.cuda(), ps.H, ps.W, ps.S_gt,
                         None if ps.pair_conf_min is None else ps.pair_conf_min.cuda())


def target_extent(ps, k):
    lo, hi = int(ps.link_off[k]), int(ps.link_off[k + 1])
    Q = torch.cat([ps.xyz[int(ps.tgt[l])] for l in range(lo, hi)]).double()
    Q = Q[torch.isfinite(Q).all(1)]
    return float((Q.max(0).values - Q.min(0).values).norm())


def compare(ctx, ps, **kw):
    ref_S, ref_st, ref_cost = ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt,
                                                ps.pair_conf_min, want_cost=True, **kw)
    torch.cuda.synchronize()
    rc, S, st, cost = call_noalloc(ps, **kw)
    assert rc == 0
    ref_S, ref_st, ref_cost = ref_S.cpu().numpy(), ref_st.cpu().numpy(), ref_cost.cpu().numpy()
    assert np.array_equal(st, ref_st)
    for k in range(ps.n_pairs):
        if ref_st[k] == 0:
            R = ref_S[k]
            assert_sim3_close(S[k], (R[0], R[1:10].reshape(3, 3), R[10:13]),
                              target_extent(ps, k), f"pair {k}")
            assert abs(cost[k] - ref_cost[k]) <= 1e-5 * ref_cost[k] + 1e-12
        else:
            assert S[k][0] == 1.0


def test_noalloc_matches_regular_entry_point_twice():
    ctx = ec3r.Context()
    # first call: a batch of loop candidates with 1..5 shared frames each
    a = cuda_set(synth.make_loop_batch(synth.SEED_BASE + 3, n_pairs=9, H=60, W=100,
                                       min_valid=500, max_valid=25000))
    compare(ctx, a)
    # second call right after, smaller and different: nothing may leak from the first
    b = cuda_set(synth.make_pair(synth.SEED_BASE + 1, H=100, W=180, sigma=0.005))
    compare(ctx, b)
    compare(ctx, b, precision="fp64", iters=4)
    ctx.close()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    ps = cuda_set(synth.make_pair(synth.SEED_BASE + 5, H=16, W=16))
    big_off = torch.zeros(MAX_PAIRS + 2, dtype=torch.int32, device="cuda")
    big = synth.PairSet(ps.xyz, ps.conf, big_off, ps.src, ps.tgt, ps.H, ps.W)
    rc, *_ = call_noalloc(big, n_pairs=MAX_PAIRS + 1)
    assert rc == 1                      # EC3R_ERR_INVALID_ARG


def test_noalloc_marks_every_pair_of_malformed_offsets():
    """Offsets [0, 3, 2, 5] would let pairs 0 and 2 both claim link 2.  The
    no-allocation entry point has no context to raise an error through, so
    every pair of the call comes back marked EC3R_PAIR_BAD_INPUT (none is
    solved from a link that two pairs claim), and the next call is clean."""
    ps = cuda_set(synth.make_pair(synth.SEED_BASE + 5, H=40, W=60))
    i32 = dict(dtype=torch.int32, device="cuda")
    src, tgt = torch.zeros(5, **i32), torch.ones(5, **i32)
    bad = synth.PairSet(ps.xyz, ps.conf, torch.tensor([0, 3, 2, 5], **i32), src, tgt, ps.H, ps.W)
    rc, S, st, _ = call_noalloc(bad)
    assert rc == 0
    assert st.tolist() == [16, 16, 16]                  # EC3R_PAIR_BAD_INPUT
    assert (S[:, 0] == 1.0).all()
    good = synth.PairSet(ps.xyz, ps.conf, torch.tensor([0, 2, 3, 5], **i32), src, tgt, ps.H,
                         ps.W)
    rc, S, st, _ = call_noalloc(good)
    assert rc == 0 and st.tolist() == [0, 0, 0]
