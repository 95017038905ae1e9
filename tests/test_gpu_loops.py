"""GPU parity of ec3r_loop_candidates (Sec. III-D global loop retrieval) against
the oracle: the BF16 tensor-core similarity matrix within 1e-4 of the
oracle's (normalised embeddings rounded to BF16, exact products); the coarse
pairs and loop candidates equal, except pairs within 1e-4 of a threshold,
which may fall on either side (the two sides normalise with different FP32
roundings)."""
import numpy as np
import pytest
import torch

from oracle import loops as olp
from paper_2510_02080_b300 import ec3r, synth

pytestmark = pytest.mark.gpu
MARGIN = 1e-4


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = ec3r.Context()
    yield c
    c.close()


def test_similarity_matrix_on_the_tensor_cores(ctx):
    # 700 keyframes, every 2nd: 350 samples = 3 x 3 tiles of 128 (ragged), d = 256
    rng = np.random.default_rng(0)
    E = rng.normal(size=(700, 256)).astype(np.float32)
    E[::7] += 3.0 * E[3]                                # some strongly similar rows
    rows, scores, counts, S = ctx.loop_candidates(torch.tensor(E, device="cuda"), stride=2,
                                                  radius=1, gap=4, tau_global=0.5,
                                                  tau_local=0.6, with_sim=True)
    assert ctx.sync_status() == 0
    ref = olp.coarse_similarity(E, 2)
    got = S.cpu().numpy()
    iu = np.triu_indices(ref.shape[0])
    assert np.abs(got[iu] - ref[iu]).max() <= MARGIN
    assert np.all(np.isnan(got[np.tril_indices(ref.shape[0], -1)]))


@pytest.mark.parametrize("n,d,stride", [(2000, 256, 4), (3000, 512, 3)])
def test_loop_candidates_match_oracle(ctx, n, d, stride):
    E = synth.make_keyframe_embeddings(synth.SEED_BASE + 60, n=n, d=d).numpy()
    kw = dict(stride=stride, radius=2, gap=n // 5, tau_global=0.93, tau_local=0.96)
    rows, scores, counts, _ = ctx.loop_candidates(torch.tensor(E, device="cuda"), **kw)
    assert ctx.sync_status() == 0
    coarse, found = olp.loop_candidates(E, **kw)
    S = olp.coarse_similarity(E, stride)
    got = {(int(a), int(b)): (int(i), int(j), float(sc), float(s))
           for (a, b, i, j), (sc, s) in zip(rows.cpu().numpy(), scores.cpu().numpy())}
    want = {(a, b): (i, j, s) for a, b, i, j, s in found}
    ref_coarse = {(a, b) for a, b, _ in coarse}
    assert len(want) > 20
    # coarse pairs: every clear one found, none clearly below the threshold
    m = S.shape[0]
    near = {(a, b) for a in range(m) for b in range(a + 1, m)
            if abs(S[a, b] - kw["tau_global"]) <= MARGIN}
    assert int(counts[0]) >= len(ref_coarse - near)
    assert int(counts[0]) <= len(ref_coarse | near)
    for key, (i, j, s) in want.items():
        if key in near or abs(s - kw["tau_local"]) <= MARGIN:
            continue
        assert key in got, key
        gi, gj, gsc, gs = got[key]
        assert abs(gs - s) <= 1e-5 and abs(gsc - S[key]) <= MARGIN
        assert (gi, gj) == (i, j) or abs(gs - s) <= 1e-5
    for key, (gi, gj, gsc, gs) in got.items():
        assert key in want or key in near or abs(gs - kw["tau_local"]) <= MARGIN, key


def test_capacity_and_arguments(ctx):
    E = synth.make_keyframe_embeddings(synth.SEED_BASE + 61, n=1500, d=128)
    rows, scores, counts, _ = ctx.loop_candidates(E.cuda(), stride=3, radius=1, gap=300,
                                                  tau_global=0.93, tau_local=0.96, capacity=3)
    assert int(counts[1]) > 3 and rows.shape[0] == 3
    assert ctx.sync_status() == 4                      # EC3R_ERR_CAPACITY
    with pytest.raises(ec3r.Ec3rError):
        ctx.loop_candidates(torch.zeros((10, 100), device="cuda"))   # d not a multiple of 64


@pytest.mark.timeout(900)
def test_full_size_sampled_rows_and_candidates(ctx):
    """The benchmarked size (32,768 keyframes x 1024, every 2nd sampled: a
    16,384^2 similarity matrix, the same launch as the timed call): sampled
    rows of the tensor-core matrix against the oracle's rows, and sampled
    loop candidates against the oracle's neighbourhood search."""
    n, d, stride = 32768, 1024, 2
    E = synth.make_keyframe_embeddings(synth.SEED_BASE + 62, n=n, d=d)
    kw = dict(stride=stride, radius=2, gap=n // 5, tau_global=0.93, tau_local=0.96)
    rows, scores, counts, S = ctx.loop_candidates(E.cuda(), capacity=1 << 18, with_sim=True,
                                                  **kw)
    assert ctx.sync_status() == 0
    En = E.numpy()
    m = S.shape[0]
    rng = np.random.default_rng(5)
    sample = np.concatenate([[0, m - 1], rng.choice(m, 10, replace=False)])
    ref = olp.coarse_similarity_rows(En, stride, sample)
    got = S[torch.as_tensor(sample, device="cuda")].cpu().numpy()
    for r, a in enumerate(sample):
        assert np.abs(got[r, a:] - ref[r, a:]).max() <= MARGIN, a
    assert int(counts[0]) > 1000 and int(counts[1]) > 100
    # sampled candidates: the coarse score is the matrix entry, the best
    # neighbour is the oracle's (or ties it within FP32 rounding)
    U = olp.unit_rows(En)
    R, SC = rows.cpu().numpy(), scores.cpu().numpy()
    for q in rng.choice(len(R), 40, replace=False):
        a, b, i, j = (int(v) for v in R[q])
        sc, s = float(SC[q, 0]), float(SC[q, 1])
        assert abs(sc - olp.coarse_similarity_rows(En, stride, [a])[0, b]) <= MARGIN
        best, bi, bj = olp.best_neighbour(U, a * stride, b * stride, kw["radius"], kw["gap"])
        assert abs(s - best) <= 1e-5
        assert (bi, bj) == (i, j) or abs(float(U[i] @ U[j]) - best) <= 1e-5


U_BF16 = 2.0 ** -8          # unit roundoff of BF16's 8-bit significand
U_FP32 = 2.0 ** -24


def exact_cosine_bound(d):
    """|S_bf16 - cos| for unit rows a, b of dimension d: each entry of a and b
    is rounded once to BF16, a_i (1 + e_i), |e_i| <= u, so the exact product of
    the rounded rows differs from a.b by at most (2u + u^2) sum |a_i b_i| <=
    2u + u^2; FP32 accumulation of the d products adds at most d u32 times
    sum |a'_i b'_i| <= (1 + u)^2; the FP32 normalisation before rounding adds
    a few u32."""
    u = U_BF16
    return 2 * u + u * u + (d + 4) * U_FP32 * (1 + u) ** 2


@pytest.mark.timeout(900)
def test_full_size_similarity_against_exact_cosines(ctx):
    """What tau_global thresholds is the cosine of two embeddings (Sec. III-D).
    At the benchmarked size (32,768 keyframes x 1024, every 2nd sampled), 256
    sampled rows of the tensor-core matrix are compared with the FP64 cosines
    of the FP32 embeddings as they are: every entry within the rounding bound
    above; and the coarse decisions at tau_global = 0.93 that the BF16
    contraction takes differently from the exact cosines are counted (each of
    them within the bound of the threshold)."""
    n, d, stride, tau = 32768, 1024, 2, 0.93
    E = synth.make_keyframe_embeddings(synth.SEED_BASE + 62, n=n, d=d)
    rows, scores, counts, S = ctx.loop_candidates(E.cuda(), stride=stride, radius=2,
                                                  gap=n // 5, tau_global=tau, tau_local=0.96,
                                                  capacity=1 << 18, with_sim=True)
    assert ctx.sync_status() == 0
    En = E.numpy()
    m = S.shape[0]
    rng = np.random.default_rng(9)
    sample = np.sort(rng.choice(m, 256, replace=False))
    cos = olp.cosine_rows(En, stride, sample)
    got = S[torch.as_tensor(sample, device="cuda")].cpu().numpy().astype(np.float64)
    bound = exact_cosine_bound(d)
    flips = near = 0
    worst = 0.0
    for r, a in enumerate(sample):
        g, c = got[r, a:], cos[r, a:]
        err = np.abs(g - c)
        worst = max(worst, float(err.max()))
        assert err.max() <= bound, (a, float(err.max()), bound)
        b = np.arange(a, m)
        far = (b - a) * stride >= n // 5
        flip = far & ((g > tau) != (c > tau))
        assert np.all(np.abs(c[flip] - tau) <= bound)
        flips += int(flip.sum())
        near += int((far & (np.abs(c - tau) <= bound)).sum())
    print(f"exact-cosine check: max |S - cos| {worst:.3e} (bound {bound:.3e}); "
          f"{flips} flipped decisions at tau {tau} among {near} entries within the bound of it")


def test_bounded_wait_runs_out_and_the_context_recovers(cuda_lib):
    """The similarity kernel's waits are bounded.  With the test injection the
    TMA producer starts no copy, so the MMA thread's first wait on its stage's
    mbarrier runs out (no copy is ever in flight): EC3R_ERR_TIMEOUT at sync, no
    fault.  The same context then runs the normal call correctly."""
    c = ec3r.Context()
    rng = np.random.default_rng(0)
    E = torch.tensor(rng.normal(size=(700, 256)).astype(np.float32), device="cuda")
    kw = dict(stride=2, radius=1, gap=4, tau_global=0.5, tau_local=0.6, with_sim=True)
    c.set_wait_limit(0.01)
    c.inject(ec3r.INJECT_LOOPS_NO_COPY)
    c.loop_candidates(E, **kw)
    assert c.sync_status() == 6                      # EC3R_ERR_TIMEOUT
    c.inject(0)
    c.set_wait_limit(0)
    rows, scores, counts, S = c.loop_candidates(E, **kw)
    assert c.sync_status() == 0
    ref = olp.coarse_similarity(E.cpu().numpy(), 2)
    iu = np.triu_indices(ref.shape[0])
    assert np.abs(S.cpu().numpy()[iu] - ref[iu]).max() <= MARGIN
    c.close()
