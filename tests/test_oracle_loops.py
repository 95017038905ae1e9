"""Pins of the loop-retrieval oracle (Sec. III-D): bfloat16 rounding, cosine
similarity, the coarse / neighbourhood thresholds and gap rule on
constructed embeddings whose similarities are known in closed form."""
import numpy as np

from oracle import loops


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 0.0],
                 dtype=np.float32)
    r = loops.bf16_round(x)
    # bfloat16 keeps 7 fraction bits: 1 + 2^-8 is a tie (to even: 1), 1 + 3 * 2^-9 rounds up
    np.testing.assert_array_equal(r, np.array([1.0, 1.0, 1.0, 1.0 + 2 ** -7, -2.5, 0.0],
                                              dtype=np.float32))


def test_coarse_similarity_of_orthonormal_and_rotated_embeddings():
    d = 64
    E = np.zeros((6, d), np.float32)
    E[0, 0] = 3.0                      # e0
    E[2, 1] = 0.5                      # e1
    E[4, 0] = E[4, 1] = 1.0            # (e0 + e1) / sqrt 2 after normalising
    S = loops.coarse_similarity(E, 2)  # samples 0, 2, 4
    assert S.shape == (3, 3)
    h = float(loops.bf16_round(np.array([np.float32(1.0) / np.sqrt(np.float32(2.0))]))[0])
    np.testing.assert_array_equal(np.diag(S), [1.0, 1.0, 2 * h * h])
    assert S[0, 1] == 0.0 and S[0, 2] == h and S[1, 2] == h


def test_thresholds_gap_and_best_neighbour():
    """Keyframes on a circle of angles theta_k (unit 2-D embeddings padded with
    zeros): cos similarity = cos(theta_i - theta_j), so every decision is
    known in closed form."""
    theta = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 0.02, 0.31, 0.9, 1.52, 2.3])
    E = np.zeros((len(theta), 8), np.float32)
    E[:, 0], E[:, 1] = np.cos(theta), np.sin(theta)
    coarse, found = loops.loop_candidates(E, stride=1, radius=1, gap=4, tau_global=0.99,
                                          tau_local=0.999)
    want = {(a, b) for a in range(10) for b in range(a + 1, 10)
            if b - a >= 4 and np.cos(theta[a] - theta[b]) > 0.99}
    assert {(a, b) for a, b, _ in coarse} == want
    for a, b, i, j, s in found:
        cands = [(np.cos(theta[p] - theta[q]), -p, -q) for p in range(max(a - 1, 0), min(a + 1, 9) + 1)
                 for q in range(max(b - 1, 0), min(b + 1, 9) + 1) if q - p >= 4]
        best = max(cands)
        assert (i, j) == (-best[1], -best[2]) and abs(s - best[0]) < 1e-6 and s > 0.999
    # (0, 5): theta 0 vs 0.02 -> cos 0.9998 passes both thresholds
    assert any((a, b) == (0, 5) for a, b, *_ in found)


def test_sampled_rows_and_neighbourhood_helpers_agree_with_the_whole_matrix():
    """The row-sampled similarities (for sizes whose matrix is too large) are
    the rows of the whole matrix; the neighbourhood search of one pair
    reproduces the candidates of the full search."""
    rng = np.random.default_rng(4)
    E = rng.normal(size=(90, 64)).astype(np.float32)
    E[42:52] = E[0:10] + 0.05 * rng.normal(size=(10, 64)).astype(np.float32)  # a revisit
    S = loops.coarse_similarity(E, 3)
    rows = [0, 5, S.shape[0] - 1]
    np.testing.assert_array_equal(loops.coarse_similarity_rows(E, 3, rows), S[rows])
    coarse, found = loops.loop_candidates(E, stride=3, radius=1, gap=20, tau_global=0.9,
                                          tau_local=0.95)
    assert found
    En = loops.unit_rows(E)
    for a, b, i, j, s in found:
        assert loops.best_neighbour(En, 3 * a, 3 * b, 1, 20) == (s, i, j)
    # a neighbourhood with no pair far enough apart
    assert loops.best_neighbour(En, 0, 3, 1, 20) == (-np.inf, -1, -1)


def test_exact_cosines_of_scaled_embeddings_on_a_circle():
    """cosine_rows is the cosine itself: embeddings (r_k cos th_k, r_k sin th_k, 0...)
    with arbitrary lengths r_k have cosines cos(th_a - th_b), whatever the
    lengths; the BF16 similarity differs from it by at most the rounding bound
    2u + u^2 (u = 2^-8, unit roundoff of an 8-bit significand) for unit rows."""
    rng = np.random.default_rng(3)
    n, d, stride = 40, 128, 3
    th = rng.uniform(0, 2 * np.pi, n)
    r = rng.uniform(0.1, 30.0, n)
    E = np.zeros((n, d), np.float32)
    E[:, 0] = r * np.cos(th)
    E[:, 1] = r * np.sin(th)
    rows = [0, 4, 13]
    got = loops.cosine_rows(E, stride, rows)
    ths = th[::stride].astype(np.float32).astype(np.float64)
    e32 = E[::stride].astype(np.float64)
    ang = np.arctan2(e32[:, 1], e32[:, 0])
    want = np.cos(ang[rows][:, None] - ang[None, :])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    assert ths.shape[0] == got.shape[1]
    u = 2.0 ** -8
    bf = loops.coarse_similarity_rows(E, stride, rows)
    assert np.abs(bf - got).max() <= 2 * u + u * u
