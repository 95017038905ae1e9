"""Global loop retrieval over keyframe embeddings: the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. III-D "Loop Retrieval and Verification": a sparse similarity
matrix is built between every N-th keyframe of the database; where two of them
are similar enough (tau_global), their neighbouring keyframes are compared
too, and when the largest similarity of that neighbourhood exceeds
tau_local the pair becomes a loop candidate (the paper then verifies it with a
homography, outside this path).  Sec. IV gives tau_global = 0.93 and
tau_local = 0.96.

Readings where the paper is silent (each also listed in the design notes):

* a keyframe's feature is one embedding vector (the encoder's output pooled
  to one vector); similarity is the cosine of two embeddings;
* the coarse similarities are those of the embeddings normalised in float32
  and rounded to bfloat16 (the precision of the tensor-core contraction),
  with exact products; the neighbourhood similarities are cosines of the
  float32 embeddings;
* sampled keyframes are 0, N, 2N, ...; a coarse pair (a, b) (sample indices,
  a < b) qualifies when its keyframes are at least ``gap`` apart and its
  similarity is strictly above tau_global;
* the neighbourhood of a coarse pair is every keyframe i within ``radius`` of
  a's keyframe and j within ``radius`` of b's keyframe with j - i >= gap; its
  best pair is the largest similarity (ties: smallest i, then j); a coarse
  pair whose best similarity is strictly above tau_local yields the loop
  candidate (a, b, i, j, similarity).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def normalise32(E):
    """Rows divided by their norm, in float32 (sum of squares in float64)."""
    E = np.asarray(E, dtype=np.float32)
    n = np.sqrt(np.sum(E.astype(np.float64) ** 2, axis=1))
    return (E / n[:, None].astype(np.float32)).astype(np.float32)


def coarse_similarity(E, stride):
    """Cosine similarities of the sampled keyframes in the contraction's precision."""
    A = bf16_round(normalise32(np.asarray(E)[::stride])).astype(np.float64)
    return A @ A.T


def coarse_similarity_rows(E, stride, rows):
    """The rows `rows` (sample indices) of coarse_similarity(E, stride), for
    sizes whose whole matrix is too large to form."""
    A = bf16_round(normalise32(np.asarray(E)[::stride])).astype(np.float64)
    return A[np.asarray(rows)] @ A.T


def unit_rows(E):
    """Embeddings normalised in float64 (the neighbourhood similarities)."""
    En = np.asarray(E, dtype=np.float32).astype(np.float64)
    return En / np.linalg.norm(En, axis=1, keepdims=True)


def cosine_rows(E, stride, rows):
    """The exact cosines of the sampled keyframes (the similarity Sec. III-D
    thresholds), rows `rows` (sample indices) against every sample: the
    float32 embeddings taken as they are, everything else in float64.  The
    tensor-core contraction approximates this in BF16 (coarse_similarity_rows
    gives its exact value)."""
    U = unit_rows(np.asarray(E)[::stride])
    return U[np.asarray(rows)] @ U.T


def best_neighbour(En, ka, kb, radius, gap):
    """The neighbourhood search of one coarse pair with keyframes ka < kb over
    unit embeddings En: (best similarity, i, j), ties to the smallest i, then
    j; (-inf, -1, -1) when no pair of the neighbourhood is `gap` apart."""
    n = En.shape[0]
    best = (-np.inf, -1, -1)
    for i in range(max(ka - radius, 0), min(ka + radius, n - 1) + 1):
        for j in range(max(kb - radius, 0), min(kb + radius, n - 1) + 1):
            if j - i < gap:
                continue
            s = float(En[i] @ En[j])
            if s > best[0]:
                best = (s, i, j)
    return best


def loop_candidates(E, stride, radius, gap, tau_global, tau_local):
    """Returns (coarse pairs [(a, b, s)], loops [(a, b, i, j, s)])."""
    E = np.asarray(E, dtype=np.float32)
    S = coarse_similarity(E, stride)
    m = S.shape[0]
    En = unit_rows(E)
    coarse, loops = [], []
    for a in range(m):
        for b in range(a + 1, m):
            ka, kb = a * stride, b * stride
            if kb - ka < gap or not S[a, b] > tau_global:
                continue
            coarse.append((a, b, float(S[a, b])))
            best = best_neighbour(En, ka, kb, radius, gap)
            if best[0] > tau_local:
                loops.append((a, b, best[1], best[2], best[0]))
    return coarse, loops
