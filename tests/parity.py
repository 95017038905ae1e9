"""Shared comparison helpers for the GPU parity tests (no method arithmetic
beyond distances between two results)."""
import numpy as np
from scipy.spatial.transform import Rotation

# tolerances of the registration outputs against the FP64 oracle
ROT_TOL = 1e-5        # rad
SCALE_TOL = 1e-6      # relative
TRANS_TOL = 1e-6      # x scene extent (bbox diagonal of the valid targets)


def sim3_errors(row, S_or, extent):
    s, R, t = float(row[0]), np.asarray(row[1:10]).reshape(3, 3), np.asarray(row[10:13])
    so, Ro, to = S_or
    rot = float(np.linalg.norm(Rotation.from_matrix(R @ np.asarray(Ro).T).as_rotvec()))
    return rot, abs(s / so - 1.0), float(np.linalg.norm(t - to)) / max(extent, 1e-30)


def assert_sim3_close(row, S_or, extent, what=""):
    rot, sc, tr = sim3_errors(row, S_or, extent)
    assert rot <= ROT_TOL and sc <= SCALE_TOL and tr <= TRANS_TOL, \
        f"{what}: rot {rot:.2e} scale {sc:.2e} trans/extent {tr:.2e}"
    return rot, sc, tr


def sub_pairset(ps, k):
    """Pair k of a (device) PairSet as a one-pair PairSet on the host: only
    its own frames are copied, so the oracle can recompute sampled pairs of
    batches whose whole frame bank is too large to move."""
    import torch
    from paper_2510_02080_b300 import synth
    lo, hi = int(ps.link_off[k]), int(ps.link_off[k + 1])
    s = ps.src[lo:hi].long()
    t = ps.tgt[lo:hi].long()
    f = hi - lo
    i32 = dict(dtype=torch.int32)
    pcm = None if ps.pair_conf_min is None else ps.pair_conf_min[k:k + 1].cpu()
    return synth.PairSet(torch.cat([ps.xyz[s], ps.xyz[t]]).cpu(),
                         torch.cat([ps.conf[s], ps.conf[t]]).cpu(),
                         torch.tensor([0, f], **i32), torch.arange(f, **i32),
                         torch.arange(f, 2 * f, **i32), ps.H, ps.W, pair_conf_min=pcm)
