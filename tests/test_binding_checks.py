"""Argument checks of the Python binding, on the host (no GPU).

The C ABI receives bare device pointers, so a mistyped or short tensor would
be misread, or read and written past its end, by the kernels.  The binding
checks dtype and size first.  Each case here passes one bad argument and
expects a ValueError that names it.  Each valid call is expected to pass every
check and stop only at the pointer marshalling, which refuses CPU tensors.
Nothing may reach the library: the stub raises if it is called.
"""
import numpy as np
import pytest
import torch

from paper_2510_02080_b300 import ec3r

I32, I64, F32, F64 = torch.int32, torch.int64, torch.float32, torch.float64


class _NoLib:
    def __getattr__(self, name):
        def call(*a, **k):
            raise AssertionError(f"{name} reached the C ABI")
        return call


@pytest.fixture
def ctx():
    c = object.__new__(ec3r.Context)
    c._h = None
    c._lib = _NoLib()
    return c


def passes_checks(fn):
    with pytest.raises(ValueError, match="expected a CUDA tensor"):
        fn()


def registration_args(n_pairs=2, n_frames=4, hw=64):
    return dict(xyz=torch.zeros((n_frames, hw, 3), dtype=F32),
                conf=torch.ones((n_frames, hw), dtype=F32),
                link_off=torch.arange(n_pairs + 1, dtype=I32),
                src=torch.arange(n_pairs, dtype=I32),
                tgt=torch.arange(n_pairs, dtype=I32) + 1)


def test_registration_index_and_output_checks(ctx):
    a = registration_args()
    passes_checks(lambda: ctx.align_submaps(**a))
    for key in ("link_off", "src", "tgt"):
        bad = dict(a, **{key: a[key].to(I64)})
        with pytest.raises(ValueError, match=f"{key} must be torch.int32"):
            ctx.align_submaps(**bad)
    with pytest.raises(ValueError, match="tgt must have 2 elements"):
        ctx.align_submaps(**dict(a, tgt=torch.ones(3, dtype=I32)))
    with pytest.raises(ValueError, match="pair_conf_min needs at least 2"):
        ctx.align_submaps(**a, pair_conf_min=torch.ones(1, dtype=F32))
    with pytest.raises(ValueError, match="out needs at least 26"):
        ctx.align_submaps(**a, out=torch.zeros((1, 13), dtype=F64))
    with pytest.raises(ValueError, match="out must be torch.float64"):
        ctx.align_submaps(**a, out=torch.zeros((2, 13), dtype=F32))
    with pytest.raises(ValueError, match="status needs at least 2"):
        ctx.align_submaps(**a, status=torch.zeros(1, dtype=I32))
    with pytest.raises(ValueError, match="cost needs at least 2"):
        ctx.align_submaps(**a, want_cost=True, cost=torch.zeros(1, dtype=F64))
    # the cost buffer is only checked when the cost is asked for
    passes_checks(lambda: ctx.align_submaps(**a, cost=torch.zeros(1, dtype=F64)))


def test_depth_registration_checks(ctx):
    n_frames, H, W = 3, 4, 8
    base = dict(depth=torch.ones((n_frames, H, W), dtype=F32),
                conf=torch.ones((n_frames, H, W), dtype=F32),
                cams=torch.zeros((n_frames, 16), dtype=F32),
                link_off=torch.tensor([0, 1, 2], dtype=I32),
                src=torch.tensor([0, 1], dtype=I32), tgt=torch.tensor([1, 2], dtype=I32))
    passes_checks(lambda: ctx.align_submaps_depth(**base))
    with pytest.raises(ValueError, match="src must be torch.int32"):
        ctx.align_submaps_depth(**dict(base, src=base["src"].long()))
    with pytest.raises(ValueError, match="status needs at least 2"):
        ctx.align_submaps_depth(**base, status=torch.zeros(1, dtype=I32))


def test_backward_checks(ctx):
    a = registration_args()
    gS, gc = torch.zeros((2, 13), dtype=F64), torch.ones(2, dtype=F64)
    passes_checks(lambda: ctx.align_submaps_backward(**a, grad_S=gS, grad_cost=gc))
    passes_checks(lambda: ctx.align_submaps_backward(**a, grad_S=gS))
    with pytest.raises(ValueError, match="grad_S must have 26"):
        ctx.align_submaps_backward(**a, grad_S=gS[:1], grad_cost=gc)
    with pytest.raises(ValueError, match="grad_S must be torch.float64"):
        ctx.align_submaps_backward(**a, grad_S=gS.float(), grad_cost=gc)
    with pytest.raises(ValueError, match="grad_cost must have 2"):
        ctx.align_submaps_backward(**a, grad_S=gS, grad_cost=gc[:1])
    with pytest.raises(ValueError, match="float32"):
        ctx.align_submaps_backward(**dict(a, xyz=a["xyz"].double()), grad_S=gS)
    with pytest.raises(ValueError, match=r"\[n_frames, hw, 3\]"):
        ctx.align_submaps_backward(**dict(a, xyz=a["xyz"][:, :, :2].contiguous()), grad_S=gS)


def test_pose_graph_checks(ctx):
    n, m = 4, 3
    nodes = torch.zeros((n, 13), dtype=F64)
    ei, ej = np.arange(m), np.arange(m) + 1
    T = torch.zeros((m, 13), dtype=F64)
    passes_checks(lambda: ctx.pose_graph_correct(nodes, ei, ej, T))
    with pytest.raises(ValueError, match="same length"):
        ctx.pose_graph_correct(nodes, ei, ej[:2], T)
    with pytest.raises(ValueError, match="Tij needs at least 39"):
        ctx.pose_graph_correct(nodes, ei, ej, T[:2])
    with pytest.raises(ValueError, match="nodes must be torch.float64"):
        ctx.pose_graph_correct(nodes.float(), ei, ej, T)
    with pytest.raises(ValueError, match="info needs at least 147"):
        ctx.pose_graph_correct(nodes, ei, ej, T, torch.zeros((2, 49), dtype=F64))
    with pytest.raises(ValueError, match="chi2 needs at least 11"):
        ctx.pose_graph_correct(nodes, ei, ej, T, iters=10, chi2=torch.zeros(10, dtype=F64))


def fusion_args(M=2, n=100, cap=50):
    return dict(xyz=torch.zeros((M, n, 3), dtype=F32), conf=torch.ones((M, n), dtype=F32),
                poses=torch.zeros((M, 13), dtype=F64),
                out_xyz=torch.zeros((cap, 3), dtype=F32),
                out_idx=torch.zeros(cap, dtype=I64), cursor=torch.zeros(1, dtype=I64))


def test_fusion_checks(ctx):
    a = fusion_args()
    passes_checks(lambda: ctx.fuse_points(**a))
    with pytest.raises(ValueError, match="out_xyz needs at least 150"):
        ctx.fuse_points(**dict(a, out_xyz=torch.zeros((49, 3), dtype=F32)))
    with pytest.raises(ValueError, match="out_idx must be torch.int64"):
        ctx.fuse_points(**dict(a, out_idx=a["out_idx"].int()))
    with pytest.raises(ValueError, match="cursor must be torch.int64"):
        ctx.fuse_points(**dict(a, cursor=a["cursor"].int()))
    with pytest.raises(ValueError, match="poses must be torch.float64"):
        ctx.fuse_points(**dict(a, poses=a["poses"].float()))
    with pytest.raises(ValueError, match="poses needs at least 26"):
        ctx.fuse_points(**dict(a, poses=a["poses"][:1]))
    with pytest.raises(ValueError, match="xyz must have 600"):
        ctx.fuse_points(**dict(a, xyz=torch.zeros((2, 99, 3), dtype=F32)))
    with pytest.raises(ValueError, match="conf must be torch.float32"):
        ctx.fuse_points(**dict(a, conf=a["conf"].double()))


def test_split_fusion_checks(ctx):
    a = fusion_args()
    passes_checks(lambda: ctx.fuse_count(a["conf"]))
    with pytest.raises(ValueError, match="conf must be torch.float32"):
        ctx.fuse_count(a["conf"].half())
    counts = torch.zeros(2, dtype=I32)
    mask = torch.zeros(512, dtype=I32)
    rest = {k: v for k, v in a.items() if k != "conf"}
    passes_checks(lambda: ctx.fuse_points_counted(counts=counts, mask=mask, **rest))
    with pytest.raises(ValueError, match="out_xyz needs at least 150"):
        ctx.fuse_points_counted(counts=counts, mask=mask,
                                **dict(rest, out_xyz=torch.zeros((10, 3), dtype=F32)))
    with pytest.raises(ValueError, match="poses needs at least 26"):
        ctx.fuse_points_counted(counts=counts, mask=mask, **dict(rest, poses=rest["poses"][:1]))


def test_depth_fusion_checks(ctx):
    nfr, H, W, frames = 4, 4, 8, 2
    a = dict(depth=torch.ones((nfr, H, W), dtype=F32), conf=torch.ones((nfr, H, W), dtype=F32),
             cams=torch.zeros((nfr, 16), dtype=F32), poses=torch.zeros((2, 13), dtype=F64),
             out_xyz=torch.zeros((8, 3), dtype=F32), out_idx=torch.zeros(8, dtype=I64),
             cursor=torch.zeros(1, dtype=I64))
    passes_checks(lambda: ctx.fuse_points_depth(**a, frames=frames))
    with pytest.raises(ValueError, match="poses needs at least 26"):
        ctx.fuse_points_depth(**dict(a, poses=a["poses"][:1]), frames=frames)
    with pytest.raises(ValueError, match="depth must be torch.float32"):
        ctx.fuse_points_depth(**dict(a, depth=a["depth"].double()), frames=frames)


def test_point_correction_checks(ctx):
    M, n, k = 2, 100, 10
    a = dict(points=torch.zeros((k, 3), dtype=F32), refs=torch.zeros(k, dtype=I64),
             xyz=torch.zeros((M, n, 3), dtype=F32), conf=torch.ones((M, n), dtype=F32),
             poses=torch.zeros((M, 13), dtype=F64))
    passes_checks(lambda: ctx.correct_points(**a))
    with pytest.raises(ValueError, match="points needs at least 30"):
        ctx.correct_points(**dict(a, points=torch.zeros((9, 3), dtype=F32)))
    with pytest.raises(ValueError, match="poses needs at least 26"):
        ctx.correct_points(**dict(a, poses=a["poses"][:1]))
    with pytest.raises(ValueError, match="n_corrected must be torch.int64"):
        ctx.correct_points(**a, n_corrected=torch.zeros(1, dtype=I32))
