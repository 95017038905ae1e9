"""ctypes binding of the C-ABI library ``libec3r.so`` (see ``include/ec3r.h``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides device memory and the current stream.  There is no
fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libec3r.so")
_lib = None

OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory",
                4: "capacity exceeded", 5: "not positive definite", 6: "timeout",
                7: "degenerate pair", 8: "workspace growth during capture"}
PAIR_FEW_POINTS, PAIR_ZERO_WEIGHT, PAIR_RANK, PAIR_NONFINITE, PAIR_BAD_INPUT = 1, 2, 4, 8, 16
INJECT_LOOPS_NO_COPY, INJECT_ALIGN_NO_EPOCH = 1, 2
PREC = {"fp32c": 0, "fp64": 1}
RULE = {"product": 0, "src": 1}

# Every symbol include/ec3r.h declares (checked by the CPU tests).
EXPORTS = ("ec3r_create", "ec3r_destroy", "ec3r_last_error", "ec3r_status_string",
           "ec3r_version", "ec3r_sync_status", "ec3r_align_opts_default",
           "ec3r_align_submaps", "ec3r_fuse_points", "ec3r_profile", "ec3r_profile_read",
           "ec3r_align_submaps_noalloc", "ec3r_pg_opts_default", "ec3r_pose_graph_correct",
           "ec3r_align_submaps_backward", "ec3r_align_submaps_depth", "ec3r_correct_points",
           "ec3r_fuse_points_depth", "ec3r_loop_candidates", "ec3r_fuse_count",
           "ec3r_fuse_points_counted", "ec3r_align_token", "ec3r_align_variant_count",
           "ec3r_align_variant_info", "ec3r_align_set_variant", "ec3r_align_last_variant",
           "ec3r_set_wait_limit", "ec3r_inject", "ec3r_align_backward_set_ctas_per_sm")


class Sim3(C.Structure):
    _fields_ = [("s", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3)]


class AlignOpts(C.Structure):
    _fields_ = [("huber_delta", C.c_float), ("iters", C.c_int), ("conf_min", C.c_float),
                ("weight_rule", C.c_int), ("precision", C.c_int), ("want_cost", C.c_int)]


class PgOpts(C.Structure):
    _fields_ = [("iters", C.c_int), ("fixed_node", C.c_int), ("lm_lambda", C.c_double),
                ("init_by_chaining", C.c_int), ("lm_adaptive", C.c_int)]


class LoopOpts(C.Structure):
    _fields_ = [("stride", C.c_int), ("radius", C.c_int), ("gap", C.c_int),
                ("tau_global", C.c_float), ("tau_local", C.c_float)]


class Ec3rError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = C.c_void_p
_I64 = C.c_int64


def _declare(l):
    l.ec3r_create.argtypes = [C.POINTER(_P), C.c_int]
    l.ec3r_destroy.argtypes = [_P]
    l.ec3r_destroy.restype = None
    l.ec3r_last_error.argtypes = [_P]
    l.ec3r_last_error.restype = C.c_char_p
    l.ec3r_status_string.argtypes = [C.c_int]
    l.ec3r_status_string.restype = C.c_char_p
    l.ec3r_version.argtypes = []
    l.ec3r_version.restype = C.c_char_p
    l.ec3r_sync_status.argtypes = [_P, _P]
    l.ec3r_align_opts_default.argtypes = [C.POINTER(AlignOpts)]
    l.ec3r_align_opts_default.restype = None
    l.ec3r_align_submaps.argtypes = [_P, _P, _P, _I64, _I64, C.c_int, _I64, _P, _P, _P, _P,
                                     C.POINTER(AlignOpts), _P, _P, _P, _P]
    l.ec3r_fuse_points.argtypes = [_P, C.c_int, _I64, _P, _P, _P, C.c_float, _I64, _P, _P,
                                   _I64, _P, _P]
    l.ec3r_profile.argtypes = [_P, C.c_int]
    l.ec3r_profile_read.argtypes = [_P, C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int)]
    l.ec3r_align_submaps_backward.argtypes = [_P, _P, _P, _I64, _I64, C.c_int, _I64, _P, _P, _P,
                                              _P, C.POINTER(AlignOpts), C.c_uint64, _P, _P, _P,
                                              _P, _P]
    l.ec3r_align_token.argtypes = [_P]
    l.ec3r_align_token.restype = C.c_uint64
    l.ec3r_align_variant_count.argtypes = []
    l.ec3r_align_variant_count.restype = C.c_int
    l.ec3r_align_variant_info.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int)]
    l.ec3r_align_set_variant.argtypes = [_P, C.c_int]
    l.ec3r_align_last_variant.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_float)]
    l.ec3r_set_wait_limit.argtypes = [_P, C.c_double]
    l.ec3r_inject.argtypes = [_P, C.c_uint]
    l.ec3r_align_backward_set_ctas_per_sm.argtypes = [_P, C.c_int]
    l.ec3r_align_submaps_depth.argtypes = [_P, _P, _P, _P, _I64, C.c_int, C.c_int, C.c_int,
                                           _I64, _P, _P, _P, _P, C.POINTER(AlignOpts), _P, _P,
                                           _P, _P]
    l.ec3r_fuse_points_depth.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P,
                                         _P, C.c_float, _I64, _P, _P, _I64, _P, _P]
    l.ec3r_loop_candidates.argtypes = [_P, _P, C.c_int, C.c_int, C.POINTER(LoopOpts), _P, _I64,
                                       _P, _P, _P]
    l.ec3r_fuse_count.argtypes = [_P, C.c_int, _I64, _P, C.c_float, _P, _P, _P]
    l.ec3r_fuse_points_counted.argtypes = [_P, C.c_int, _I64, _P, _P, _P, _P, _I64, _P, _P,
                                           _I64, _P, _P]
    l.ec3r_correct_points.argtypes = [_P, _I64, _P, _P, C.c_int, _I64, _P, _P, _P, C.c_float,
                                      _P, _P]
    l.ec3r_pg_opts_default.argtypes = [C.POINTER(PgOpts)]
    l.ec3r_pg_opts_default.restype = None
    l.ec3r_pose_graph_correct.argtypes = [_P, C.c_int, _P, C.c_int, _P, _P, _P, _P,
                                          C.POINTER(PgOpts), _P, _P]
    for name in ("ec3r_create", "ec3r_sync_status", "ec3r_align_submaps", "ec3r_fuse_points",
                 "ec3r_profile", "ec3r_profile_read", "ec3r_pose_graph_correct",
                 "ec3r_align_submaps_backward", "ec3r_align_submaps_depth", "ec3r_correct_points",
                 "ec3r_fuse_points_depth", "ec3r_loop_candidates", "ec3r_fuse_count",
                 "ec3r_fuse_points_counted", "ec3r_align_variant_info", "ec3r_align_set_variant",
                 "ec3r_align_last_variant", "ec3r_set_wait_limit", "ec3r_inject",
                 "ec3r_align_backward_set_ctas_per_sm"):
        getattr(l, name).restype = C.c_int


def lib():
    """Load (once) and return the library; raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2510_02080_b300.build`")
        l = C.CDLL(LIB_PATH)
        _declare(l)
        _lib = l
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _want(t, name, dtype, numel=None, at_least=None):
    """Check a tensor's dtype and element count before its pointer crosses the
    C ABI, which sees only the pointer: a mistyped buffer would be misread and a
    short one read or written past its end by the kernels."""
    if t is None:
        return
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    if at_least is not None and t.numel() < at_least:
        raise ValueError(f"{name} needs at least {at_least} elements, has {t.numel()}")


def _want_links(link_off, src, tgt, pair_conf_min, n_pairs):
    _want(link_off, "link_off", torch.int32)
    _want(src, "src", torch.int32)
    _want(tgt, "tgt", torch.int32, numel=int(src.numel()))
    _want(pair_conf_min, "pair_conf_min", torch.float32, at_least=n_pairs)


def _want_outputs(out_xyz, out_idx, cursor):
    _want(out_idx, "out_idx", torch.int64)
    _want(out_xyz, "out_xyz", torch.float32, at_least=3 * int(out_idx.numel()))
    _want(cursor, "cursor", torch.int64, at_least=1)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """Owns an ``ec3r_ctx`` (workspace, cached graphs) on one device."""

    def __init__(self, device=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self._lib = lib()
        h = C.c_void_p()
        st = self._lib.ec3r_create(C.byref(h), dev.index)
        if st != OK:
            raise Ec3rError(st, "ec3r_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ec3r_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise Ec3rError(st, self._lib.ec3r_last_error(self._h).decode())

    def sync_status(self, stream=None):
        """Waits for the stream; returns the status code (0 = ok) of device-side checks."""
        return self._lib.ec3r_sync_status(self._h, _stream(stream))

    def set_wait_limit(self, seconds):
        """Limit of the kernels' bounded waits in seconds (0: the default, 2 s)."""
        self._check(self._lib.ec3r_set_wait_limit(self._h, float(seconds)))

    def set_backward_ctas_per_sm(self, ctas_per_sm):
        """CTAs per SM of the backward call's reduction sweeps (0: one per tile)."""
        self._check(self._lib.ec3r_align_backward_set_ctas_per_sm(self._h, int(ctas_per_sm)))

    def inject(self, what):
        """Test-only: make a bounded wait run out (INJECT_* bits; 0 = off)."""
        self._check(self._lib.ec3r_inject(self._h, int(what)))

    def profile(self, enable=True):
        """Per-kernel CUDA-event timing of every launch (bypasses cached graphs)."""
        self._check(self._lib.ec3r_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kernel: (total_ms, launches)} since the last read; waits for the events."""
        cap, nl = 64, 64
        names = C.create_string_buffer(cap * nl)
        ms = (C.c_double * cap)()
        cnt = (C.c_int64 * cap)()
        n = C.c_int()
        self._check(self._lib.ec3r_profile_read(self._h, cap, names, nl, ms, cnt, C.byref(n)))
        out = {}
        for i in range(min(n.value, cap)):
            nm = names.raw[i * nl:(i + 1) * nl].split(b"\0", 1)[0].decode()
            out[nm] = (ms[i], cnt[i])
        return out

    def last_error(self):
        return self._lib.ec3r_last_error(self._h).decode()

    def align_token(self):
        """Token of the last align_submaps call (0: none); see align_submaps_backward."""
        return int(self._lib.ec3r_align_token(self._h))

    def set_align_variant(self, v):
        """Force registration sweep variant v for later calls (-1: choose by timing)."""
        self._check(self._lib.ec3r_align_set_variant(self._h, int(v)))

    def last_align_variant(self):
        """(variant of the last align_submaps call or -1, {variant: median ms} of its
        size bucket's timing, empty if it was not timed)."""
        v = C.c_int()
        n = align_variant_count()
        ms = (C.c_float * n)()
        self._check(self._lib.ec3r_align_last_variant(self._h, C.byref(v), ms))
        return v.value, {i: float(ms[i]) for i in range(n) if ms[i] >= 0.0}

    # -- registration ------------------------------------------------------
    def align_submaps(self, xyz, conf, link_off, src, tgt, pair_conf_min=None, *, delta=0.02,
                      iters=10, conf_min=0.0, rule="product", precision="fp32c",
                      want_cost=False, out=None, status=None, cost=None, stream=None):
        """Returns (S [n_pairs,13] float64 = (s, R row-major, t), status int32, cost|None)."""
        n_frames, hw = int(conf.shape[0]), int(conf.shape[1])
        if xyz.dtype != torch.float32 or conf.dtype != torch.float32:
            raise ValueError("xyz and conf must be float32")
        if tuple(xyz.shape) != (n_frames, hw, 3):
            raise ValueError("xyz must be [n_frames, hw, 3]")
        n_pairs = int(link_off.numel()) - 1
        _want_links(link_off, src, tgt, pair_conf_min, n_pairs)
        dev = xyz.device
        if out is None:
            out = torch.empty((n_pairs, 13), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty((n_pairs,), dtype=torch.int32, device=dev)
        if want_cost and cost is None:
            cost = torch.empty((n_pairs,), dtype=torch.float64, device=dev)
        _want(out, "out", torch.float64, at_least=13 * n_pairs)
        _want(status, "status", torch.int32, at_least=n_pairs)
        _want(cost if want_cost else None, "cost", torch.float64, at_least=n_pairs)
        o = AlignOpts(float(delta), int(iters), float(conf_min), RULE[rule], PREC[precision],
                      1 if want_cost else 0)
        st = self._lib.ec3r_align_submaps(
            self._h, _ptr(xyz), _ptr(conf), n_frames, hw, n_pairs, int(src.numel()),
            _ptr(link_off), _ptr(src), _ptr(tgt), _ptr(pair_conf_min), C.byref(o), _ptr(out),
            _ptr(status), _ptr(cost) if want_cost else None, _stream(stream))
        self._check(st)
        return out, status, (cost if want_cost else None)

    def align_submaps_depth(self, depth, conf, cams, link_off, src, tgt, pair_conf_min=None, *,
                            delta=0.02, iters=10, conf_min=0.0, rule="product", want_cost=False,
                            out=None, status=None, cost=None, stream=None):
        """Registration from depth [n_frames, H, W] float32, conf (same shape) and cameras
        [n_frames, 16] float32 (fx, fy, cx, cy, R row-major, t: camera -> submap).
        Returns (S [n_pairs,13] float64, status int32, cost|None)."""
        if depth.dim() != 3 or tuple(conf.shape) != tuple(depth.shape):
            raise ValueError("depth and conf must be [n_frames, H, W]")
        n_frames, H, W = (int(v) for v in depth.shape)
        if depth.dtype != torch.float32 or conf.dtype != torch.float32 or \
                cams.dtype != torch.float32:
            raise ValueError("depth, conf and cams must be float32")
        if tuple(cams.shape) != (n_frames, 16):
            raise ValueError("cams must be [n_frames, 16]")
        n_pairs = int(link_off.numel()) - 1
        _want_links(link_off, src, tgt, pair_conf_min, n_pairs)
        dev = depth.device
        if out is None:
            out = torch.empty((n_pairs, 13), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty((n_pairs,), dtype=torch.int32, device=dev)
        if want_cost and cost is None:
            cost = torch.empty((n_pairs,), dtype=torch.float64, device=dev)
        _want(out, "out", torch.float64, at_least=13 * n_pairs)
        _want(status, "status", torch.int32, at_least=n_pairs)
        _want(cost if want_cost else None, "cost", torch.float64, at_least=n_pairs)
        o = AlignOpts(float(delta), int(iters), float(conf_min), RULE[rule], PREC["fp32c"],
                      1 if want_cost else 0)
        st = self._lib.ec3r_align_submaps_depth(
            self._h, _ptr(depth), _ptr(conf), _ptr(cams), n_frames, H, W, n_pairs,
            int(src.numel()), _ptr(link_off), _ptr(src), _ptr(tgt), _ptr(pair_conf_min),
            C.byref(o), _ptr(out), _ptr(status), _ptr(cost) if want_cost else None,
            _stream(stream))
        self._check(st)
        return out, status, (cost if want_cost else None)

    def align_submaps_backward(self, xyz, conf, link_off, src, tgt, grad_S, grad_cost=None,
                               pair_conf_min=None, *, delta=0.02, iters=10, conf_min=0.0,
                               rule="product", fwd_token=0, stream=None):
        """Gradients (dL/dxyz [n_frames,hw,3], dL/dconf [n_frames,hw]) of the registration.

        ``fwd_token`` = 0 runs the forward pass first; the token of the last
        ``align_submaps`` call (``align_token()``) with the same inputs reuses its
        checkpoints, asserting that the inputs were not modified since."""
        n_frames, hw = int(conf.shape[0]), int(conf.shape[1])
        if xyz.dtype != torch.float32 or conf.dtype != torch.float32:
            raise ValueError("xyz and conf must be float32")
        if tuple(xyz.shape) != (n_frames, hw, 3):
            raise ValueError("xyz must be [n_frames, hw, 3]")
        n_pairs = int(link_off.numel()) - 1
        _want_links(link_off, src, tgt, pair_conf_min, n_pairs)
        _want(grad_S, "grad_S", torch.float64, numel=13 * n_pairs)
        _want(grad_cost, "grad_cost", torch.float64, numel=n_pairs)
        gx = torch.empty_like(xyz)
        gc = torch.empty_like(conf)
        o = AlignOpts(float(delta), int(iters), float(conf_min), RULE[rule], PREC["fp32c"], 1)
        st = self._lib.ec3r_align_submaps_backward(
            self._h, _ptr(xyz), _ptr(conf), n_frames, hw, n_pairs, int(src.numel()),
            _ptr(link_off), _ptr(src), _ptr(tgt), _ptr(pair_conf_min), C.byref(o),
            int(fwd_token), _ptr(grad_S.contiguous()),
            _ptr(None if grad_cost is None else grad_cost.contiguous()),
            _ptr(gx), _ptr(gc), _stream(stream))
        self._check(st)
        return gx, gc

    # -- pose graph --------------------------------------------------------
    def pose_graph_correct(self, nodes, ei, ej, Tij, info=None, *, iters=10, fixed=0,
                           lm_lambda=0.0, init=True, chi2=None, lm_adaptive=False,
                           stream=None):
        """Refines ``nodes`` ([n,13] float64, device) in place; returns chi^2 history.

        ``ei``/``ej`` are the edge endpoints on the host (the graph structure is
        planned there); ``Tij`` [m,13] and ``info`` [m,49] live on the device.
        """
        import numpy as np
        hi = np.ascontiguousarray(np.asarray(ei.cpu() if hasattr(ei, "cpu") else ei,
                                             dtype=np.int32))
        hj = np.ascontiguousarray(np.asarray(ej.cpu() if hasattr(ej, "cpu") else ej,
                                             dtype=np.int32))
        n, m = int(nodes.shape[0]), int(hi.shape[0])
        if hi.ndim != 1 or hj.shape != hi.shape:
            raise ValueError("ei and ej must be 1-D and of the same length")
        _want(nodes, "nodes", torch.float64, numel=13 * n)
        _want(Tij, "Tij", torch.float64, at_least=13 * m)
        _want(info, "info", torch.float64, at_least=49 * m)
        if chi2 is None:
            chi2 = torch.empty((iters + 1,), dtype=torch.float64, device=nodes.device)
        _want(chi2, "chi2", torch.float64, at_least=int(iters) + 1)
        o = PgOpts(int(iters), int(fixed), float(lm_lambda), 1 if init else 0,
                   1 if lm_adaptive else 0)
        st = self._lib.ec3r_pose_graph_correct(
            self._h, n, _ptr(nodes), m, hi.ctypes.data_as(C.c_void_p),
            hj.ctypes.data_as(C.c_void_p), _ptr(Tij) if m else None, _ptr(info), C.byref(o),
            _ptr(chi2), _stream(stream))
        self._check(st)
        return chi2

    # -- fusion ------------------------------------------------------------
    def fuse_points(self, xyz, conf, poses, out_xyz, out_idx, cursor, *, threshold=1.0,
                    index_base=0, stream=None):
        """Appends kept points of xyz [M, n, 3] / conf [M, n] at ``cursor`` (int64 [1])."""
        M = int(conf.shape[0])
        n = int(conf.numel() // max(M, 1))
        _want(conf, "conf", torch.float32, numel=M * n)
        _want(xyz, "xyz", torch.float32, numel=3 * M * n)
        _want(poses, "poses", torch.float64, at_least=13 * M)
        _want_outputs(out_xyz, out_idx, cursor)
        st = self._lib.ec3r_fuse_points(
            self._h, M, n, _ptr(xyz), _ptr(conf), _ptr(poses), float(threshold), int(index_base),
            _ptr(out_xyz), _ptr(out_idx), int(out_idx.numel()), _ptr(cursor), _stream(stream))
        self._check(st)


    def fuse_count(self, conf, counts=None, mask=None, *, threshold=1.0, stream=None):
        """Kept points of every 8192-point tile of conf [M, n] and the keep mask
        (int32 counts [n_tiles], int32 mask words [n_tiles * 256], returned);
        the first half of fuse_points, needing no pose."""
        M = int(conf.shape[0])
        n = int(conf.numel() // max(M, 1))
        n_tiles = M * ((n + 8191) // 8192)
        _want(conf, "conf", torch.float32, numel=M * n)
        if counts is None:
            counts = torch.empty((max(n_tiles, 1),), dtype=torch.int32, device=conf.device)
        if mask is None:
            mask = torch.empty((max(n_tiles, 1) * 256,), dtype=torch.int32, device=conf.device)
        if counts.dtype != torch.int32 or counts.numel() < n_tiles:
            raise ValueError(f"counts must be int32 with at least {n_tiles} entries")
        if mask.dtype != torch.int32 or mask.numel() < 256 * n_tiles:
            raise ValueError(f"mask must be int32 with at least {256 * n_tiles} entries")
        st = self._lib.ec3r_fuse_count(self._h, M, n, _ptr(conf), float(threshold),
                                       _ptr(counts), _ptr(mask), _stream(stream))
        self._check(st)
        return counts, mask

    def fuse_points_counted(self, xyz, counts, mask, poses, out_xyz, out_idx, cursor, *,
                            index_base=0, stream=None):
        """fuse_points from the tile counts and keep mask of fuse_count."""
        M = int(xyz.shape[0])
        n = int(xyz.numel() // max(3 * M, 1))
        n_tiles = M * ((n + 8191) // 8192)
        if counts.dtype != torch.int32 or counts.numel() < n_tiles or \
                mask.dtype != torch.int32 or mask.numel() < 256 * n_tiles:
            raise ValueError("counts and mask must be those of fuse_count")
        _want(xyz, "xyz", torch.float32, numel=3 * M * n)
        _want(poses, "poses", torch.float64, at_least=13 * M)
        _want_outputs(out_xyz, out_idx, cursor)
        st = self._lib.ec3r_fuse_points_counted(
            self._h, M, n, _ptr(xyz), _ptr(counts), _ptr(mask), _ptr(poses), int(index_base),
            _ptr(out_xyz), _ptr(out_idx), int(out_idx.numel()), _ptr(cursor), _stream(stream))
        self._check(st)

    def fuse_points_depth(self, depth, conf, cams, poses, out_xyz, out_idx, cursor, *,
                          frames, threshold=1.0, index_base=0, stream=None):
        """Appends kept points of depth / conf [M*frames, H, W] with cameras
        [M*frames, 16] at ``cursor`` (int64 [1])."""
        if depth.dim() != 3 or tuple(conf.shape) != tuple(depth.shape):
            raise ValueError("depth and conf must be [n_frames, H, W]")
        nfr, H, W = (int(v) for v in depth.shape)
        if nfr % frames:
            raise ValueError("the frame count must be a multiple of frames")
        if tuple(cams.shape) != (nfr, 16) or cams.dtype != torch.float32:
            raise ValueError("cams must be float32 [n_frames, 16]")
        _want(depth, "depth", torch.float32)
        _want(conf, "conf", torch.float32)
        _want(poses, "poses", torch.float64, at_least=13 * (nfr // frames))
        _want_outputs(out_xyz, out_idx, cursor)
        st = self._lib.ec3r_fuse_points_depth(
            self._h, nfr // frames, int(frames), H, W, _ptr(depth), _ptr(conf), _ptr(cams),
            _ptr(poses), float(threshold), int(index_base), _ptr(out_xyz), _ptr(out_idx),
            int(out_idx.numel()), _ptr(cursor), _stream(stream))
        self._check(st)

    # -- global loop retrieval ----------------------------------------------
    def loop_candidates(self, emb, *, stride=5, radius=2, gap=50, tau_global=0.93,
                        tau_local=0.96, capacity=1 << 16, with_sim=False, stream=None):
        """Loop candidates of keyframe embeddings emb [n, d] (float32, device).

        Returns (rows int32 [k, 4] = (a, b, i, j), scores float32 [k, 2] =
        (coarse, local), counts int64 [2] = (coarse pairs, candidates), S or None)."""
        n, d = int(emb.shape[0]), int(emb.shape[1])
        if emb.dtype != torch.float32:
            raise ValueError("emb must be float32")
        buf = torch.empty((max(int(capacity), 1), 6), dtype=torch.int32, device=emb.device)
        counts = torch.empty((2,), dtype=torch.int64, device=emb.device)
        m = (n + stride - 1) // stride
        sim = torch.full((m, m), float("nan"), device=emb.device) if with_sim else None
        o = LoopOpts(int(stride), int(radius), int(gap), float(tau_global), float(tau_local))
        st = self._lib.ec3r_loop_candidates(self._h, _ptr(emb), n, d, C.byref(o), _ptr(buf),
                                            int(capacity), _ptr(counts), _ptr(sim),
                                            _stream(stream))
        self._check(st)
        k = min(int(counts[1]), int(capacity))
        return buf[:k, :4], buf[:k, 4:].view(torch.float32), counts, sim

    # -- point correction --------------------------------------------------
    def correct_points(self, points, refs, xyz, conf, poses, *, threshold=1.0, n_corrected=None,
                       stream=None):
        """Sparse-map points [n, 3] (float32, in place) take the global coordinates of
        their referenced submap points (refs int64 [n], -1 = none); xyz [M, n_sub, 3]."""
        M = int(conf.shape[0])
        n = int(conf.numel() // max(M, 1))
        if points.dtype != torch.float32 or refs.dtype != torch.int64:
            raise ValueError("points must be float32 and refs int64")
        _want(points, "points", torch.float32, at_least=3 * int(refs.numel()))
        _want(conf, "conf", torch.float32, numel=M * n)
        _want(xyz, "xyz", torch.float32, numel=3 * M * n)
        _want(poses, "poses", torch.float64, at_least=13 * M)
        _want(n_corrected, "n_corrected", torch.int64, at_least=1)
        st = self._lib.ec3r_correct_points(
            self._h, int(refs.numel()), _ptr(points), _ptr(refs), M, n, _ptr(xyz), _ptr(conf),
            _ptr(poses), float(threshold), _ptr(n_corrected), _stream(stream))
        self._check(st)


def align_variant_count():
    """Number of registration sweep variants (FP32 moments)."""
    return int(lib().ec3r_align_variant_count())


def align_variant_info(v):
    """(pixels per tile, CTAs per SM, persistent: bool) of registration sweep
    variant v (persistent False: one grid per sweep and per solve)."""
    t, c, p = C.c_int(), C.c_int(), C.c_int()
    st = lib().ec3r_align_variant_info(int(v), C.byref(t), C.byref(c), C.byref(p))
    if st != OK:
        raise Ec3rError(st, f"no variant {v}")
    return t.value, c.value, bool(p.value)


def sim3_row(row):
    """(s, R 3x3, t) from one 13-wide row (host numpy)."""
    import numpy as np
    r = np.asarray(row, dtype=np.float64)
    return float(r[0]), r[1:10].reshape(3, 3), r[10:13].copy()


def sim3_rows(S, R, t):
    """Pack float64 tensors s [n], R [n,3,3], t [n,3] into [n,13] rows."""
    return torch.cat([S.reshape(-1, 1), R.reshape(-1, 9), t.reshape(-1, 3)], 1).contiguous()


class EC3RAlign(torch.autograd.Function):
    """Differentiable batched registration: (xyz, conf) -> (S [n,13], cost [n]).

    ``EC3RAlign.apply(ctx, xyz, conf, link_off, src, tgt, pair_conf_min, delta, iters,
    conf_min, rule)``; the backward pass is the library's adjoint
    (``ec3r_align_submaps_backward``).  It reuses the forward call's checkpoints
    when that call is still the context's last registration (its token), else
    it recomputes them; autograd's saved-tensor version check rejects inputs
    modified in place in between.  The returned status and cost tensors are the
    caller's: the backward never reads them.
    """

    @staticmethod
    def forward(fctx, ctx, xyz, conf, link_off, src, tgt, pair_conf_min=None, delta=0.02,
                iters=10, conf_min=0.0, rule="product"):
        S, status, cost = ctx.align_submaps(xyz, conf, link_off, src, tgt, pair_conf_min,
                                            delta=delta, iters=iters, conf_min=conf_min,
                                            rule=rule, want_cost=True)
        fctx.save_for_backward(xyz, conf, link_off, src, tgt, pair_conf_min)
        fctx.ec3r = (ctx, delta, iters, conf_min, rule, ctx.align_token())
        fctx.mark_non_differentiable(status)
        return S, cost, status

    @staticmethod
    def backward(fctx, gS, gcost, _gstatus):
        xyz, conf, link_off, src, tgt, pcm = fctx.saved_tensors
        ctx, delta, iters, conf_min, rule, token = fctx.ec3r
        if token != ctx.align_token():
            token = 0        # another registration ran on this context since
        if gS is None:
            gS = torch.zeros((int(link_off.numel()) - 1, 13), dtype=torch.float64,
                             device=xyz.device)
        gx, gc = ctx.align_submaps_backward(xyz, conf, link_off, src, tgt,
                                            gS.to(torch.float64), gcost, pcm, delta=delta,
                                            iters=iters, conf_min=conf_min, rule=rule,
                                            fwd_token=token)
        return None, gx, gc, None, None, None, None, None, None, None, None
