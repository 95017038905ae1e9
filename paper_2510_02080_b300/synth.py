"""Seeded synthetic workloads shaped like the paper's submaps.

This module only *synthesises inputs*: scenes, camera paths, ray-cast
pointmaps, ground-truth similarity transforms, noise, outliers and
confidences.  It holds none of the registration, pose-graph or fusion
arithmetic, so both the CPU oracle and the CUDA path can read what it makes.

Shapes follow the paper: a submap is the per-pixel pointmap of a few
keyframes with one confidence per pixel, expressed in the frame of its first
camera (Sec. III-C, "Feed-Forward Inference"); five frames per submap
(Sec. IV hyper-parameters, N = 5); images resized so the long side is 518
(Sec. IV "Datasets"); consecutive submaps share the most recent keyframe
(Sec. III-B, "Keyframe Buffer").  The paper's datasets and network outputs
are not available, so ray-cast synthetic scenes stand in for them.

Scene recipe: a 10 m box (six walls) plus 4 random planes and 8 random
spheres (radius 0.2-1.5 m); pinhole cameras with a horizontal field of view
of 60-90 degrees move inside the box; every pixel ray hits a wall.  Each
submap has a random scale in [0.5, 2] (the feed-forward model's scale
ambiguity).  Noise is i.i.d. Gaussian on every coordinate, a fraction of the
pixels are replaced by uniform points of the box, and confidences are
log-normal(0, 0.5).

Generation is deterministic for a given (seed, device): every random draw
comes from one ``torch.Generator`` in a fixed order.  CPU and CUDA generators
produce different streams, so a test generates once and feeds the same
tensors to both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

SEED_BASE = 2510020800
BOX = 10.0
HW_294 = (294, 518)
HW_392 = (392, 518)


# ----------------------------------------------------------------------------
# small helpers (input synthesis only)
# ----------------------------------------------------------------------------
def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(g, shape, lo, hi, device, dtype=torch.float64):
    return lo + (hi - lo) * torch.rand(shape, generator=g, device=device, dtype=dtype)


def _normal(g, shape, device, dtype=torch.float64):
    return torch.randn(shape, generator=g, device=device, dtype=dtype)


def _quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def random_rotation(g, n: int, device) -> torch.Tensor:
    """Haar-uniform rotations: normalised Gaussian quaternions."""
    return _quat_to_rot(_normal(g, (n, 4), device))


def small_rotation(g, n: int, max_angle: float, device) -> torch.Tensor:
    axis = _normal(g, (n, 3), device)
    axis = axis / axis.norm(dim=-1, keepdim=True)
    ang = _uniform(g, (n, 1), -max_angle, max_angle, device)
    q = torch.cat([torch.cos(ang / 2), axis * torch.sin(ang / 2)], -1)
    return _quat_to_rot(q)


@dataclass
class Sim3:
    """A similarity x -> s R x + t in float64 (ground truth bookkeeping)."""
    s: torch.Tensor   # [...]
    R: torch.Tensor   # [..., 3, 3]
    t: torch.Tensor   # [..., 3]

    def to(self, device):
        return Sim3(self.s.to(device), self.R.to(device), self.t.to(device))

    def numpy(self):
        return (self.s.cpu().numpy(), self.R.cpu().numpy(), self.t.cpu().numpy())


def _apply(s, R, t, X):
    """Ground-truth transform of synthetic points (input synthesis)."""
    return s * (X @ R.transpose(-1, -2)) + t


# ----------------------------------------------------------------------------
# scene and ray casting
# ----------------------------------------------------------------------------
@dataclass
class Scene:
    plane_n: torch.Tensor  # [P,3]  n . X = d
    plane_d: torch.Tensor  # [P]
    sph_c: torch.Tensor    # [S,3]
    sph_r: torch.Tensor    # [S]


def make_scene(g, device, n_planes: int = 4, n_spheres: int = 8) -> Scene:
    eye = torch.eye(3, dtype=torch.float64, device=device)
    wall_n = torch.cat([eye, -eye], 0)
    wall_d = torch.cat([torch.zeros(3, dtype=torch.float64, device=device),
                        torch.full((3,), -BOX, dtype=torch.float64, device=device)])
    n = _normal(g, (n_planes, 3), device)
    n = n / n.norm(dim=-1, keepdim=True)
    p0 = _uniform(g, (n_planes, 3), 2.0, 8.0, device)
    d = (n * p0).sum(-1)
    c = _uniform(g, (n_spheres, 3), 1.5, 8.5, device)
    r = _uniform(g, (n_spheres,), 0.2, 1.5, device)
    return Scene(torch.cat([wall_n, n]), torch.cat([wall_d, d]), c, r)


def _clear_of(scene, pos, clearance):
    """True when ``pos`` is at least ``clearance`` from every surface of the scene."""
    if scene is None:
        return True
    if (pos < clearance).any() or (pos > BOX - clearance).any():
        return False
    n_wall = 6
    dp = (scene.plane_n[n_wall:] @ pos - scene.plane_d[n_wall:]).abs()
    if (dp < clearance).any():
        return False
    ds = (scene.sph_c - pos).norm(dim=-1) - scene.sph_r
    return bool((ds.abs() >= clearance).all())


def _view_depth(scene, pos, R):
    """Distance along the optical axis to the first surface."""
    d = R[:, 2]
    nd = scene.plane_n @ d
    tp = (scene.plane_d - scene.plane_n @ pos) / torch.where(nd.abs() < 1e-12,
                                                            torch.full_like(nd, 1e-12), nd)
    tp = torch.where(tp > 1e-6, tp, torch.full_like(tp, float("inf")))
    oc = pos - scene.sph_c
    b = oc @ d
    cc = (oc * oc).sum(-1) - scene.sph_r ** 2
    disc = b * b - cc
    sq = torch.sqrt(torch.clamp(disc, min=0.0))
    ts = torch.where(-b - sq > 1e-6, -b - sq, -b + sq)
    ts = torch.where((disc >= 0) & (ts > 1e-6), ts, torch.full_like(ts, float("inf")))
    return float(torch.minimum(tp.min(), ts.min()))


def camera_path(g, n: int, device, step: float = 0.12, turn_deg: float = 6.0, scene=None,
                clearance: float = 0.8, min_view: float = 1.5):
    """Smooth random walk of camera centres inside the box, with small turns.

    With a scene, every centre keeps ``clearance`` from all surfaces and the
    optical axis meets the first surface at least ``min_view`` away (a
    keyframe never stares at a patch of a few centimetres); a rejected
    proposal is redrawn, up to 50 times, else the camera stays put.
    """
    c = torch.empty(n, 3, dtype=torch.float64, device=device)
    R = torch.empty(n, 3, 3, dtype=torch.float64, device=device)
    pos = _uniform(g, (3,), 3.0, 7.0, device)
    rot = random_rotation(g, 1, device)[0]
    for _ in range(200):
        if _clear_of(scene, pos, clearance) and (scene is None or
                                                 _view_depth(scene, pos, rot) >= min_view):
            break
        pos = _uniform(g, (3,), 1.5, 8.5, device)
        rot = random_rotation(g, 1, device)[0]
    for k in range(n):
        c[k] = pos
        R[k] = rot
        for _ in range(50):
            p2 = torch.clamp(pos + step * _normal(g, (3,), device), 1.0, BOX - 1.0)
            r2 = rot @ small_rotation(g, 1, math.radians(turn_deg), device)[0]
            if scene is None or (_clear_of(scene, p2, clearance)
                                 and _view_depth(scene, p2, r2) >= min_view):
                pos, rot = p2, r2
                break
    return c, R


def hfovs(g, n: int, device):
    return _uniform(g, (n,), math.radians(60.0), math.radians(90.0), device)


def cast_rays(scene: Scene, cam_c, cam_R, hfov, H: int, W: int, dtype=torch.float32):
    """World points hit by every pixel ray of each camera: [n, H*W, 3]."""
    device = cam_c.device
    n = cam_c.shape[0]
    out = torch.empty(n, H * W, 3, dtype=dtype, device=device)
    v, u = torch.meshgrid(torch.arange(H, device=device, dtype=dtype),
                          torch.arange(W, device=device, dtype=dtype), indexing="ij")
    pn, pd = scene.plane_n.to(dtype), scene.plane_d.to(dtype)
    sc, sr = scene.sph_c.to(dtype), scene.sph_r.to(dtype)
    for k in range(n):
        f = (W / 2.0) / math.tan(float(hfov[k]) / 2.0)
        dcam = torch.stack([(u + 0.5 - W / 2.0) / f, (v + 0.5 - H / 2.0) / f,
                            torch.ones_like(u)], -1).reshape(-1, 3)
        d = dcam @ cam_R[k].to(dtype).T                       # [HW,3]
        o = cam_c[k].to(dtype)
        nd = d @ pn.T                                         # [HW,P]
        tp = (pd - pn @ o)[None, :] / torch.where(nd.abs() < 1e-12, torch.full_like(nd, 1e-12), nd)
        tp = torch.where(tp > 1e-6, tp, torch.full_like(tp, float("inf")))
        oc = o[None, :] - sc                                  # [S,3]
        a = (d * d).sum(-1, keepdim=True)                     # [HW,1]
        b = d @ oc.T                                          # [HW,S]
        cc = (oc * oc).sum(-1) - sr * sr                      # [S]
        disc = b * b - a * cc[None, :]
        sq = torch.sqrt(torch.clamp(disc, min=0.0))
        t1 = (-b - sq) / a
        t2 = (-b + sq) / a
        ts = torch.where(t1 > 1e-6, t1, t2)
        ts = torch.where((disc >= 0) & (ts > 1e-6), ts, torch.full_like(ts, float("inf")))
        t = torch.minimum(tp.min(-1).values, ts.min(-1).values)
        out[k] = (o[None, :] + t[:, None] * d).to(dtype)
    return out


def _lognormal_conf(g, shape, device, sigma=0.5):
    return torch.exp(sigma * _normal(g, shape, device, torch.float32))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
@dataclass
class PairSet:
    """Frames plus correspondence links between them.

    ``xyz[n_frames, HW, 3]`` / ``conf[n_frames, HW]`` hold every frame that a
    pair refers to.  Pair ``k`` owns links ``link_off[k]:link_off[k+1]``;
    link ``l`` says that pixel ``i`` of frame ``src[l]`` (a point ``p`` of the
    current submap) corresponds to pixel ``i`` of frame ``tgt[l]`` (its
    counterpart ``q`` in the other submap).
    """
    xyz: torch.Tensor
    conf: torch.Tensor
    link_off: torch.Tensor  # int32 [n_pairs+1]
    src: torch.Tensor       # int32 [n_links]
    tgt: torch.Tensor       # int32 [n_links]
    H: int
    W: int
    S_gt: Sim3 | None = None            # per pair, maps p -> q
    pair_conf_min: torch.Tensor | None = None  # float32 [n_pairs]
    extent: torch.Tensor | None = None  # float64 [n_pairs]: target bbox diagonal
    meta: dict = field(default_factory=dict)

    @property
    def n_pairs(self):
        return int(self.link_off.numel() - 1)

    @property
    def hw(self):
        return self.H * self.W


def make_pair(seed: int, H: int = 294, W: int = 518, sigma: float = 0.005,
              outlier_frac: float = 0.1, device="cpu") -> PairSet:
    """One shared frame: p in camera coordinates, q = S_gt p, both noisy."""
    g = _gen(seed, device)
    scene = make_scene(g, device)
    c, R = camera_path(g, 1, device, scene=scene)
    fov = hfovs(g, 1, device)
    X = cast_rays(scene, c, R, fov, H, W, torch.float64)[0]        # world, float64
    p = (X - c[0]) @ R[0]                                          # camera frame
    s = _uniform(g, (1,), 0.5, 2.0, device)
    Rg = random_rotation(g, 1, device)[0]
    t = _normal(g, (3,), device)
    q = _apply(s, Rg, t, p)
    n = H * W
    p = p + sigma * _normal(g, (n, 3), device)
    q = q + sigma * _normal(g, (n, 3), device)
    out_mask = torch.rand(n, generator=g, device=device) < outlier_frac
    U = _uniform(g, (n, 3), 0.0, BOX, device)
    Uq = _apply(s, Rg, t, (U - c[0]) @ R[0])
    q = torch.where(out_mask[:, None], Uq, q)
    cp = _lognormal_conf(g, (n,), device)
    cq = _lognormal_conf(g, (n,), device)
    xyz = torch.stack([p, q]).to(torch.float32).contiguous()
    conf = torch.stack([cp, cq]).contiguous()
    return PairSet(xyz, conf,
                   torch.tensor([0, 1], dtype=torch.int32, device=device),
                   torch.tensor([0], dtype=torch.int32, device=device),
                   torch.tensor([1], dtype=torch.int32, device=device),
                   H, W, Sim3(s.reshape(1), Rg.reshape(1, 3, 3), t.reshape(1, 3)),
                   meta=dict(kind="pair", sigma=sigma, outlier_frac=outlier_frac, seed=seed))


@dataclass
class Chain:
    """Submaps of ``F`` frames, consecutive submaps sharing one keyframe.

    ``xyz[M, F, HW, 3]`` and ``conf[M, F, HW]`` (float32) are the submaps in
    their own coordinates.  ``T_gt`` maps submap coordinates to the world.
    Pair ``m`` registers submap ``m+1`` (source, frame 0) onto submap ``m``
    (target, frame F-1); its ground truth is ``T_gt[m]^-1 T_gt[m+1]``.
    """
    xyz: torch.Tensor
    conf: torch.Tensor
    T_gt: Sim3
    H: int
    W: int
    F: int
    meta: dict = field(default_factory=dict)

    @property
    def M(self):
        return int(self.xyz.shape[0])

    def pairs(self) -> PairSet:
        M, F = self.M, self.F
        dev = self.xyz.device
        m = torch.arange(M - 1, device=dev, dtype=torch.int32)
        return PairSet(self.xyz.view(M * F, self.H * self.W, 3), self.conf.view(M * F, -1),
                       torch.arange(M, device=dev, dtype=torch.int32),
                       (m + 1) * F, m * F + (F - 1), self.H, self.W,
                       meta=dict(kind="chain"))


def make_chain(seed: int, M: int, F: int = 5, H: int = 294, W: int = 518, sigma: float = 0.01,
               outlier_frac: float = 0.1, device="cpu", cast_dtype=torch.float32) -> Chain:
    g = _gen(seed, device)
    scene = make_scene(g, device)
    K = (F - 1) * M + 1
    cc, cR = camera_path(g, K, device, scene=scene)
    fov = hfovs(g, K, device)
    lam = _uniform(g, (M,), 0.5, 2.0, device)         # world -> submap scale
    n = H * W
    xyz = torch.empty(M, F, n, 3, dtype=torch.float32, device=device)
    conf = torch.empty(M, F, n, dtype=torch.float32, device=device)
    Ts, TR, Tt = 1.0 / lam, cR[0:K:F - 1][:M].clone(), cc[0:K:F - 1][:M].clone()
    for m in range(M):
        kf = torch.arange((F - 1) * m, (F - 1) * m + F, device=device)
        X = cast_rays(scene, cc[kf], cR[kf], fov[kf], H, W, cast_dtype).to(torch.float64)  # [F,n,3]
        x = lam[m] * ((X - Tt[m]) @ TR[m])
        x = x + sigma * _normal(g, (F, n, 3), device)
        om = torch.rand((F, n), generator=g, device=device) < outlier_frac
        U = _uniform(g, (F, n, 3), 0.0, BOX, device)
        xu = lam[m] * ((U - Tt[m]) @ TR[m])
        xyz[m] = torch.where(om[..., None], xu, x).to(torch.float32)
        conf[m] = _lognormal_conf(g, (F, n), device)
    return Chain(xyz, conf, Sim3(Ts, TR, Tt), H, W, F,
                 meta=dict(kind="chain", sigma=sigma, outlier_frac=outlier_frac, seed=seed))


@dataclass
class DepthPairSet:
    """Frames as depth maps with their cameras, plus correspondence links.

    ``depth[n_frames, H, W]`` and ``conf[n_frames, H, W]`` (float32);
    ``cams[n_frames, 16]`` (float32) = (fx, fy, cx, cy, R row-major, t) with
    camera -> submap pose (R, t).  Links as in ``PairSet``.
    """
    depth: torch.Tensor
    conf: torch.Tensor
    cams: torch.Tensor
    link_off: torch.Tensor
    src: torch.Tensor
    tgt: torch.Tensor
    H: int
    W: int
    meta: dict = field(default_factory=dict)

    @property
    def n_pairs(self):
        return int(self.link_off.numel()) - 1


@dataclass
class DepthChain:
    """Submaps of ``F`` frames given as depth maps and cameras, consecutive
    submaps sharing ``overlap`` keyframes (the last ``overlap`` frames of
    submap m are the first ``overlap`` frames of submap m+1).

    Pair ``m`` registers submap ``m+1`` (source) onto submap ``m`` (target)
    through ``overlap`` links; its ground truth is ``T_gt[m]^-1 T_gt[m+1]``.
    """
    depth: torch.Tensor   # [M, F, H, W]
    conf: torch.Tensor    # [M, F, H, W]
    cams: torch.Tensor    # [M, F, 16]
    T_gt: Sim3
    H: int
    W: int
    F: int
    overlap: int
    meta: dict = field(default_factory=dict)

    @property
    def M(self):
        return int(self.depth.shape[0])

    def pairs(self) -> DepthPairSet:
        M, F, ov = self.M, self.F, self.overlap
        dev = self.depth.device
        m = torch.arange(M - 1, device=dev, dtype=torch.int64)
        j = torch.arange(ov, device=dev, dtype=torch.int64)
        src = ((m[:, None] + 1) * F + j[None, :]).reshape(-1).to(torch.int32)
        tgt = (m[:, None] * F + (F - ov) + j[None, :]).reshape(-1).to(torch.int32)
        off = (torch.arange(M, device=dev, dtype=torch.int32) * ov)
        return DepthPairSet(self.depth.view(M * F, self.H, self.W),
                            self.conf.view(M * F, self.H, self.W),
                            self.cams.view(M * F, 16), off, src, tgt, self.H, self.W,
                            meta=dict(kind="depth_chain", overlap=ov))


def make_depth_chain(seed: int, M: int, F: int = 5, H: int = 294, W: int = 518,
                     overlap: int = 1, sigma: float = 0.01, outlier_frac: float = 0.1,
                     device="cpu", cast_dtype=torch.float32) -> DepthChain:
    """Like ``make_chain`` but each frame is a depth map (along the optical
    axis, in submap units) with its pinhole camera and camera -> submap pose.

    Intrinsics: fx = fy = (W/2)/tan(hfov/2), cx = W/2 - 1/2, cy = H/2 - 1/2
    (the ray-casting camera).  Noise is N(0, sigma^2) on the depth; a fraction
    ``outlier_frac`` of the pixels get a depth uniform in (0, 2 x the frame's
    largest depth).
    """
    if not 1 <= overlap < F:
        raise ValueError("need 1 <= overlap < F")
    g = _gen(seed, device)
    scene = make_scene(g, device)
    step = F - overlap
    K = step * M + overlap
    cc, cR = camera_path(g, K, device, scene=scene)
    fov = hfovs(g, K, device)
    lam = _uniform(g, (M,), 0.5, 2.0, device)         # world -> submap scale
    n = H * W
    depth = torch.empty(M, F, H, W, dtype=torch.float32, device=device)
    conf = torch.empty(M, F, H, W, dtype=torch.float32, device=device)
    cams = torch.empty(M, F, 16, dtype=torch.float32, device=device)
    first = torch.arange(M, device=device) * step
    Ts, TR, Tt = 1.0 / lam, cR[first].clone(), cc[first].clone()
    for m in range(M):
        kf = torch.arange(step * m, step * m + F, device=device)
        X = cast_rays(scene, cc[kf], cR[kf], fov[kf], H, W, cast_dtype).to(torch.float64)
        z = torch.einsum("fnk,fk->fn", X - cc[kf][:, None, :], cR[kf][:, :, 2])  # optical axis
        d = lam[m] * z + sigma * _normal(g, (F, n), device)
        om = torch.rand((F, n), generator=g, device=device) < outlier_frac
        du = _uniform(g, (F, n), 0.0, 1.0, device) * 2.0 * d.max(dim=1, keepdim=True).values
        depth[m] = torch.where(om, du, d).to(torch.float32).view(F, H, W)
        conf[m] = _lognormal_conf(g, (F, n), device).view(F, H, W)
        f = (W / 2.0) / torch.tan(fov[kf] / 2.0)
        Rc = TR[m].T[None] @ cR[kf]                                  # camera -> submap
        tc = lam[m] * ((cc[kf] - Tt[m]) @ TR[m])
        cams[m, :, 0] = f.to(torch.float32)
        cams[m, :, 1] = f.to(torch.float32)
        cams[m, :, 2] = W / 2.0 - 0.5
        cams[m, :, 3] = H / 2.0 - 0.5
        cams[m, :, 4:13] = Rc.reshape(F, 9).to(torch.float32)
        cams[m, :, 13:16] = tc.to(torch.float32)
    return DepthChain(depth, conf, cams, Sim3(Ts, TR, Tt), H, W, F, overlap,
                      meta=dict(kind="depth_chain", sigma=sigma, outlier_frac=outlier_frac,
                                seed=seed))


def make_keyframe_embeddings(seed: int, n: int, d: int = 1024, laps: int = 2,
                             spacing: float = 0.1, sigma: float = 0.35, noise: float = 0.15,
                             device="cpu") -> torch.Tensor:
    """Keyframe embeddings of a closed route driven ``laps`` times, one keyframe
    every ``spacing`` metres (float32 [n, d]).

    A keyframe's embedding stands for its image's pooled encoder feature: random
    Fourier features of its place, sqrt(2/d) cos(W p + b) with W ~ N(0, I /
    sigma^2), so two embeddings' cosine is close to exp(-|p - q|^2 / (2 sigma^2)),
    plus N(0, noise^2 / d) per dimension (a noise vector of norm about
    ``noise``, independent of d).  Later laps revisit earlier places with a
    lateral offset drawn per lap, which makes the global loop candidates.
    """
    g = _gen(seed, device)
    length = n * spacing / laps
    radius = length / (2.0 * math.pi)
    k = torch.arange(n, device=device, dtype=torch.float64)
    lap = torch.div(k, n / laps, rounding_mode="floor").clamp(max=laps - 1)
    ang = 2.0 * math.pi * (k * spacing / length)
    off = _uniform(g, (laps,), -0.1, 0.1, device)[lap.long()]
    r = radius + off
    p = torch.stack([r * torch.cos(ang), r * torch.sin(ang), torch.zeros_like(ang)], -1)
    W = _normal(g, (d, 3), device) / sigma
    b = _uniform(g, (d,), 0.0, 2.0 * math.pi, device)
    E = (math.sqrt(2.0 / d) * torch.cos(p @ W.T + b) +
         (noise / math.sqrt(d)) * _normal(g, (n, d), device))
    return E.to(torch.float32)


def chain_pair_truth(chain: Chain) -> Sim3:
    """Ground truth of pair m (submap m+1 -> submap m): T_m^-1 T_{m+1}."""
    s, R, t = chain.T_gt.s, chain.T_gt.R, chain.T_gt.t
    si, Ri, ti = s[:-1], R[:-1], t[:-1]
    sj, Rj, tj = s[1:], R[1:], t[1:]
    RiT = Ri.transpose(-1, -2)
    s_ij = sj / si
    R_ij = RiT @ Rj
    t_ij = ((tj - ti)[:, None, :] @ Ri)[:, 0, :] / si[:, None]
    return Sim3(s_ij, R_ij, t_ij)


def _conf_threshold_for_fraction(frac: torch.Tensor, sigma=0.5) -> torch.Tensor:
    """tau with P(c_p > tau and c_q > tau) = frac for i.i.d. log-normal(0, sigma)."""
    one_side = torch.sqrt(frac.clamp(1e-9, 1.0))
    z = math.sqrt(2.0) * torch.special.erfinv(1.0 - 2.0 * one_side)   # Phi^-1(1 - one_side)
    return torch.exp(sigma * z)


def make_loop_batch(seed: int, n_pairs: int, H: int = 294, W: int = 518, max_frames: int = 5,
                    min_valid: int = 20_000, max_valid: int = 760_000, sigma: float = 0.01,
                    outlier_frac: float = 0.1, device="cpu") -> PairSet:
    """Loop-closure candidates with 1..max_frames shared frames each.

    Each pair has its own scene view and ground truth; its valid count is set
    through a per-pair confidence threshold whose expected valid count is
    U[min_valid, min(max_valid, f*H*W)].
    """
    g = _gen(seed, device)
    scene = make_scene(g, device)
    n = H * W
    nf = torch.randint(1, max_frames + 1, (n_pairs,), generator=g, device=device)
    nf_l = [int(v) for v in nf.tolist()]
    total = sum(nf_l)
    xyz = torch.empty(2 * total, n, 3, dtype=torch.float32, device=device)
    conf = torch.empty(2 * total, n, dtype=torch.float32, device=device)
    s = _uniform(g, (n_pairs,), 0.5, 2.0, device)
    Rg = random_rotation(g, n_pairs, device)
    t = _normal(g, (n_pairs, 3), device)
    hi = torch.clamp(nf.to(torch.float64) * n, max=float(max_valid))
    target = min_valid + (hi - min_valid) * torch.rand(n_pairs, generator=g, device=device,
                                                       dtype=torch.float64)
    frac = target / (nf.to(torch.float64) * n)
    thr = _conf_threshold_for_fraction(frac).to(torch.float32)
    src, tgt, off = [], [], [0]
    fi = 0
    for k in range(n_pairs):
        f = nf_l[k]
        c, R = camera_path(g, f, device, step=0.25, turn_deg=10.0, scene=scene)
        fov = hfovs(g, f, device)
        X = cast_rays(scene, c, R, fov, H, W, torch.float32).to(torch.float64)
        p = (X - c[0]) @ R[0]
        q = _apply(s[k], Rg[k], t[k], p)
        p = p + sigma * _normal(g, (f, n, 3), device)
        q = q + sigma * _normal(g, (f, n, 3), device)
        om = torch.rand((f, n), generator=g, device=device) < outlier_frac
        U = _uniform(g, (f, n, 3), 0.0, BOX, device)
        Uq = _apply(s[k], Rg[k], t[k], (U - c[0]) @ R[0])
        q = torch.where(om[..., None], Uq, q)
        xyz[fi:fi + f] = p.to(torch.float32)
        xyz[fi + f:fi + 2 * f] = q.to(torch.float32)
        conf[fi:fi + 2 * f] = _lognormal_conf(g, (2 * f, n), device)
        src += list(range(fi, fi + f))
        tgt += list(range(fi + f, fi + 2 * f))
        fi += 2 * f
        off.append(off[-1] + f)
    i32 = dict(dtype=torch.int32, device=device)
    return PairSet(xyz, conf, torch.tensor(off, **i32), torch.tensor(src, **i32),
                   torch.tensor(tgt, **i32), H, W, Sim3(s, Rg, t), pair_conf_min=thr,
                   meta=dict(kind="loop_batch", sigma=sigma, outlier_frac=outlier_frac,
                             seed=seed, frames=nf_l, expected_valid=target.tolist()))


# ----------------------------------------------------------------------------
# pose graphs
# ----------------------------------------------------------------------------
@dataclass
class PoseGraphInput:
    T_gt: Sim3              # [n] node poses (submap -> world)
    ei: torch.Tensor        # int32 [m]
    ej: torch.Tensor        # int32 [m]
    T_meas: Sim3            # [m] measured T_ij, noisy
    meta: dict = field(default_factory=dict)


def make_pose_graph(seed: int, n_nodes: int, n_loops: int, min_gap: int = 10,
                    rot_noise: float = 0.01, trans_noise: float = 0.01, scale_noise: float = 0.005,
                    device="cpu") -> PoseGraphInput:
    """Odometry chain i -> i+1 plus random loop edges with |i - j| >= min_gap.

    Node poses follow a random walk; every measured edge is the true relative
    transform T_i^-1 T_j perturbed by a random rotation (angle N(0, rot_noise)),
    translation N(0, trans_noise^2 I) and log-scale N(0, scale_noise^2).
    """
    g = _gen(seed, device)
    c, R = camera_path(g, n_nodes, device, step=0.3, turn_deg=8.0)
    s = torch.exp(0.2 * _normal(g, (n_nodes,), device))
    s[0] = 1.0
    ei = list(range(n_nodes - 1))
    ej = list(range(1, n_nodes))
    seen = set()
    while len(seen) < n_loops:
        a = int(torch.randint(0, n_nodes, (1,), generator=g, device=device))
        b = int(torch.randint(0, n_nodes, (1,), generator=g, device=device))
        i, j = min(a, b), max(a, b)
        if j - i >= min_gap and (i, j) not in seen:
            seen.add((i, j))
            ei.append(i)
            ej.append(j)
    m = len(ei)
    I = torch.tensor(ei, device=device)
    J = torch.tensor(ej, device=device)
    si, Ri, ti = s[I], R[I], c[I]
    sj, Rj, tj = s[J], R[J], c[J]
    s_ij = sj / si
    R_ij = Ri.transpose(-1, -2) @ Rj
    t_ij = ((tj - ti)[:, None, :] @ Ri)[:, 0, :] / si[:, None]
    axis = _normal(g, (m, 3), device)
    axis = axis / axis.norm(dim=-1, keepdim=True)
    ang = rot_noise * _normal(g, (m, 1), device)
    q = torch.cat([torch.cos(ang / 2), axis * torch.sin(ang / 2)], -1)
    R_ij = R_ij @ _quat_to_rot(q)
    t_ij = t_ij + trans_noise * _normal(g, (m, 3), device)
    s_ij = s_ij * torch.exp(scale_noise * _normal(g, (m,), device))
    i32 = dict(dtype=torch.int32, device=device)
    return PoseGraphInput(Sim3(s, R, c), torch.tensor(ei, **i32), torch.tensor(ej, **i32),
                          Sim3(s_ij, R_ij, t_ij), meta=dict(seed=seed, n_loops=n_loops))
