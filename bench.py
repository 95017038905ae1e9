"""Benchmark of the submap-fusion hot path on synthetic submaps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one "step"): the 200-submap chain (5 frames of 294x518 per submap,
one shared keyframe between consecutive submaps): batched Huber-IRLS
registration of the 199 consecutive pairs (10 solves, FP32 moments, FP64
solve), the FP64 Sim(3) pose graph over the 200 submaps with the 199
registered edges (chaining + 10 Gauss-Newton iterations), and the
confidence > 1 compaction + global transform of all 152,292,000 points under
the corrected poses, then the adjoint of the registration for a fixed
synthetic upstream gradient (the backward pass of a training step).

Metric: Sim(3)-registered points per second per IRLS iteration
(valid correspondences x iterations / step time), whole job over all ranks.
Inputs (2.4 GB per rank) exceed the 126 MB L2, so no flush is needed.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sim(3)-registered points/s per IRLS iter (batched, FP32) and % HBM roofline"
UNIT = "pt-iter/s"
M_SUBMAPS, F_FRAMES, H, W = 200, 5, 294, 518   # the chain workload
ITERS, DELTA = 10, 0.02
PG_ITERS = 10
SEED_CORRECT = 2510020800 + 56
# Algorithmic bytes per link pixel of one Huber-IRLS sweep.  Sweep 1 reads p,
# q (2 x 12 B) and c_p, c_q (2 x 4 B) and writes the pixel's weight (4 B);
# every later sweep (and the final sweep with the cost) reads p, q and that
# weight.
SWEEP1_BYTES_PER_PIXEL = 36
SWEEP_BYTES_PER_PIXEL = 28
# The metric's own count: one correspondence of one iteration read as p, q,
# c_p and c_q.
METRIC_BYTES_PER_PT_ITER = 32
# DRAM bytes (read + write) per link pixel and sweep of the persistent launch
# of sweeps 2 .. 9, by sweep variant: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of that launch on this workload at full size (one-pass
# counters; 199 links x 152,292 px, 8 sweeps).  Variants without a capture of
# this build report null.  Emptied whenever the kernel changes.
REGISTER_TRAFFIC_BYTES_PER_PIXEL_SWEEP = {6: 28.10, 9: 28.07}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands, on a bounded sample
# ----------------------------------------------------------------------------
def _oracle_workload_inproc(name):
    """The oracle timed on a bounded sample of one of the other workloads (one
    thread); returns {"value", "unit", "sample", "seconds"} and, for some,
    further timed parts."""
    import numpy as np
    import torch
    from oracle import adjoint as oadj
    from oracle import fuse as ofuse
    from oracle import loops as olp
    from oracle import pose_graph as opg
    from oracle import register as reg
    from oracle import unproject as oup
    from oracle import sim3 as osim3
    from paper_2510_02080_b300 import synth

    torch.set_num_threads(1)

    def reg_rate(ps):
        t0 = time.perf_counter()
        res = reg.align_pairs(ps, delta=DELTA, iters=ITERS)
        dt = time.perf_counter() - t0
        return sum(r["n_valid"] for r in res) * ITERS / dt, dt

    def pg_iteration_ms(seed, n, loops):
        g = synth.make_pose_graph(seed, n, loops, device="cpu")
        Tij = [(float(g.T_meas.s[k]), g.T_meas.R[k].numpy(), g.T_meas.t[k].numpy())
               for k in range(len(g.ei))]
        ei, ej = g.ei.numpy(), g.ej.numpy()
        init = opg.chain_init(n, ei, ej, Tij)
        t0 = time.perf_counter()
        opg.gauss_newton(init, ei, ej, Tij, iters=1)
        return 1e3 * (time.perf_counter() - t0)

    out = {"unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle"}
    if name == "pair1":
        ps = synth.make_pair(synth.SEED_BASE + 1, H=294, W=518, sigma=0.005, device="cpu")
        rate, dt = reg_rate(ps)
        out.update(value=rate, seconds=dt, sample="the whole pair (FP64 numpy, 10 IRLS solves)")
    elif name == "adjoint1":
        ps = synth.make_pair(synth.SEED_BASE + 4, H=294, W=518, sigma=0.005, device="cpu")
        xyz, conf = ps.xyz.double().numpy(), ps.conf.double().numpy()
        lo, src, tgt = ps.link_off.numpy(), ps.src.numpy(), ps.tgt.numpy()
        P, Q, cp, cq, valid = reg.pair_correspondences(xyz, conf, lo, src, tgt, 0, 0.0)
        w = cp[valid] * cq[valid]
        t0 = time.perf_counter()
        S, tape, cost = oadj.irls_forward(P[valid], Q[valid], w, DELTA, ITERS)
        L, gs, gR, gt = oadj.geodesic_loss_grad(S, osim3.identity())
        oadj.irls_backward(P[valid], Q[valid], w, DELTA, tape, S, gs, gR, gt, 1.0)
        dt = time.perf_counter() - t0
        out.update(value=1e3 * dt, unit="ms per forward + backward", seconds=dt,
                   sample="the whole pair, FP64 numpy reverse mode")
    elif name == "loops512":
        ps = synth.make_loop_batch(synth.SEED_BASE + 3, n_pairs=2, H=294, W=518, device="cpu")
        rate, dt = reg_rate(ps)
        out.update(value=rate, seconds=dt,
                   sample="2 loop pairs of the same recipe (1-5 shared frames, per-pair "
                          "thresholds), 10 IRLS solves",
                   pose_graph_ms_per_iteration=pg_iteration_ms(synth.SEED_BASE + 3, 200, 40))
    elif name == "map1000":
        ch = synth.make_chain(synth.SEED_BASE + 5, M=3, F=5, H=392, W=518, device="cpu")
        rate, dt = reg_rate(ch.pairs())
        xyz = ch.xyz.view(3, -1, 3)[:1].double().numpy()
        conf = ch.conf.view(3, -1)[:1].double().numpy()
        pose = [osim3.identity()]
        t0 = time.perf_counter()
        ofuse.fuse_points(xyz, conf, pose)
        fdt = time.perf_counter() - t0
        out.update(value=rate, seconds=dt,
                   sample="2 chain pairs at 392x518, 10 IRLS solves; fusion of one submap "
                          "(5 x 392 x 518 points); one Gauss-Newton iteration of a "
                          "200-node / 40-loop graph",
                   fusion_points_per_s=xyz.shape[1] / fdt,
                   pose_graph_ms_per_iteration_200_nodes=pg_iteration_ms(
                       synth.SEED_BASE + 3, 200, 40))
    elif name == "pg1000":
        ms = pg_iteration_ms(synth.SEED_BASE + 3, 200, 40)
        out.update(value=ms, unit="ms per Gauss-Newton iteration", seconds=ms * 1e-3,
                   sample="one Gauss-Newton iteration of a 200-node / 40-loop graph (the "
                          "1000-node graph's dense FP64 normal equations would take minutes)")
    elif name == "depth200":
        ch = synth.make_depth_chain(synth.SEED_BASE + 46, M=3, F=5, H=294, W=518, device="cpu")
        dps = ch.pairs()
        t0 = time.perf_counter()
        xyz = oup.unproject(dps.depth.double().numpy(), dps.cams.numpy())
        dt_un = time.perf_counter() - t0
        nf, H_, W_ = dps.depth.shape
        ps = synth.PairSet(torch.as_tensor(xyz, dtype=torch.float32),
                           dps.conf.reshape(nf, H_ * W_), dps.link_off, dps.src, dps.tgt, H_, W_)
        rate, dt = reg_rate(ps)
        out.update(value=rate * dt / (dt + dt_un), seconds=dt + dt_un,
                   sample="2 depth pairs: FP64 unprojection of their frames, then 10 IRLS "
                          "solves")
    elif name == "loops32k":
        E = synth.make_keyframe_embeddings(synth.SEED_BASE + 62, n=32768, d=1024).numpy()
        rows = np.arange(0, 16384, 128)
        t0 = time.perf_counter()
        olp.coarse_similarity_rows(E, 2, rows)
        dt = time.perf_counter() - t0
        m, d = 16384, 1024
        flops = 2.0 * len(rows) * m * d
        out.update(value=flops / dt / 1e12, unit="TFLOP/s", seconds=dt,
                   sample="128 of the 16,384 rows of the similarity matrix (BF16-rounded "
                          "embeddings, FP64 products)")
    return out


def oracle_workload(name):
    """_oracle_workload_inproc in a child process pinned to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-workload",
                          name], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def _oracle_pair_job(job):
    """One pair registered by the oracle (runs in a worker process pinned to one
    BLAS thread): job = (xyz_p [hw,3], xyz_q [hw,3], conf_p [hw], conf_q [hw]),
    float32.  Returns the Sim(3), status, cost, valid count, extent and the
    seconds the registration took."""
    import numpy as np
    from oracle import register as reg
    xp, xq, cp, cq = job
    xyz = np.stack([xp, xq])
    conf = np.stack([cp, cq])
    t0 = time.perf_counter()
    P, Q, wp, wq, valid = reg.pair_correspondences(xyz, conf, [0, 1], [0], [1], 0, 0.0)
    w = reg.base_weights(wp[valid], wq[valid])
    res = reg.irls(P[valid], Q[valid], w, DELTA, ITERS)
    dt = time.perf_counter() - t0
    Qv = Q[valid]
    ext = float(np.linalg.norm(Qv.max(0) - Qv.min(0))) if len(Qv) else 0.0
    S = res["S"]
    return {"S": (float(S[0]), np.asarray(S[1]).tolist(), np.asarray(S[2]).tolist()),
            "status": int(res["status"]), "cost": float(res["cost"]),
            "n_valid": int(valid.sum()), "extent": ext, "seconds": dt}


def oracle_pool(workers):
    """A pool of `workers` processes started with spawn (never forked from a
    process that holds a CUDA context), each pinned to one BLAS thread and
    without a GPU."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                           "MKL_NUM_THREADS", "CUDA_VISIBLE_DEVICES")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                      CUDA_VISIBLE_DEVICES="")
    try:
        pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        list(pool.map(_pool_warm, range(workers)))     # workers started, numpy imported
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool


def _pool_warm(_):
    import numpy  # noqa: F401
    from oracle import register  # noqa: F401
    return os.getpid()


def oracle_pairs(pool, jobs):
    """The oracle on every job, in parallel; returns (results, wall seconds)."""
    t0 = time.perf_counter()
    res = list(pool.map(_oracle_pair_job, jobs))
    return res, time.perf_counter() - t0


def sim3_error(row, ref):
    """(rotation angle rad, |s/s_ref - 1|, |t - t_ref|) of one 13-wide row."""
    import numpy as np
    s, R, t = float(row[0]), np.asarray(row[1:10]).reshape(3, 3), np.asarray(row[10:13])
    so, Ro, to = ref[0], np.asarray(ref[1]).reshape(3, 3), np.asarray(ref[2])
    # angle from the chord |R - Ro|_F = 2 sqrt(2) sin(angle / 2): accurate when small
    ang = 2.0 * np.arcsin(min(1.0, np.linalg.norm(R - Ro) / (2.0 * np.sqrt(2.0))))
    return float(ang), abs(s / so - 1.0), float(np.linalg.norm(t - to))


def oracle_check(args, ch, ps, S, poses, out_xyz, out_idx, M):
    """The oracle on sampled pairs of the benchmarked chain, one process per
    host core: its rate (cpu_baseline: pairs' work over the pool's wall time;
    the single-thread rate from each job's own time) and the error of the
    GPU's results against it (oracle_error): the registration of the sampled
    pairs, the fused points of one sampled submap under the GPU's corrected
    poses, and the corrected poses against the oracle's chaining plus one
    Gauss-Newton step on the GPU's registered edges."""
    import numpy as np
    from oracle import fuse as ofuse
    from oracle import pose_graph as opg
    workers = os.cpu_count() or 1
    n_jobs = min(ps.n_pairs, 2 * workers)
    ks = sorted({int(k) for k in np.linspace(0, ps.n_pairs - 1, n_jobs).round()})
    src, tgt = ps.src.cpu().numpy(), ps.tgt.cpu().numpy()
    jobs = [(ps.xyz[src[k]].cpu().numpy(), ps.xyz[tgt[k]].cpu().numpy(),
             ps.conf[src[k]].cpu().numpy(), ps.conf[tgt[k]].cpu().numpy()) for k in ks]
    pool = oracle_pool(workers)
    try:
        res, wall = oracle_pairs(pool, jobs)
    finally:
        pool.shutdown()
    n = sum(r["n_valid"] for r in res) * ITERS
    busy = sum(r["seconds"] for r in res)
    cpu = {"value": n / wall, "unit": UNIT, "cores": workers, "host_cores": os.cpu_count(),
           "kind": "oracle", "single_thread": n / busy,
           "sample": f"{len(ks)} of the {ps.n_pairs} chain pairs ({ps.hw:,} correspondences "
                     f"each, {ITERS} IRLS solves), FP64 numpy, one process per core ({workers}): "
                     f"{wall:.1f} s wall, {busy:.1f} s of CPU work"}
    Sh = S.cpu().numpy()
    reg_err = [sim3_error(Sh[k], r["S"]) for k, r in zip(ks, res)]
    rot = max(e[0] for e in reg_err)
    sc = max(e[1] for e in reg_err)
    tr = max(e[2] / max(r["extent"], 1e-30) for e, r in zip(reg_err, res))
    registration = {"pairs": len(ks), "statuses_zero": all(r["status"] == 0 for r in res),
                    "max_rotation_rad": rot, "max_relative_scale": sc,
                    "max_translation_over_extent": tr,
                    "within_tolerances": bool(rot <= 1e-5 and sc <= 1e-6 and tr <= 1e-6)}
    # fusion: the submap in the middle, at its offset in the fused buffer
    m = M // 2
    conf_h = ch.conf.view(M, -1)[:m + 1].cpu().numpy()
    npts = conf_h.shape[1]
    start = int((conf_h[:m] > 1.0).sum())
    ph = poses.cpu().numpy()
    pose_m = (float(ph[m, 0]), ph[m, 1:10].reshape(3, 3), ph[m, 10:13])
    ox, oi = ofuse.fuse_points(ch.xyz.view(M, -1, 3)[m:m + 1].cpu().numpy(), conf_h[m:m + 1],
                               [pose_m], 1.0, index_base=m * npts)
    gi = out_idx[start:start + len(oi)].cpu().numpy()
    gx = out_xyz[start:start + len(oi)].cpu().numpy().astype(np.float64)
    fext = max(float(np.linalg.norm(ox.max(0) - ox.min(0))), float(np.abs(ox).max()))
    fusion = {"submap": m, "points": int(len(oi)), "indices_equal": bool(np.array_equal(gi, oi)),
              "max_point_error_over_extent": float(np.abs(gx - ox).max() / fext),
              "within_tolerances": bool(np.array_equal(gi, oi) and
                                        np.abs(gx - ox).max() <= 1e-6 * fext)}
    # pose graph: the chain is a tree, so chaining satisfies every edge and
    # Gauss-Newton keeps it; the oracle chains the GPU's registered edges and
    # takes one step
    ei = np.arange(ps.n_pairs)
    Tij = [(float(Sh[k, 0]), Sh[k, 1:10].reshape(3, 3), Sh[k, 10:13])
           for k in range(ps.n_pairs)]
    init = opg.chain_init(M, ei, ei + 1, Tij)
    ref, hist, _ = opg.gauss_newton(init, ei, ei + 1, Tij, iters=1)
    pe = [sim3_error(ph[v], ref[v]) for v in range(M)]
    traj = np.stack([np.asarray(T[2]) for T in ref])
    text = max(float(np.linalg.norm(traj.max(0) - traj.min(0))), 1.0)
    pose_graph = {"nodes": M, "max_rotation_rad": max(e[0] for e in pe),
                  "max_relative_scale": max(e[1] for e in pe),
                  "max_translation_over_extent": max(e[2] for e in pe) / text,
                  "note": "GPU: chaining + 10 Gauss-Newton iterations; oracle: chaining + 1 "
                          "(the chain's graph is a tree: both stay at the chained poses)"}
    return cpu, {"registration": registration, "fusion": fusion, "pose_graph": pose_graph}


def _host_pair(ps, k):
    """Pair k of a device PairSet as a one-pair host PairSet (its frames only)."""
    import torch
    from paper_2510_02080_b300 import synth
    lo, hi = int(ps.link_off[k]), int(ps.link_off[k + 1])
    s, t = ps.src[lo:hi].long(), ps.tgt[lo:hi].long()
    f = hi - lo
    i32 = dict(dtype=torch.int32)
    pcm = None if ps.pair_conf_min is None else ps.pair_conf_min[k:k + 1].cpu()
    return synth.PairSet(torch.cat([ps.xyz[s], ps.xyz[t]]).cpu(),
                         torch.cat([ps.conf[s], ps.conf[t]]).cpu(),
                         torch.tensor([0, f], **i32), torch.arange(f, **i32),
                         torch.arange(f, 2 * f, **i32), ps.H, ps.W, pair_conf_min=pcm)


def registration_error(S, st, host_pairs, ks):
    """Error of the GPU's rows S[k] (and statuses) against the oracle on each
    listed pair's own frames."""
    from oracle import register as reg
    Sh, sth = S.cpu().numpy(), st.cpu().numpy()
    rot = sc = tr = 0.0
    same = True
    for k, hp in zip(ks, host_pairs):
        r = reg.align_pairs(hp, delta=DELTA, iters=ITERS)[0]
        same &= int(sth[k]) == r["status"]
        if r["status"] == 0:
            e = sim3_error(Sh[k], r["S"])
            rot, sc = max(rot, e[0]), max(sc, e[1])
            tr = max(tr, e[2] / max(r["extent"], 1e-30))
    return {"pairs": [int(k) for k in ks], "statuses_equal": bool(same),
            "max_rotation_rad": rot, "max_relative_scale": sc,
            "max_translation_over_extent": tr,
            "within_tolerances": bool(same and rot <= 1e-5 and sc <= 1e-6 and tr <= 1e-6)}


def pose_graph_error(ctx, ei, ej, Tij_rows, n, iters):
    """The GPU's pose graph (chaining + `iters` Gauss-Newton steps) against the
    oracle's on the same edges: chi^2 history and poses (relative to the
    trajectory's extent)."""
    import numpy as np
    import torch
    from oracle import pose_graph as opg
    nodes = torch.zeros((n, 13), dtype=torch.float64, device=Tij_rows.device)
    nodes[:, 0] = 1.0
    nodes[:, [1, 5, 9]] = 1.0
    chi2 = ctx.pose_graph_correct(nodes, ei, ej, Tij_rows, iters=iters).cpu().numpy()
    R = Tij_rows.cpu().numpy()
    Tij = [(float(r[0]), r[1:10].reshape(3, 3), r[10:13]) for r in R]
    ref, hist, _ = opg.gauss_newton(opg.chain_init(n, ei, ej, Tij), ei, ej, Tij, iters=iters)
    got = nodes.cpu().numpy()
    pe = [sim3_error(got[v], ref[v]) for v in range(n)]
    traj = np.stack([np.asarray(T[2]) for T in ref])
    text = max(float(np.linalg.norm(traj.max(0) - traj.min(0))), 1.0)
    return {"nodes": n, "gn_iters": iters,
            "max_chi2_relative": float(np.max(np.abs(chi2 - np.asarray(hist)) /
                                              np.maximum(np.abs(np.asarray(hist)), 1e-300))),
            "max_rotation": max(e[0] for e in pe), "max_relative_scale": max(e[1] for e in pe),
            "max_translation_over_extent": max(e[2] for e in pe) / text}


def _host_depth_pair(dps, k):
    """Pair k of a device depth pair set as a one-pair host PairSet of the
    oracle's pointmaps (its frames unprojected in FP64)."""
    import torch
    from oracle import unproject as oup
    from paper_2510_02080_b300 import synth
    lo, hi = int(dps.link_off[k]), int(dps.link_off[k + 1])
    fr = torch.cat([dps.src[lo:hi], dps.tgt[lo:hi]]).long()
    xyz = oup.unproject(dps.depth[fr].double().cpu().numpy(), dps.cams[fr].cpu().numpy())
    f = hi - lo
    i32 = dict(dtype=torch.int32)
    return synth.PairSet(torch.from_numpy(xyz), dps.conf[fr].reshape(2 * f, -1).cpu(),
                         torch.tensor([0, f], **i32), torch.arange(f, **i32),
                         torch.arange(f, 2 * f, **i32), dps.H, dps.W)


def map_fusion_error(xyz, conf, ox, oi, pts, refs, m=7):
    """The map's fusion (identity poses) on submap m and the point correction of
    the sampled references into submaps 0..m, against the oracle."""
    import numpy as np
    from oracle import fuse as ofuse
    eye = (1.0, np.eye(3), np.zeros(3))
    ch = conf[:m + 1].cpu().numpy()
    n = ch.shape[1]
    start = int((ch[:m] > 1.0).sum())
    xm = xyz[:m + 1].cpu().numpy()
    rx, ri = ofuse.fuse_points(xm[m:m + 1], ch[m:m + 1], [eye], 1.0, index_base=m * n)
    gi = oi[start:start + len(ri)].cpu().numpy()
    gx = ox[start:start + len(ri)].cpu().numpy().astype(np.float64)
    ext = max(float(np.linalg.norm(rx.max(0) - rx.min(0))), float(np.abs(rx).max()))
    fusion = {"submap": m, "points": int(len(ri)), "indices_equal": bool(np.array_equal(gi, ri)),
              "max_point_error_over_extent": float(np.abs(gx - rx).max() / ext)}
    r = refs.cpu().numpy()
    sel = np.flatnonzero((r >= 0) & (r < (m + 1) * n))
    before = np.zeros((len(sel), 3))
    ref_pts = ofuse.correct_points(before, r[sel], xm, ch, [eye] * (m + 1), 1.0)[0]
    got = pts[torch_index(sel, pts)].cpu().numpy().astype(np.float64)
    cext = max(float(np.abs(ref_pts).max()), 1.0)
    correction = {"references": int(len(sel)),
                  "max_point_error_over_extent": float(np.abs(got - ref_pts).max() / cext)}
    return fusion, correction


def torch_index(idx, like):
    import torch
    return torch.as_tensor(idx, dtype=torch.int64, device=like.device)


def similarity_error(ctx, E, kw, n_rows=64):
    """The BF16 tensor-core similarity on sampled rows against the exact FP64
    cosines of the FP32 embeddings, and the coarse decisions at tau_global that
    differ (far pairs only)."""
    import numpy as np
    import torch
    from oracle import loops as olp
    _, _, _, S = ctx.loop_candidates(E, with_sim=True, **kw)
    En = E.cpu().numpy()
    stride, tau, gap = kw["stride"], kw["tau_global"], kw["gap"]
    m = S.shape[0]
    rows = np.sort(np.random.default_rng(9).choice(m, min(n_rows, m), replace=False))
    cos = olp.cosine_rows(En, stride, rows)
    got = S[torch.as_tensor(rows, device=S.device)].cpu().numpy().astype(np.float64)
    worst, flips = 0.0, 0
    for r, a in enumerate(rows):
        g, c = got[r, a:], cos[r, a:]
        worst = max(worst, float(np.abs(g - c).max()))
        far = (np.arange(a, m) - a) * stride >= gap
        flips += int((far & ((g > tau) != (c > tau))).sum())
    return {"rows": int(len(rows)), "max_abs_error_vs_exact_cosine": worst,
            "flipped_coarse_decisions": flips}


def adjoint_error(ctx, ps, gS, gc, delta=DELTA, iters=ITERS):
    """The backward call's gradients against the oracle's FP64 reverse mode
    (element by element, |d| <= 2e-3 |g| + 1e-5 max|g| + f32, points away from
    the Huber kink; f32 = twice the largest change of the oracle's gradient
    when its weighting estimate is rounded to FP32, the FP32-residual design's
    own effect): the largest ratio of error to bound per gradient, and the
    ratio without f32."""
    import numpy as np
    from oracle import adjoint as oadj
    from oracle import register as reg
    gx, gcf = ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, gS, gc)
    xyz, conf = ps.xyz.double().cpu().numpy(), ps.conf.double().cpu().numpy()
    P, Q, cp, cq, valid = reg.pair_correspondences(xyz, conf, [0, 1], [0], [1], 0, 0.0)
    w = cp[valid] * cq[valid]
    Sh, tape, _ = oadj.irls_forward(P[valid], Q[valid], w, delta, iters)
    g = gS.cpu().numpy()[0]
    gP, gQ, gw = oadj.irls_backward(P[valid], Q[valid], w, delta, tape, Sh, g[0],
                                    g[1:10].reshape(3, 3), g[10:13], float(gc[0]))
    gcp, gcq = oadj.weight_grads(gw, cp[valid], cq[valid])
    S32, tape32, _ = oadj.irls_forward(P[valid], Q[valid], w, delta, iters,
                                       estimate_dtype=np.float32)
    gP32, gQ32, gw32 = oadj.irls_backward(P[valid], Q[valid], w, delta, tape32, S32, g[0],
                                          g[1:10].reshape(3, 3), g[10:13], float(gc[0]))
    gcp32, gcq32 = oadj.weight_grads(gw32, cp[valid], cq[valid])
    far = np.ones(int(valid.sum()), bool)
    for rec in tape[1:]:
        far &= np.abs(rec["r"] - delta) >= 1e-4
    gxh, gch = gx.cpu().double().numpy(), gcf.cpu().double().numpy()
    f32x = 2.0 * max(np.abs(gP32 - gP)[far].max(), np.abs(gQ32 - gQ)[far].max())
    f32c = 2.0 * max(np.abs(gcp32 - gcp)[far].max(), np.abs(gcq32 - gcq)[far].max())

    def ratio(got, ref, f32):
        b = 2e-3 * np.abs(ref) + 1e-5 * np.abs(ref).max() + f32
        return float((np.abs(got - ref) / b).max())

    def both(a, b, c, d, f32):
        return max(ratio(a, b, f32), ratio(c, d, f32)), max(ratio(a, b, 0.0), ratio(c, d, 0.0))
    dx = both(gxh[0][valid][far], gP[far], gxh[1][valid][far], gQ[far], f32x)
    dc = both(gch[0][valid][far], gcp[far], gch[1][valid][far], gcq[far], f32c)
    return {"points": int(far.sum()),
            "dxyz_error_over_bound": dx[0], "dconf_error_over_bound": dc[0],
            "dxyz_error_over_bound_without_f32": dx[1],
            "dconf_error_over_bound_without_f32": dc[1],
            "f32_over_max": {"dxyz": f32x / max(np.abs(gP).max(), np.abs(gQ).max()),
                             "dconf": f32c / max(np.abs(gcp).max(), np.abs(gcq).max())},
            "bound": "|GPU - oracle| <= 2e-3 |oracle| + 1e-5 max|oracle| + f32 per element"}


def run_reference(args):
    """The oracle as it stands, one process per host core, on consecutive pairs
    of a chain of the benchmark's recipe generated on the host (one pair per
    core per step); same metric and unit.  Rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2510_02080_b300 import synth
    workers = os.cpu_count() or 1
    ch = synth.make_chain(synth.SEED_BASE + 2, M=workers + 1, F=F_FRAMES, H=H, W=W,
                          device="cpu")
    ps = ch.pairs()
    jobs = [(ps.xyz[int(ps.src[k])].numpy(), ps.xyz[int(ps.tgt[k])].numpy(),
             ps.conf[int(ps.src[k])].numpy(), ps.conf[int(ps.tgt[k])].numpy())
            for k in range(ps.n_pairs)]
    pool = oracle_pool(workers)
    try:
        for _ in range(args.warmup):
            oracle_pairs(pool, jobs)
        n, wall, busy = 0, 0.0, 0.0
        for _ in range(args.steps):
            res, dt = oracle_pairs(pool, jobs)
            n += sum(r["n_valid"] for r in res) * ITERS
            wall += dt
            busy += sum(r["seconds"] for r in res)
    finally:
        pool.shutdown()
    rate = n / wall
    sample = (f"{ps.n_pairs} chain pairs per step (152,292 correspondences each, {ITERS} IRLS "
              f"solves) of a {ps.n_pairs + 1}-submap chain of the benchmark's recipe, FP64 "
              f"numpy, one process per core ({workers})")
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "chain200_294x518", "sample_pairs_per_step": ps.n_pairs,
                       "iters": ITERS, "delta": DELTA},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": workers,
                             "host_cores": os.cpu_count(), "kind": "oracle",
                             "single_thread": n / busy, "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_2510_02080_b300 import build, ec3r, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    ctx = ec3r.Context(local)
    if args.variant >= 0:
        ctx.set_align_variant(args.variant)
    ctx.set_backward_ctas_per_sm(args.bwd_ctas_per_sm)

    # per-rank synthetic chain (weak scaling: every rank owns its own map)
    M = args.submaps
    ch = synth.make_chain(synth.SEED_BASE + 2 + 1000 * rank, M=M, F=F_FRAMES, H=H, W=W,
                          device=dev)
    ps = ch.pairs()
    n_frames, hw = ps.conf.shape
    xyz_f, conf_f = ps.xyz, ps.conf
    fin = torch.isfinite(xyz_f).all(-1) & torch.isfinite(conf_f) & (conf_f > 0)
    n_valid = int((fin[ps.src.long()] & fin[ps.tgt.long()]).sum())
    del fin
    pix = ps.n_pairs * hw
    n_fuse = M * F_FRAMES * hw
    conf_m = ch.conf.view(M, -1)
    kept = int((conf_m > 1.0).sum())
    out_xyz = torch.empty((kept, 3), device=dev)
    out_idx = torch.empty((kept,), dtype=torch.int64, device=dev)
    S = torch.empty((ps.n_pairs, 13), dtype=torch.float64, device=dev)
    st = torch.empty((ps.n_pairs,), dtype=torch.int32, device=dev)
    # pose graph: node m = submap m, edge (m, m+1) carries pair m's estimate
    import numpy as np
    ei = np.arange(ps.n_pairs, dtype=np.int32)
    ej = ei + 1
    poses = torch.zeros((M, 13), dtype=torch.float64, device=dev)
    poses[:, 0] = 1.0
    poses[:, [1, 5, 9]] = 1.0          # identity; node 0 stays fixed (world = submap 0)
    chi2 = torch.empty((PG_ITERS + 1,), dtype=torch.float64, device=dev)
    n_cursor = 2 * args.steps + args.warmup + 8
    cursors = torch.zeros((n_cursor,), dtype=torch.int64, device=dev)
    ci = [0]

    # adjoint: a fixed synthetic upstream gradient dL/dS, dL/dcost per pair
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    gS = torch.randn((ps.n_pairs, 13), generator=gen, dtype=torch.float64, device=dev)
    gcost = torch.ones((ps.n_pairs,), dtype=torch.float64, device=dev)
    cost = torch.empty((ps.n_pairs,), dtype=torch.float64, device=dev)
    gxyz = torch.empty((n_frames, hw, 3), dtype=torch.float32, device=dev)
    gconf = torch.empty((n_frames, hw), dtype=torch.float32, device=dev)

    # The adjoint needs only the registration's checkpoints, so the pose graph
    # (which needs the registered edges) runs on a second, high-priority
    # stream while the adjoint runs on the main one; the latency-bound
    # pose-graph launches then fill the gaps of the HBM-bound adjoint sweeps.
    # Beside the adjoint the pose graph is the longer branch, so the fusion's
    # keep counts (no pose needed) follow the adjoint on the main stream; its
    # scan and scatter (HBM-bound, they need the corrected poses) follow them
    # once the pose graph is done.
    side = torch.cuda.Stream(device=dev, priority=-1)
    tile_counts = torch.empty((M * ((n_frames // M * hw + 8191) // 8192),), dtype=torch.int32,
                              device=dev)
    keep_mask = torch.empty((tile_counts.numel() * 256,), dtype=torch.int32, device=dev)
    ev_reg, ev_side = torch.cuda.Event(), torch.cuda.Event()

    def step(xyz_in, conf_in, overlap=True):
        main = torch.cuda.current_stream()
        sec = side if overlap else main
        ctx.align_submaps(xyz_in.view(n_frames, hw, 3), conf_in.view(n_frames, hw), ps.link_off,
                          ps.src, ps.tgt, delta=DELTA, iters=ITERS, out=S, status=st,
                          want_cost=True, cost=cost, stream=main)
        ev_reg.record(main)
        sec.wait_event(ev_reg)
        ctx.pose_graph_correct(poses, ei, ej, S, iters=PG_ITERS, chi2=chi2, stream=sec)
        ev_side.record(sec)
        if not args.no_adjoint:
            lib = ec3r.lib()
            o = ec3r.AlignOpts(DELTA, ITERS, 0.0, 0, 0, 1)
            ctx._check(lib.ec3r_align_submaps_backward(
                ctx._h, ec3r._ptr(xyz_in), ec3r._ptr(conf_in), n_frames, hw, ps.n_pairs,
                int(ps.src.numel()), ec3r._ptr(ps.link_off), ec3r._ptr(ps.src),
                ec3r._ptr(ps.tgt), None, ec3r.C.byref(o), ctx.align_token(), ec3r._ptr(gS),
                ec3r._ptr(gcost), ec3r._ptr(gxyz), ec3r._ptr(gconf), ec3r._stream(main)))
        # the fusion's keep counts need no pose: in the adjoint branch's slack
        ctx.fuse_count(conf_in.view(M, -1), tile_counts, keep_mask, stream=main)
        main.wait_event(ev_side)
        c = cursors[ci[0] % n_cursor:ci[0] % n_cursor + 1]
        ci[0] += 1
        ctx.fuse_points_counted(xyz_in.view(M, -1, 3), tile_counts, keep_mask, poses,
                                out_xyz, out_idx, c, stream=main)

    for _ in range(args.warmup):
        step(ch.xyz, ch.conf)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0, ctx.last_error()
    assert int((st != 0).sum()) == 0

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- timed region: inputs resident in HBM, every call replayed from its
    # cached CUDA graph ------------------------------------------------------
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step(ch.xyz, ch.conf)
    e1.record(s)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    assert ctx.sync_status() == 0, ctx.last_error()
    # ---- the same K steps again with every kernel bracketed by CUDA events on
    # its launching stream (direct launches, one stream, so that each kernel's
    # duration is its own): per-kernel durations -------------------------------
    ctx.profile(True)
    ctx.profile_read()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(s)
    for _ in range(args.steps):
        step(ch.xyz, ch.conf, overlap=False)
    p1.record(s)
    torch.cuda.synchronize()
    ms_profiled = p0.elapsed_time(p1)
    prof = ctx.profile_read()
    ctx.profile(False)
    assert ctx.sync_status() == 0, ctx.last_error()
    # ---- comparator: the plain single-pair FP64-accumulation path, looped over
    # the same pairs (one call per pair, direct launches) ----------------------
    comparator = None
    if not args.no_comparator and rank == 0:
        # direct launches without per-kernel events: the allocation-free entry
        # point runs the same set-up, FP64 sweeps and solves with no graph
        one = torch.tensor([0, 1], dtype=torch.int32, device=dev)
        S1 = torch.empty((1, 13), dtype=torch.float64, device=dev)
        st1 = torch.empty((1,), dtype=torch.int32, device=dev)
        o64 = ec3r.AlignOpts(DELTA, ITERS, 0.0, 0, ec3r.PREC["fp64"], 0)
        f = ec3r.lib().ec3r_align_submaps_noalloc
        f.argtypes = [ec3r._P, ec3r._P, ec3r._I64, ec3r._I64, ec3r.C.c_int, ec3r._I64,
                      ec3r._P, ec3r._P, ec3r._P, ec3r._P, ec3r.C.POINTER(ec3r.AlignOpts),
                      ec3r._P, ec3r._P, ec3r._P, ec3r._P]
        f.restype = ec3r.C.c_int
        xyz_p, conf_p = ec3r._ptr(ch.xyz), ec3r._ptr(ch.conf)
        lo_p, so_p, sto_p = ec3r._ptr(one), ec3r._ptr(S1), ec3r._ptr(st1)
        src_p = [ec3r.C.c_void_p(ps.src.data_ptr() + 4 * k) for k in range(ps.n_pairs)]
        tgt_p = [ec3r.C.c_void_p(ps.tgt.data_ptr() + 4 * k) for k in range(ps.n_pairs)]
        sp = ec3r._stream(s)

        def loop_pairs():
            for k in range(ps.n_pairs):
                rc = f(xyz_p, conf_p, n_frames, hw, 1, 1, lo_p, src_p[k], tgt_p[k], None,
                       ec3r.C.byref(o64), so_p, sto_p, None, sp)
                assert rc == 0
        loop_pairs()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(s)
        loop_pairs()
        c1.record(s)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        comparator = {"impl": "single-pair FP64-accumulation registration looped over the 199 "
                              "pairs (same inputs; one set-up and 10 x (FP64 sweep, solve) "
                              "launches per pair, no per-kernel events)",
                      "pt_iter_per_s": n_valid * ITERS / (cms * 1e-3), "ms": cms}
    ms_max = ms
    if ws > 1:
        from paper_2510_02080_b300 import shard
        ms_max = shard.max_over_ranks(ms)
    value = n_valid * ITERS * args.steps * ws / (ms_max * 1e-3)

    # ---- end to end: host buffers, copies inside the timed region ------------
    e2e = None
    if not args.no_e2e:
        hx = torch.empty(ch.xyz.shape, dtype=torch.float32, pin_memory=True)
        hc = torch.empty(ch.conf.shape, dtype=torch.float32, pin_memory=True)
        hx.copy_(ch.xyz)
        hc.copy_(ch.conf)
        # two device input buffers: step s+1's inputs are copied on a copy
        # stream while step s computes (every step still copies all of its
        # inputs from pinned host memory and reads its result back)
        dxs = [torch.empty(hx.shape, dtype=torch.float32, device=dev) for _ in range(2)]
        dcs = [torch.empty(hc.shape, dtype=torch.float32, device=dev) for _ in range(2)]
        ready = [torch.cuda.Event() for _ in range(2)]
        free = [torch.cuda.Event() for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=dev)
        hS = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
        e2e_steps = max(1, min(args.steps, 5))

        def upload(b):
            copy_stream.wait_event(free[b])
            with torch.cuda.stream(copy_stream):
                dxs[b].copy_(hx, non_blocking=True)
                dcs[b].copy_(hc, non_blocking=True)
            ready[b].record(copy_stream)

        def run(n):
            main = torch.cuda.current_stream()
            for b in range(2):
                free[b].record(main)
            upload(0)
            for i in range(n):
                b = i % 2
                if i + 1 < n:
                    upload(1 - b)
                main.wait_event(ready[b])
                step(dxs[b], dcs[b])
                free[b].record(main)
                hS.copy_(S, non_blocking=True)
            torch.cuda.synchronize()

        run(2)
        barrier()
        t0 = time.perf_counter()
        run(e2e_steps)
        barrier()
        dt = time.perf_counter() - t0
        e2e = {"value": n_valid * ITERS * e2e_steps * ws / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(hx.numel() * 4 + hc.numel() * 4),
               "d2h_bytes_per_step": int(hS.numel() * 8), "steps": e2e_steps,
               "pipelining": "double-buffered inputs: copy of step s+1 overlaps step s"}
        del hx, hc, dxs, dcs

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    # the dominant kernel: the persistent registration launch of sweeps 2 ..
    # K-1 (sweep 1 runs in its own launch before it; the last sweep and solve
    # in the final-sweep launch, since the adjoint needs the cost), 28 B per
    # link pixel per sweep
    sweeps = (ITERS - 1 if "irls_final_sweep" in prof else ITERS) - 1
    reg_k = prof.get("irls_register", (0.0, 0))
    reg_launch_ms = reg_k[0] / max(reg_k[1], 1)
    reg_bytes = SWEEP_BYTES_PER_PIXEL * pix * sweeps
    achieved = reg_bytes / (reg_launch_ms * 1e-3) / 1e9 if reg_launch_ms > 0 else 0.0
    total_prof = sum(v[0] for v in prof.values())
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                   "share": v[0] / total_prof if total_prof else None} for k, v in prof.items()}
    fuse_ms = sum(prof.get(k, (0.0, 0))[0] for k in ("fuse_count", "fuse_scan", "fuse_scatter"))
    pg_ms = sum(v[0] for k, v in prof.items() if k.startswith("pg_"))
    adj_ms = sum(v[0] for k, v in prof.items() if k.startswith("adj_"))
    # the whole registration call: set-up, the persistent launch, and the final
    # sweep with the last solve and the cost that the adjoint needs (or, for
    # the grid variant, every sweep, solve and the cost sweep as grids)
    reg_ms = sum(prof.get(k, (0.0, 0))[0]
                 for k in ("align_setup", "irls_sweep1", "irls_register", "irls_final_sweep",
                           "irls_cost", "irls_sweep_fp32", "sim3_solve"))
    reg_rate = n_valid * ITERS * args.steps / (reg_ms * 1e-3) if reg_ms else None
    # bytes the registration call streams per correspondence and iteration
    call_bytes_pt_iter = (SWEEP1_BYTES_PER_PIXEL + SWEEP_BYTES_PER_PIXEL * (ITERS - 1)) / ITERS
    fuse_gbs = 26.0 * n_fuse * args.steps / (fuse_ms * 1e-3) / 1e9 if fuse_ms else None
    variant, tune_ms = ctx.last_align_variant()
    vt, vc, vp = ec3r.align_variant_info(variant) if variant >= 0 else (None, None, None)
    # ---- the oracle on sampled pairs of this workload, on every host core:
    # its rate (cpu_baseline) and each result's error against it (oracle_error)
    cpu_base = oracle_error = None
    if not args.no_cpu_baseline and ws == 1:
        cpu_base, oracle_error = oracle_check(args, ch, ps, S, poses, out_xyz, out_idx, M)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"chain{M}_294x518", "submaps": M, "frames": F_FRAMES,
                   "H": H, "W": W, "pairs": ps.n_pairs, "valid_correspondences": n_valid,
                   "iters": ITERS, "huber_delta": DELTA, "precision": "fp32 moments, fp64 solve",
                   "fused_points": n_fuse, "kept_points": kept,
                   "pose_graph": {"nodes": M, "edges": ps.n_pairs, "gn_iters": PG_ITERS},
                   "rows": ["registration", "pose graph", "fusion"] +
                           ([] if args.no_adjoint else ["adjoint"]),
                   "l2": "inputs 2.4 GB per rank > 126 MB L2; no flush"},
        "roofline": {"bound": "hbm", "kernel": "irls_register", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (REGISTER_TRAFFIC_BYTES_PER_PIXEL_SWEEP[variant] * pix * sweeps
                                 if variant in REGISTER_TRAFFIC_BYTES_PER_PIXEL_SWEEP else None),
                     "algorithmic_bytes_per_launch": reg_bytes,
                     "launch_ms": reg_launch_ms,
                     "sweeps_per_launch": sweeps,
                     "note": "the persistent launch of Huber-IRLS sweeps 2 .. K-1 and their "
                             "per-pair FP64 solves (sweep 1 has its own launch before it, "
                             "the last sweep and solve the final-sweep launch after it); "
                             "28 B per link pixel per sweep: p, q and the stored weight",
                     "registration": {
                         "pt_iter_per_s": reg_rate,
                         "bytes_per_pt_iter": call_bytes_pt_iter,
                         "achieved": (call_bytes_pt_iter * reg_rate / 1e9
                                      if reg_rate else None),
                         "frac": (call_bytes_pt_iter * reg_rate / 1e9 / peak
                                  if reg_rate else None),
                         "effective_gbs_at_32B": (METRIC_BYTES_PER_PT_ITER * reg_rate / 1e9
                                                  if reg_rate else None),
                         "note": "the whole registration call (set-up, sweep-1 launch, "
                                 "persistent launch, final sweep with the last solve and the "
                                 "cost the adjoint needs: 10 sweeps streamed, 36 B per pixel "
                                 "in the first and 28 B in each other); effective_gbs_at_32B "
                                 "counts the metric's 32 B per correspondence and iteration"}},
        "sweep_variant": {"variant": variant, "tile_pixels": vt, "ctas_per_sm": vc,
                          "persistent": vp,
                          "tuning_ms": {str(k): v for k, v in tune_ms.items()}},
        "kernels": kernels,
        "profiled_pass": {"ms_per_step": ms_profiled / args.steps,
                          "note": "same K steps, direct launches on one stream (no overlap), "
                                  "an event pair per kernel"},
        "fusion": {"ms_per_step": fuse_ms / args.steps, "gbs_at_26B_per_point": fuse_gbs},
        "pose_graph": {"ms_per_step": pg_ms / args.steps},
        "adjoint": {"ms_per_step": adj_ms / args.steps},
        "registration": {"ms_per_step": reg_ms / args.steps, "pt_iter_per_s": reg_rate},
        "clocks": clk,
        "comparator": comparator,
        "gpu_launches": int(sum(v[1] for v in prof.values())),
    }
    if e2e:
        line["e2e"] = e2e
    if cpu_base is not None:
        line["cpu_baseline"] = cpu_base
        line["oracle_error"] = oracle_error
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_strong(args):
    """--scaling strong: ONE 200-submap map split over the ranks (shard.map_step):
    each rank registers its share of the pairs (balanced by correspondence
    count) over only the frames they use and runs their adjoint, the Sim(3)
    rows meet on rank 0, which solves the pose graph and broadcasts the
    corrected poses, and each rank fuses its share of the submaps at an offset
    from one all-gathered count.  Total work is fixed as N grows."""
    import numpy as np
    import torch
    from paper_2510_02080_b300 import build, ec3r, shard, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    ctx = ec3r.Context(local)
    if args.variant >= 0:
        ctx.set_align_variant(args.variant)
    M = args.submaps
    ch = synth.make_chain(synth.SEED_BASE + 2, M=M, F=F_FRAMES, H=H, W=W, device=dev)
    ps = ch.pairs()
    n_frames, hw = ps.conf.shape
    fin = torch.isfinite(ps.xyz).all(-1) & torch.isfinite(ps.conf) & (ps.conf > 0)
    n_valid = int((fin[ps.src.long()] & fin[ps.tgt.long()]).sum())
    del fin
    plan = shard.plan_shard(ps.link_off.cpu(), ps.src.cpu(), ps.tgt.cpu(), [hw] * ps.n_pairs, M)
    f = plan.frames.to(dev)
    lx, lc = ps.xyz.index_select(0, f).contiguous(), ps.conf.index_select(0, f).contiguous()
    m0, m1 = plan.submaps
    sx = ch.xyz.view(M, -1, 3)[m0:m1].contiguous()
    sc = ch.conf.view(M, -1)[m0:m1].contiguous()
    a, b = plan.pairs
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    gS = torch.randn((ps.n_pairs, 13), generator=gen, dtype=torch.float64, device=dev)
    gcost = torch.ones((ps.n_pairs,), dtype=torch.float64, device=dev)
    kern = shard.GpuKernels(ctx, DELTA, ITERS, PG_ITERS,
                            adjoint=lambda n: (gS[a:b].contiguous(), gcost[a:b].contiguous()))
    ei = np.arange(ps.n_pairs, dtype=np.int32)
    npts = F_FRAMES * hw

    def step():
        return shard.map_step(kern, plan, lx, lc, ei, ei + 1, sx, sc, npts)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0, ctx.last_error()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        out = step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ms = shard.max_over_ranks(e0.elapsed_time(e1))
    clk = clocks.stop()
    assert ctx.sync_status() == 0, ctx.last_error()
    total = out["total"]
    if rank == 0:
        line = {"metric": METRIC, "value": n_valid * ITERS * args.steps / (ms * 1e-3),
                "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"chain{M}_294x518", "pairs": ps.n_pairs,
                           "valid_correspondences": n_valid, "iters": ITERS,
                           "fused_points_kept": total,
                           "parallelism": f"one map over {ws} rank(s): pairs and submaps "
                                          "split, Sim(3) rows gathered on rank 0, corrected "
                                          "poses broadcast, fusion offsets all-gathered",
                           "rows": ["registration", "adjoint", "pose graph", "fusion"],
                           "l2": "inputs 2.4 GB > 126 MB L2; no flush"},
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# the other workloads (one JSON line each; not the benchmark line)
# ----------------------------------------------------------------------------
def _time(fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _valid_count(ps, pcm=None):
    import torch
    fin = torch.isfinite(ps.xyz).all(-1) & torch.isfinite(ps.conf)
    lo = ps.link_off.cpu().tolist()
    n = 0
    for k in range(ps.n_pairs):
        thr = 0.0 if pcm is None else float(pcm[k])
        for l in range(lo[k], lo[k + 1]):
            a, b = int(ps.src[l]), int(ps.tgt[l])
            n += int((fin[a] & fin[b] & (ps.conf[a] > thr) & (ps.conf[b] > thr)).sum())
    return n


def run_workload(args):
    import numpy as np
    import torch
    from paper_2510_02080_b300 import build, ec3r, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    ctx = ec3r.Context(0)
    if args.variant >= 0:
        ctx.set_align_variant(args.variant)
    peak, peak_kind = peaks()
    out = {"workload": args.workload, "unit": UNIT, "data": "synthetic"}

    def reg_rate(ps, precision="fp32c", reps=5):
        n_valid = _valid_count(ps, ps.pair_conf_min)
        S = torch.empty((ps.n_pairs, 13), dtype=torch.float64, device=dev)
        st = torch.empty((ps.n_pairs,), dtype=torch.int32, device=dev)
        ms = _time(lambda: ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt,
                                             ps.pair_conf_min, delta=DELTA, iters=ITERS,
                                             precision=precision, out=S, status=st), reps)
        assert ctx.sync_status() == 0, ctx.last_error()
        v, tms = ctx.last_align_variant()
        if v >= 0:
            t, c, pers = ec3r.align_variant_info(v)
            out.setdefault("sweep_variants", []).append(
                {"pairs": ps.n_pairs, "variant": v, "tile_pixels": t, "ctas_per_sm": c,
                 "persistent": pers,
                 "tuning_ms": {str(k): x for k, x in tms.items()}})
        return n_valid, ms, S, st

    if args.workload == "pair1":
        ps = synth.make_pair(synth.SEED_BASE + 1, H=294, W=518, sigma=0.005, device=dev)
        for prec in ("fp64", "fp32c"):
            n, ms, S, st = reg_rate(ps, prec, reps=50)
            out[prec] = {"pt_iter_per_s": n * ITERS / (ms * 1e-3), "ms_per_call": ms,
                         "valid": n}
        out["note"] = "one 294x518 pair, 10 IRLS solves: latency-bound (4.9 MB, L2-resident)"
        host = [_host_pair(ps, 0)]
        out["oracle_error"] = {}
        for prec in ("fp64", "fp32c"):
            n, ms, S, st = reg_rate(ps, prec, reps=1)
            out["oracle_error"][prec] = registration_error(S, st, host, [0])
    elif args.workload == "adjoint1":
        ps = synth.make_pair(synth.SEED_BASE + 4, H=294, W=518, sigma=0.005, device=dev)
        n, ms_f, S, st = reg_rate(ps, reps=50)
        gS = torch.randn((1, 13), dtype=torch.float64, device=dev)
        gc = torch.ones((1,), dtype=torch.float64, device=dev)
        cost = torch.empty((1,), dtype=torch.float64, device=dev)

        def fwd_bwd():
            ctx.align_submaps(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, want_cost=True,
                              out=S, status=st, cost=cost)
            ctx.align_submaps_backward(ps.xyz, ps.conf, ps.link_off, ps.src, ps.tgt, gS, gc,
                                       fwd_token=ctx.align_token())
        ms = _time(fwd_bwd, 20)
        out.update({"forward_ms": ms_f, "forward_backward_ms": ms, "valid": n,
                    "note": "config-1 pair, 10 checkpointed IRLS iterations differentiated"})
        out["oracle_error"] = adjoint_error(ctx, ps, gS, gc)
    elif args.workload == "loops512":
        npairs = args.loop_pairs
        ps = synth.make_loop_batch(synth.SEED_BASE + 3, n_pairs=npairs, H=294, W=518,
                                   device=dev)
        n, ms, S, st = reg_rate(ps, reps=5)
        px = int(ps.link_off[-1]) * ps.hw
        out["registration"] = {"pairs": npairs, "valid": n, "ms": ms,
                               "pt_iter_per_s": n * ITERS / (ms * 1e-3),
                               "gbs_at_32B_per_pixel": 32.0 * px * ITERS / (ms * 1e-3) / 1e9}
        g = synth.make_pose_graph(synth.SEED_BASE + 3, 200, 40, device="cpu")
        Tij = ec3r.sim3_rows(g.T_meas.s, g.T_meas.R, g.T_meas.t).to(dev)
        nodes = torch.zeros((200, 13), dtype=torch.float64, device=dev)
        nodes[:, 0] = 1.0
        nodes[:, [1, 5, 9]] = 1.0
        pg_ms = _time(lambda: ctx.pose_graph_correct(nodes, g.ei.numpy(), g.ej.numpy(), Tij,
                                                     iters=10), 5)
        out["pose_graph"] = {"nodes": 200, "edges": len(g.ei), "gn_iters": 10, "ms": pg_ms}
        ks = [0, npairs // 2, npairs - 1]
        out["oracle_error"] = {
            "registration": registration_error(S, st, [_host_pair(ps, k) for k in ks], ks),
            "pose_graph": pose_graph_error(ctx, g.ei.numpy(), g.ej.numpy(), Tij, 200, 2)}
    elif args.workload == "map1000":
        M = 1000
        ch = synth.make_chain(synth.SEED_BASE + 5, M=M, F=5, H=392, W=518, device=dev)
        lb = synth.make_loop_batch(synth.SEED_BASE + 55, n_pairs=300, H=392, W=518,
                                   max_valid=760_000, device=dev)
        cp = ch.pairs()
        nf = cp.xyz.shape[0]
        bank = synth.PairSet(torch.cat([cp.xyz, lb.xyz]), torch.cat([cp.conf, lb.conf]),
                             torch.cat([cp.link_off[:-1], lb.link_off + int(cp.link_off[-1])]),
                             torch.cat([cp.src, lb.src + nf]), torch.cat([cp.tgt, lb.tgt + nf]),
                             392, 518,
                             pair_conf_min=torch.cat([torch.zeros(cp.n_pairs, device=dev),
                                                      lb.pair_conf_min]))
        del lb
        n, ms, S, st = reg_rate(bank, reps=3)
        px = int(bank.link_off[-1]) * bank.hw
        out["registration"] = {"pairs": bank.n_pairs, "valid": n, "ms": ms,
                               "pt_iter_per_s": n * ITERS / (ms * 1e-3),
                               "gbs_at_32B_per_pixel": 32.0 * px * ITERS / (ms * 1e-3) / 1e9}
        ks = [0, 500, 998, 1000, 1150, 1298]
        err = {"registration": registration_error(S, st, [_host_pair(bank, k) for k in ks], ks)}
        del bank
        g = synth.make_pose_graph(synth.SEED_BASE + 5, M, 300, device="cpu")
        Tij = ec3r.sim3_rows(g.T_meas.s, g.T_meas.R, g.T_meas.t).to(dev)
        nodes = torch.zeros((M, 13), dtype=torch.float64, device=dev)
        nodes[:, 0] = 1.0
        nodes[:, [1, 5, 9]] = 1.0
        pg_ms = _time(lambda: ctx.pose_graph_correct(nodes, g.ei.numpy(), g.ej.numpy(), Tij,
                                                     iters=10), 1, warm=1)
        out["pose_graph"] = {"nodes": M, "edges": len(g.ei), "gn_iters": 10, "ms": pg_ms}
        err["pose_graph"] = pose_graph_error(ctx, g.ei.numpy(), g.ej.numpy(), Tij, M, 1)
        xyz = ch.xyz.view(M, -1, 3)
        conf = ch.conf.view(M, -1)
        kept = int((conf > 1.0).sum())
        ox = torch.empty((kept, 3), device=dev)
        oi = torch.empty((kept,), dtype=torch.int64, device=dev)
        cur = torch.zeros((1,), dtype=torch.int64, device=dev)
        poses = torch.zeros((M, 13), dtype=torch.float64, device=dev)
        poses[:, 0] = 1.0
        poses[:, [1, 5, 9]] = 1.0

        def fuse():
            cur.zero_()
            ctx.fuse_points(xyz, conf, poses, ox, oi, cur)
        fms = _time(fuse, 3)
        assert ctx.sync_status() == 0 and int(cur) == kept
        npts = conf.numel()
        out["fusion"] = {"points": npts, "kept": kept, "ms": fms,
                         "gbs_at_26B_per_point": 26.0 * npts / (fms * 1e-3) / 1e9}
        # point correction: 2M sparse-map points, each referencing a random pixel
        gen = torch.Generator(device=dev)
        gen.manual_seed(SEED_CORRECT)
        n_sp = 2_000_000
        refs = torch.randint(0, npts, (n_sp,), generator=gen, device=dev, dtype=torch.int64)
        pts = torch.zeros((n_sp, 3), device=dev)
        ncor = torch.zeros((1,), dtype=torch.int64, device=dev)
        cms = _time(lambda: ctx.correct_points(pts, refs, xyz, conf, poses, threshold=1.0,
                                               n_corrected=ncor), 5)
        assert ctx.sync_status() == 0
        err["fusion"], err["point_correction"] = map_fusion_error(xyz, conf, ox, oi, pts, refs)
        out["oracle_error"] = err
        out["point_correction"] = {"points": n_sp, "ms": cms,
                                   "points_per_s": n_sp / (cms * 1e-3),
                                   "note": "random references: 16 B gathered per point"}
    elif args.workload == "pg1000":
        # config 5's pose graph alone: 1000 nodes, 999 odometry + 300 loop edges,
        # chaining + 10 Gauss-Newton iterations (block Cholesky with the
        # minimum-degree ordering and the dense trailing supernode)
        M = 1000
        g = synth.make_pose_graph(synth.SEED_BASE + 5, M, 300, device="cpu")
        Tij = ec3r.sim3_rows(g.T_meas.s, g.T_meas.R, g.T_meas.t).to(dev)
        nodes = torch.zeros((M, 13), dtype=torch.float64, device=dev)
        nodes[:, 0] = 1.0
        nodes[:, [1, 5, 9]] = 1.0
        pg_ms = _time(lambda: ctx.pose_graph_correct(nodes, g.ei.numpy(), g.ej.numpy(), Tij,
                                                     iters=10), 5, warm=2)
        assert ctx.sync_status() == 0, ctx.last_error()
        ctx.profile(True)
        ctx.profile_read()
        ctx.pose_graph_correct(nodes, g.ei.numpy(), g.ej.numpy(), Tij, iters=10)
        prof = ctx.profile_read()
        ctx.profile(False)
        out["pose_graph"] = {"nodes": M, "edges": len(g.ei), "gn_iters": 10, "ms": pg_ms,
                             "kernels_ms_event_pass": {k: v[0] for k, v in prof.items()},
                             "launches": {k: v[1] for k, v in prof.items()}}
        if not args.no_oracle:
            out["oracle_error"] = {"pose_graph": pose_graph_error(
                ctx, g.ei.numpy(), g.ej.numpy(), Tij, M, 1)}
    elif args.workload == "depth200":
        # the 200-submap chain given as depth maps + cameras (the paper's submaps
        # are unprojected depths): registration straight from depth, 16 B per
        # correspondence and sweep instead of 32 (d_p, d_q, c_p, c_q); the first
        # sweep also writes each correspondence's weight, which the later sweeps
        # read instead of both confidences (20 B, then 12 B)
        M = args.submaps
        ch = synth.make_depth_chain(synth.SEED_BASE + 46, M=M, F=5, H=294, W=518, device=dev)
        dps = ch.pairs()
        fin = (torch.isfinite(dps.depth) & (dps.depth > 0) & torch.isfinite(dps.conf) &
               (dps.conf > 0)).view(dps.depth.shape[0], -1)
        n = int((fin[dps.src.long()] & fin[dps.tgt.long()]).sum())
        del fin
        S = torch.empty((dps.n_pairs, 13), dtype=torch.float64, device=dev)
        st = torch.empty((dps.n_pairs,), dtype=torch.int32, device=dev)
        ms = _time(lambda: ctx.align_submaps_depth(dps.depth, dps.conf, dps.cams, dps.link_off,
                                                   dps.src, dps.tgt, delta=DELTA, iters=ITERS,
                                                   out=S, status=st), 10)
        assert ctx.sync_status() == 0 and int((st != 0).sum()) == 0
        ks = sorted({0, dps.n_pairs // 2, dps.n_pairs - 1})
        out["oracle_error"] = {"registration": registration_error(
            S, st, [_host_depth_pair(dps, k) for k in ks], ks)}
        ctx.profile(True)
        ctx.profile_read()
        ctx.align_submaps_depth(dps.depth, dps.conf, dps.cams, dps.link_off, dps.src, dps.tgt,
                                delta=DELTA, iters=ITERS, out=S, status=st)
        prof = ctx.profile_read()
        ctx.profile(False)
        sw = prof["depth_sweep"]
        sweep_ms = sw[0] / sw[1]
        px = int(dps.link_off[-1]) * dps.H * dps.W
        bpp = (20.0 + 12.0 * (ITERS - 1)) / ITERS   # mean bytes per pixel and sweep
        achieved = bpp * px / (sweep_ms * 1e-3) / 1e9
        out["registration"] = {"pairs": dps.n_pairs, "valid": n, "ms": ms,
                               "pt_iter_per_s": n * ITERS / (ms * 1e-3),
                               "sweep_ms": sweep_ms, "sweep_bytes_per_pixel": bpp,
                               "sweep_gbs": achieved, "sweep_frac_of_peak": achieved / peak,
                               "sweep_gbs_at_16B_per_pixel": 16.0 * px / (sweep_ms * 1e-3) / 1e9,
                               "kernels": {k: v[0] for k, v in prof.items()}}
        # fusion of every frame straight from depth (identity poses)
        npts = dps.depth.numel()
        kept = int(((dps.conf > 1.0) & (dps.depth > 0) & torch.isfinite(dps.depth)).sum())
        ox = torch.empty((kept, 3), device=dev)
        oi = torch.empty((kept,), dtype=torch.int64, device=dev)
        cur = torch.zeros((1,), dtype=torch.int64, device=dev)
        poses = torch.zeros((M, 13), dtype=torch.float64, device=dev)
        poses[:, 0] = 1.0
        poses[:, [1, 5, 9]] = 1.0

        def fuse():
            cur.zero_()
            ctx.fuse_points_depth(dps.depth, dps.conf, dps.cams, poses, ox, oi, cur, frames=5)
        fms = _time(fuse, 5)
        assert ctx.sync_status() == 0 and int(cur) == kept
        out["fusion"] = {"points": npts, "kept": kept, "ms": fms,
                         "gbs_at_16B_plus_20B_per_kept":
                             (16.0 * npts + 20.0 * kept) / (fms * 1e-3) / 1e9,
                         # the bytes moved: the count reads depth and confidence
                         # and writes a 1-bit keep mask; the scatter reads the
                         # depth and the mask and writes 20 B per kept point
                         "gbs": ((12.25 * npts + 20.0 * kept) / (fms * 1e-3) / 1e9),
                         "bytes_per_point_read": 12.25}
    elif args.workload == "loops32k":
        # global loop retrieval over 32,768 keyframe embeddings of 1,024 dimensions
        # (two laps of a 1.6 km route, a keyframe every 0.1 m), every 2nd keyframe
        # in the BF16 tensor-core similarity matrix
        n, d, stride = args.keyframes, 1024, 2
        E = synth.make_keyframe_embeddings(synth.SEED_BASE + 62, n=n, d=d, device=dev)
        kw = dict(stride=stride, radius=2, gap=n // 5, tau_global=0.93, tau_local=0.96,
                  capacity=1 << 18)
        ms = _time(lambda: ctx.loop_candidates(E, **kw), 5)
        assert ctx.sync_status() == 0
        ctx.profile(True)
        ctx.profile_read()
        rows, scores, counts, _ = ctx.loop_candidates(E, **kw)
        prof = ctx.profile_read()
        ctx.profile(False)
        m = (n + stride - 1) // stride
        side = (m + 127) // 128
        tiles = side * (side + 1) // 2
        flops = 2.0 * tiles * 128 * 128 * d      # the 128 x 128 blocks meeting the upper triangle
        tc_ms = prof["loop_sim_tc"][0]
        bf16_peak = 1800.0
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak = float(json.load(f)["bf16_tflops"])
        except Exception:
            pass
        out["loop_retrieval"] = {
            "keyframes": n, "dim": d, "stride": stride, "coarse_pairs": int(counts[0]),
            "candidates": int(counts[1]), "ms": ms,
            "kernels_ms": {k: v[0] for k, v in prof.items()},
            "similarity_tflops": flops / (tc_ms * 1e-3) / 1e12,
            "similarity_frac_of_bf16_peak": flops / (tc_ms * 1e-3) / 1e12 / bf16_peak,
            "bf16_peak_tflops": bf16_peak}
        out["oracle_error"] = similarity_error(ctx, E, kw)
    out["peak_gbs"] = peak
    out["peak_kind"] = peak_kind
    if not args.no_oracle:
        out["cpu_baseline"] = oracle_workload(args.workload)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--workload", default="chain200",
                    choices=["chain200", "pair1", "loops512", "adjoint1", "map1000",
                             "pg1000", "depth200", "loops32k"],
                    help="chain200 is the benchmark; the others measure the other workloads")
    ap.add_argument("--bwd-ctas-per-sm", type=int, default=0,
                    help="CTAs per SM of the backward's reduction sweeps in the step "
                         "(0: one CTA per tile)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="leave the adjoint out of the step (profiling only)")
    ap.add_argument("--submaps", type=int, default=M_SUBMAPS,
                    help="chain length (default 200); smaller values are for profiling only")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="weak (default): every rank registers and fuses its own chain; "
                         "strong: one map split over the ranks")
    ap.add_argument("--variant", type=int, default=-1,
                    help="force registration sweep variant V (default: chosen by timing)")
    ap.add_argument("--loop-pairs", type=int, default=512,
                    help="pairs of loops512 (default 512); smaller values are for profiling "
                         "only")
    ap.add_argument("--keyframes", type=int, default=32768,
                    help="keyframes of loops32k (default 32768); smaller values are for "
                         "profiling only")
    ap.add_argument("--oracle-workload", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-oracle", action="store_true",
                    help="other workloads: leave out the oracle timing on a sample")
    args = ap.parse_args()
    if args.oracle_workload:
        print(json.dumps(_oracle_workload_inproc(args.oracle_workload)))
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "chain200":
        run_workload(args)
    elif args.scaling == "strong":
        run_strong(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
