"""Throughput of the segmented-Quickhull hot path on GB300.

Workload (one step): the convex hulls of three seeded 16M-point float32
clouds in the plane (uniform in the unit square, uniform in the unit disk,
on the unit circle with N(0, 1e-4) radial jitter), FP32-filtered exact
predicates, the three hulls in one persistent launch (qh_hull2d_multi; the
same clouds as three single-cloud launches are reported beside it).  value =
points hulled per second over the whole job (Mpoints/s), inputs resident in
HBM.

Also reported: the 3D hull (8M points in the ball, 1M on the sphere) with the
FP32 filter and with FP64 predicates; the batched 3D hull (4096 clouds in one
graph-replayed launch); the differentiable hulls (forward and hand-written
backward, bwd/fwd); selection (medians) on the segmented primitives; the
CPU/GPU switchover of one 2D hull; the plain GPU path (FP64 predicates,
host-driven loop with a live-count readback per iteration); the end-to-end
number through the C ABI with host buffers; the HBM roofline of the
persistent kernel; and the CPU oracle on the host cores.  `--impl reference`
times the oracle alone.

Multi-GPU (torchrun, one rank per GPU): every rank hulls its own clouds
(independent problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hull Mpoints/s (2D, 3D, batched) vs plain GPU path; % HBM roofline; bwd/fwd"
UNIT = "Mpoints/s"
N_PER_CLOUD = 16 * 1024 * 1024
WORKLOAD = ("2D at scale: 3 x 16M float32 points (uniform unit square, uniform unit disk, "
            "unit circle with N(0,1e-4) radial jitter), FP32-filtered exact predicates, "
            "the three hulls in one persistent launch")
# DRAM bytes (read + write) per algorithmic byte of the persistent 2D kernel
# (all clouds in one launch) from one ncu capture of a smaller case (3 clouds
# x 8M points, profiles/qh2d_multi_traffic_3x8M.md), keyed by the hash of the
# kernel's sources it was taken on; the bench scales it by its own
# algorithmic bytes per launch.  Absent (traffic null) for any other source
# state.
NCU_TRAFFIC = {"08104a037af05474": 1995.04 / 2164.09}


KERNEL_2D_SOURCES = ("qh2d.cu", "pred2.cuh", "qh_common.cuh")


def _code_only(src: str) -> str:
    """The source without comments and blank space (what the compiler sees)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_sources_sha() -> str:
    """Hash of the code (comments and spacing ignored) of the sources the
    persistent 2D kernels are built from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1201_2936_gb300", "csrc")
    for fn in KERNEL_2D_SOURCES:
        with open(os.path.join(d, fn), encoding="utf-8") as f:
            h.update(fn.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def clouds(rank: int, n: int):
    from paper_1201_2936_gb300 import workloads as w
    s = w.SEED_BASE + 1 + 1000 * rank
    return [("square", w.uniform_square(n, s)),
            ("disk", w.uniform_disk(n, s + 10)),
            ("circle1e-4", w.circle_jitter(n, s + 20, 1e-4))]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"qh_clocks_gpu{self.gpu}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def oracle_step(data, limit=None):
    import oracle
    t0 = time.perf_counter()
    pts = 0
    for _, (x, y) in data:
        if limit:
            x, y = x[:limit], y[:limit]
        oracle.hull2d(x, y)
        pts += len(x)
    return pts, time.perf_counter() - t0


def clouds_3d(rank: int, scale: int = 1):
    from paper_1201_2936_gb300 import workloads as w
    s = w.SEED_BASE + 2 + 1000 * rank
    return [("ball8M", w.uniform_ball(w.N_BALL_3D // scale, s)),
            ("sphere1M", w.on_sphere(w.N_SPHERE_3D // scale, s + 10)),
            ("nearsphere8M", w.near_sphere(w.N_BALL_3D // scale, s + 20, 1e-4))]


def bench_3d(args, qh, dev, rank, peak, peak_kind):
    """Per-cloud device time of qh_hull3d (extrema to canonical faces, host
    readbacks of the output sizes included) with the FP32 filter and with
    FP64 predicates.  Algorithmic bytes: 12 B per point for the extrema and
    the first split's read, 16 B (x, y, z, idx) per live point read and per
    survivor written afterwards."""
    import torch
    reps = max(3, args.steps // 10)
    out = []
    for name, (x, y, z) in clouds_3d(rank, args.scale_3d):
        n = len(x)
        P = torch.from_numpy(np.stack([x, y, z])).to(dev)
        ws = qh.Workspace(dev)
        row = {"cloud": name, "n": n}
        verts = {}
        for pred in ("f32", "f64"):
            for _ in range(2):
                (v, off, idx), r = qh.hull3d(P, pred=pred, workspace=ws, return_result=True)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
            torch.cuda.synchronize()
            e[0].record()
            for k in range(reps):
                qh.hull3d(P, pred=pred, workspace=ws)
                e[k + 1].record()
            torch.cuda.synchronize()
            ms = statistics.median(e[k].elapsed_time(e[k + 1]) for k in range(reps))
            verts[pred] = (v.cpu(), off.cpu(), idx.cpu())
            algo = 24 * n + 32 * r["survivor_total"]
            row[pred] = {"ms": round(ms, 3), "Mpoints_s": round(n / ms / 1e3, 1),
                         "iterations": r["iterations"], "algo_bytes": algo,
                         "GBps": round(algo / (ms / 1e3) / 1e9, 1),
                         "frac": round(algo / (ms / 1e3) / 1e9 / peak, 4),
                         "fallback_frac": r["filter_fallbacks"] / max(1, r["live_total"]),
                         "exact_argmax_segments": r["exact_argmax"]}
        a, b = verts["f32"], verts["f64"]
        row["hull_vertices"] = int(a[0].numel())
        row["faces"] = int(a[1].numel() - 1)
        row["same_hull_f32_f64"] = all(torch.equal(p, q) for p, q in zip(a, b))
        row["speedup_f32_over_f64"] = round(row["f64"]["ms"] / row["f32"]["ms"], 2)
        out.append(row)
        del P, ws
        torch.cuda.empty_cache()
    return {"workload": "3D: 8M uniform in the unit ball, 1M on the unit sphere, 8M near the "
                        "unit sphere (radius 1 + 1e-4 N(0,1)) (float32)",
            "peak": peak, "peak_kind": peak_kind, "reps": reps, "clouds": out}


def bench_4d(args, qh, dev, rank, peak, peak_kind):
    """The 4D hull (qh_hull4d, host-driven iterations): device time per call
    on 1M points uniform in the 4-ball and 100K near the 3-sphere.
    Algorithmic bytes: 16 B per point for the extrema and first-assignment
    reads, 20 B (x, y, z, w, index) per live point read and per survivor
    written afterwards."""
    import torch
    from paper_1201_2936_gb300 import workloads as w
    s = w.SEED_BASE + 7 + 1000 * rank
    out = []
    for name, pts in (("ball4d_1M", w.uniform_ball_4d(1 << 20, s)),
                      ("nearsphere4d_100K", w.near_sphere_4d(100_000, s + 1, 1e-3))):
        n = len(pts[0])
        P = torch.from_numpy(np.stack(pts)).to(dev)
        ws = qh.Workspace(dev)
        for _ in range(2):
            (v, off, idx), r = qh.hull4d(P, workspace=ws, return_result=True)
        reps = 3
        e = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        torch.cuda.synchronize()
        e[0].record()
        for k in range(reps):
            qh.hull4d(P, workspace=ws)
            e[k + 1].record()
        torch.cuda.synchronize()
        ms = statistics.median(e[k].elapsed_time(e[k + 1]) for k in range(reps))
        algo = 32 * n + 40 * r["survivor_total"]
        out.append({"cloud": name, "n": n, "ms": round(ms, 3), "Mpoints_s": round(n / ms / 1e3, 1),
                    "iterations": r["iterations"], "vertices": int(v.numel()),
                    "facets": int(off.numel() - 1), "algo_bytes": algo,
                    "frac": round(algo / (ms / 1e3) / 1e9 / peak, 4),
                    "fallback_frac": r["filter_fallbacks"] / max(1, r["live_total"])})
        del P, ws
        torch.cuda.empty_cache()
    return {"workload": "4D: 1M uniform in the unit 4-ball, 100K near the unit 3-sphere (float32)",
            "loop": "host-driven (one launch per phase, sizes read back each iteration)",
            "peak": peak, "peak_kind": peak_kind, "clouds": out}


def bench_batched(args, qh, dev, rank, peak, peak_kind):
    """The batched 3D workload: 4096 anisotropic Gaussian clouds (sizes
    log-uniform in [16, 65536]) in one persistent launch, launch shape from
    the autotuner, replayed from a CUDA graph; against it the plain path (one
    FP64 qh_hull3d call per cloud, host-synchronised) on the first clouds."""
    import torch
    from paper_1201_2936_gb300 import workloads as w
    x, y, z, off = w.batched_clouds_3d(args.batch_clouds, w.SEED_BASE + 3 + 1000 * rank)
    n = len(x)
    P = torch.from_numpy(np.stack([x, y, z])).to(dev)
    O = torch.from_numpy(off).to(dev)
    b = qh.Hull3DBatch(P, cloud_off=O)
    table = b.tune(reps=2)
    b.capture()
    reps = max(5, args.steps // 5)
    for _ in range(3):
        b.replay()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    e[0].record()
    for k in range(reps):
        b.replay()
        e[k + 1].record()
    torch.cuda.synchronize()
    ms = statistics.median(e[k].elapsed_time(e[k + 1]) for k in range(reps))
    r = b.result_dict()
    st = b.cloud_status.cpu().numpy()
    # the same batch enqueued directly (no graph)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.enqueue()
    e1.record()
    torch.cuda.synchronize()
    ms_direct = e0.elapsed_time(e1) / reps
    algo = 24 * n + 32 * r["survivor_total"]
    out = {"workload": f"{args.batch_clouds} clouds, sizes log-uniform in [16, 65536], "
                       "anisotropic Gaussian, float32",
           "points": n, "ms": round(ms, 3), "Mpoints_s": round(n / ms / 1e3, 1),
           "ms_without_graph": round(ms_direct, 3), "iterations": r["iterations"],
           "hull_vertices": r["extra"][0], "faces": r["extra"][1],
           "clouds_ok": int((st == 0).sum()),
           "algo_bytes": algo, "GBps": round(algo / (ms / 1e3) / 1e9, 1),
           "frac": round(algo / (ms / 1e3) / 1e9 / peak, 4), "peak_kind": peak_kind,
           "fallback_frac": r["filter_fallbacks"] / max(1, r["live_total"]),
           "tuned": {"block": b.opts.block, "items": b.opts.items,
                     "ctas_per_sm": b.opts.blocks_per_sm, "small_cloud": b.opts.small_cloud},
           "tune_table_ms": [[bl, it, c, sc, round(t, 3)] for bl, it, c, sc, t in table]}
    # the switchover: the tuned launch with and without the small-cloud route
    # (clouds of at most small_cloud points hulled whole by one warp)
    sc_rows = {int(sc): round(t, 3) for bl, it, c, sc, t in table
               if (bl, it, c) == (b.opts.block, b.opts.items, b.opts.blocks_per_sm)}
    out["small_cloud_route"] = {
        "what": "batched 3D: clouds of 4..threshold points hulled whole by one warp in the "
                "setup, the rest by the segmented iterations; threshold chosen by the autotuner",
        "threshold_ms": sc_rows, "chosen": int(b.opts.small_cloud),
        "clouds_on_route": int(((np.diff(off) >= 4) & (np.diff(off) <= b.opts.small_cloud)).sum())
        if b.opts.small_cloud > 0 else 0}
    # the switchover on a batch of many small clouds (32768 clouds, sizes
    # log-uniform in [16, 256]): tuned launch, route on and off
    xs, ys, zs, offs = w.batched_clouds_3d(32768, w.SEED_BASE + 13 + 1000 * rank, nmin=16,
                                           nmax=256)
    Ps = torch.from_numpy(np.stack([xs, ys, zs])).to(dev)
    Os = torch.from_numpy(offs).to(dev)
    bs = qh.Hull3DBatch(Ps, cloud_off=Os)
    stab = bs.tune(reps=2)
    sc_small = {int(sc): round(t, 3) for bl, it, c, sc, t in stab
                if (bl, it, c) == (bs.opts.block, bs.opts.items, bs.opts.blocks_per_sm)}
    out["small_cloud_route"]["many_small_clouds"] = {
        "workload": "32768 clouds, sizes log-uniform in [16, 256], anisotropic Gaussian",
        "points": int(len(xs)), "threshold_ms": sc_small, "chosen": int(bs.opts.small_cloud),
        "speedup_of_route": round(sc_small.get(0, 0.0) /
                                  max(1e-9, sc_small.get(int(bs.opts.small_cloud), 1.0)), 2)}
    del bs, Ps, Os
    # plain path on a bounded sample of clouds
    ns = min(args.batch_clouds, args.plain_clouds)
    ws = qh.Workspace(dev)
    pts = 0
    torch.cuda.synchronize()
    e0.record()
    for c in range(ns):
        a, bb = int(off[c]), int(off[c + 1])
        if bb - a >= 4:
            qh.hull3d(P[:, a:bb], pred="f64", workspace=ws)
        pts += bb - a
    e1.record()
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1)
    out["plain_gpu"] = {"Mpoints_s": round(pts / pms / 1e3, 2), "clouds": ns, "points": pts,
                        "ms": round(pms, 2),
                        "pred": "f64-filter+exact", "calls": "one synchronous qh_hull3d per cloud",
                        "speedup_of_batched": round((n / ms) / (pts / pms), 1)}
    del b, P, O, ws
    torch.cuda.empty_cache()
    return out


def _time(fn, reps):
    import torch
    for _ in range(2):
        fn()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    e[0].record()
    for k in range(reps):
        fn()
        e[k + 1].record()
    torch.cuda.synchronize()
    return statistics.median(e[k].elapsed_time(e[k + 1]) for k in range(reps))


def bench_diff(args, qh, dev, rank):
    """Differentiable hulls: forward = batched hull + FP64 measures, backward
    = the hand-written gradient kernel, both timed on the device (CUDA
    events), for 1024 clouds x 4096 points in the disk (perimeter + area)
    and 256 clouds x 16384 points in the ball (area + volume)."""
    import torch
    from paper_1201_2936_gb300 import workloads as w
    reps = max(5, args.steps // 5)
    out = []
    x, y, off = w.batched_disk_2d(1024, 4096, w.SEED_BASE + 4 + 1000 * rank)
    x3, y3, z3, off3 = w.batched_ball_3d(256, 16384, w.SEED_BASE + 5 + 1000 * rank)
    for dim, pts, o in ((2, np.stack([x, y]), off), (3, np.stack([x3, y3, z3]), off3)):
        P = torch.from_numpy(pts).to(dev)
        O = torch.from_numpy(o).to(dev)
        nc = len(o) - 1
        b = (qh.Hull2DBatch(P, None, O) if dim == 2 else qh.Hull3DBatch(P, None, None, O))
        meas = torch.empty(nc, 2, dtype=torch.float64, device=dev)
        gm = torch.ones(nc, 2, dtype=torch.float64, device=dev)
        grad = torch.empty_like(P)

        def fwd():
            b.enqueue()
            b.measures(meas)

        fwd_ms = _time(fwd, reps)
        bwd_ms = _time(lambda: b.backward(gm, grad), reps)
        # the same through autograd (host round trip for the status check included)
        Pg = P.clone().requires_grad_(True)
        f = qh.hull_measures_2d if dim == 2 else qh.hull_measures_3d

        def step():
            m = f(Pg, O)
            m.sum().backward()
            Pg.grad = None

        step()  # first use of the autograd engine
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ag_ms = (time.perf_counter() - t0) / 3 * 1e3
        # the plain per-cloud path: one FP64-predicate batch of one cloud per
        # call (hull, measures, backward), synchronised per cloud, on the
        # first clouds; its gradients against the fast path's
        npl = min(nc, 256 if dim == 2 else 64)
        grad_fast = grad.clone()
        b.enqueue()
        b.measures(meas)
        b.backward(gm, grad_fast)
        one = torch.tensor([0, 0], dtype=torch.int64, device=dev)
        plain = []
        for c in range(npl):
            a, e = int(o[c]), int(o[c + 1])
            O1 = one.clone()
            O1[1] = e - a
            pb = (qh.Hull2DBatch(P[:, a:e], None, O1, pred="f64") if dim == 2 else
                  qh.Hull3DBatch(P[:, a:e], None, None, O1, pred="f64"))
            plain.append((pb, torch.empty(1, 2, dtype=torch.float64, device=dev),
                          torch.empty(dim, e - a, dtype=torch.float32, device=dev), a, e))
        gm1 = torch.ones(1, 2, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for pb, m1, g1, _, _ in plain:
            pb.enqueue()
            pb.measures(m1)
            pb.backward(gm1, g1)
            torch.cuda.synchronize()
        plain_ms = (time.perf_counter() - t0) * 1e3
        npts = int(o[npl])
        gerr, merr = 0.0, 0.0
        for c, (pb, m1, g1, a, e) in enumerate(plain):
            gf = grad_fast[:, a:e].double()
            den = max(float(gf.abs().max()), 1e-30)
            gerr = max(gerr, float((g1.double() - gf).abs().max()) / den)
            merr = max(merr, float(((m1[0] - meas[c]).abs() / meas[c].abs().clamp_min(1e-300)).max()))
        fast_per_pt = fwd_ms + bwd_ms
        n = pts.shape[1]
        plain_rec = {"clouds": npl, "points": npts, "ms": round(plain_ms, 3),
                     "Mpoints_s": round(npts / plain_ms / 1e3, 2),
                     "how": "per cloud: one FP64-predicate hull, measures and backward, "
                            "synchronised (host timer)",
                     "fast_Mpoints_s_fwd_bwd": round(n / fast_per_pt / 1e3, 1),
                     "speedup_of_fast_path": round((plain_ms / npts) / (fast_per_pt / n), 1),
                     "max_rel_grad_diff": gerr, "max_rel_measure_diff": merr}
        del plain
        out.append({"workload": (f"2D: {nc} clouds x {n // nc} points in the disk, "
                                 "loss = sum of perimeters + areas") if dim == 2 else
                                (f"3D: {nc} clouds x {n // nc} points in the ball, "
                                 "loss = sum of volumes + surface areas"),
                    "fwd_ms": round(fwd_ms, 3), "bwd_ms": round(bwd_ms, 3),
                    "bwd_over_fwd": round(bwd_ms / fwd_ms, 4),
                    "fwd_Mpoints_s": round(n / fwd_ms / 1e3, 1),
                    "autograd_step_ms": round(ag_ms, 3), "plain_gpu": plain_rec})
        del b, P, O
        torch.cuda.empty_cache()
    return out


def bench_select(args, qh, dev, rank, peak, peak_kind):
    """Selection on the segmented primitives (Section 6): the median of each
    of 4096 segments of 4096 float32 values (16.7M values), a 3-state split
    around each segment's pivot and a compaction of the kept part per round.
    The persistent form (all rounds in one launch) against the round-by-round
    host loop, and against the plain definition (sort per segment) on the
    host for the first 256 segments.  L2 is flushed before every timed call
    (the values are 67 MB, below L2)."""
    import torch
    import oracle
    rng = np.random.default_rng(1207 + 1000 * rank)
    nseg, L = 4096, 4096
    v = rng.standard_normal(nseg * L).astype(np.float32)
    off = np.arange(nseg + 1, dtype=np.int64) * L
    k = np.full(nseg, L // 2 - 1, np.int64)
    V, O, K = (torch.from_numpy(a).to(dev) for a in (v, off, k))
    out, iters = qh.select(V, O, K, return_iters=True)
    host_out, host_iters = qh.select(V, O, K, return_iters=True, loop="host")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    reps = max(5, args.steps // 10)

    def timed(loop):
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            qh.select(V, O, K, loop=loop)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    ms = timed("device")
    ms_host = timed("host")
    ns = 256
    t0 = time.perf_counter()
    want = oracle.select(v[: ns * L], off[: ns + 1], k[:ns])
    cpu_s = time.perf_counter() - t0
    same = out[:ns].cpu().numpy().tolist() == want.tolist()
    # algorithmic bytes: every value read once, the offsets and ranks read,
    # the answers written
    algo = 4 * nseg * L + 8 * (nseg + 1) + 8 * nseg + 4 * nseg
    gbps = algo / (ms * 1e-3) / 1e9
    return {"workload": "median of each of 4096 segments x 4096 float32 values",
            "ms": round(ms, 3), "Melements_s": round(nseg * L / ms / 1e3, 1), "rounds": iters,
            "loop": "device (one persistent launch, no readback between rounds)",
            "timing": "CUDA events around the synchronous call (launch and status readback "
                      "included), median of %d, L2 flushed before each" % reps,
            "algo_bytes": algo, "GBps": round(gbps, 1), "peak": peak, "peak_kind": peak_kind,
            "frac": round(gbps / peak, 4),
            "host_loop": {"ms": round(ms_host, 3), "rounds": host_iters,
                          "loop": "host (kept count read back each round)",
                          "same_result": host_out.cpu().tolist() == out.cpu().tolist(),
                          "speedup_of_device_loop": round(ms_host / ms, 2)},
            "matches_definition_first_256_segments": same,
            "cpu_definition_Melements_s": round(ns * L / cpu_s / 1e6, 2),
            "cpu_sample": "first 256 segments, numpy lexsort per segment, 1 thread"}


def bench_switchover(args, qh, dev):
    """CPU/GPU switchover (Section 6's open question), per dimension: wall
    time of one synchronous hull call through the C ABI (device-resident
    points) against the oracle on the host, over n; the smallest n from which
    the GPU call is faster.  (Inside a batch the switchover is the small-cloud
    route's threshold, reported with the batched workload.)"""
    import torch
    import oracle
    from paper_1201_2936_gb300 import workloads as w
    ws = qh.Workspace(dev)

    def sweep(sizes, gen, gpu, cpu):
        rows, cross = [], None
        for n in sizes:
            pts = gen(n)
            P = torch.from_numpy(np.stack(pts)).to(dev)
            for _ in range(2):
                gpu(P)
            reps = 10
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                gpu(P)
            torch.cuda.synchronize()
            g = (time.perf_counter() - t0) / reps * 1e6
            reps_c = max(1, min(20, 1_000_000 // n))
            t0 = time.perf_counter()
            for _ in range(reps_c):
                cpu(*pts)
            c = (time.perf_counter() - t0) / reps_c * 1e6
            rows.append({"n": n, "gpu_us": round(g, 1), "cpu_oracle_us": round(c, 1)})
            if cross is None and g < c:
                cross = n
        return rows, cross

    out = {"note": "GPU: one synchronous call incl. launch and result readback; CPU: the exact "
                   "FP64 oracle, one thread"}
    r2, c2 = sweep((64, 256, 1024, 4096, 16384, 65536, 262144, 1048576),
                   lambda n: w.uniform_disk(n, 1208 + n),
                   lambda P: qh.hull2d(P, workspace=ws), oracle.hull2d)
    out["2d"] = {"workload": "uniform disk", "rows": r2, "gpu_faster_from_n": c2}
    r3, c3 = sweep((64, 256, 1024, 4096, 16384, 65536, 262144),
                   lambda n: w.uniform_ball(n, 1218 + n),
                   lambda P: qh.hull3d(P, workspace=ws), oracle.hull3d)
    out["3d"] = {"workload": "uniform ball", "rows": r3, "gpu_faster_from_n": c3}
    r4, c4 = sweep((64, 256, 1024, 4096, 16384, 65536),
                   lambda n: w.uniform_ball_4d(n, 1228 + n),
                   lambda P: qh.hull4d(P, workspace=ws), oracle.hull4d)
    out["4d"] = {"workload": "uniform 4-ball", "rows": r4, "gpu_faster_from_n": c4}
    return out


def run_reference(args, ws, rank):
    # the oracle on the host cores, rank 0 only
    if rank != 0:
        return 0
    sample = int(os.environ.get("QH_REF_SAMPLE", 2 * 1024 * 1024))
    data = clouds(0, N_PER_CLOUD)
    for _ in range(args.warmup):
        oracle_step(data, sample)
    tot_pts, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, t = oracle_step(data, sample)
        tot_pts += p
        tot_t += t
    value = tot_pts / tot_t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_points_per_cloud": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {sample} points of each of the 3 clouds per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_PER_CLOUD,
                    help="points per cloud (profiling of smaller cases)")
    ap.add_argument("--only", default="", help="comma-separated cloud names to keep")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-4d", action="store_true")
    ap.add_argument("--independent", action="store_true",
                    help="N > 1: every rank hulls its own 3 x 16M set (weak scaling) instead of "
                         "one set sharded over the ranks")
    ap.add_argument("--sharded", action="store_true",
                    help="the sharded path also at N = 1 (one rank; the exchange is a copy)")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-select", action="store_true")
    ap.add_argument("--no-switchover", action="store_true")
    ap.add_argument("--batch-clouds", type=int, default=4096)
    ap.add_argument("--plain-clouds", type=int, default=256,
                    help="clouds timed on the per-cloud plain path")
    ap.add_argument("--scale-3d", type=int, default=1, help="divide the 3D cloud sizes")
    ap.add_argument("--timeline", action="store_true",
                    help="print the per-iteration device timeline of each cloud to stderr")
    ap.add_argument("--sections", default="",
                    help="comma-separated subset of 3d,4d,batched,diff,select,switchover,plain,e2e,cpu to run "
                         "besides the 2D headline (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.sections:
        keep = set(args.sections.split(","))
        args.no_3d = "3d" not in keep
        args.no_batched = "batched" not in keep
        args.no_4d = "4d" not in keep
        args.no_diff = "diff" not in keep
        args.no_select = "select" not in keep
        args.no_switchover = "switchover" not in keep
        args.no_plain = "plain" not in keep
        args.no_e2e = "e2e" not in keep
        args.no_cpu_baseline = "cpu" not in keep

    ws, rank = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist

    import paper_1201_2936_gb300 as qh
    from paper_1201_2936_gb300 import build as qbuild

    if (ws > 1 and not args.independent) or args.sharded:
        return run_sharded(args, ws, rank)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl")
        if local == 0:
            qbuild.build()
        dist.barrier()
    else:
        qbuild.build()

    ncl = args.n
    data = clouds(rank, ncl)
    if args.only:
        keep = set(args.only.split(","))
        data = [d for d in data if d[0] in keep]
    stream = torch.cuda.current_stream()
    dev_pts = [torch.from_numpy(np.stack([x, y])).to(dev) for _, (x, y) in data]
    outs = [torch.empty(ncl, dtype=torch.int32, device=dev) for _ in data]
    results = [torch.zeros(qh.RESULT_BYTES, dtype=torch.uint8, device=dev) for _ in data]
    wss = [qh.Workspace(dev) for _ in data]
    opts = qh.make_opts("f32", "persistent")

    # the headline: every cloud of the step in one persistent launch
    # (qh_hull2d_multi: the clouds share the segment table, the passes and the
    # grid barriers)
    mres = torch.zeros(len(data) * qh.RESULT_BYTES, dtype=torch.uint8, device=dev)
    mws = qh.Workspace(dev)
    nl = len(dev_pts)

    def step():
        qh.hull2d_multi_async(dev_pts, outs, mres, mws, opts)

    def mresults():
        return [qh.result_from_tensor(mres[i * qh.RESULT_BYTES:(i + 1) * qh.RESULT_BYTES])
                for i in range(nl)]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for r in mresults():
        if r.status != 0:
            raise SystemExit(f"hull failed: {qh.status_str(r.status)}")

    # ---- timed region: K steps (one launch each), events per launch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    launch_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    res = mresults()
    # the headline's hulls, index for index, for the comparisons below
    head_idx = [outs[i][: res[i].count].clone() for i in range(nl)]
    # per-pass HBM rate of the last timed launch (device clock between the
    # pass's grid barriers): pass t reads its L_t live records (the first
    # split: the callers' 8-byte coordinates) and writes its survivors, the
    # L_{t+1} records of the next pass, 12 bytes each; listed for passes with
    # at least half a cloud's worth of live points
    passes = []
    rows = qh.debug_timeline_2d(mws, nl * ncl + 2 * nl)
    if args.timeline:
        print("# timeline (all clouds): iter L S pass_us update_us", file=sys.stderr)
        for r in rows:
            print(f"#   {r[0]:3d} {r[1]:10d} {r[2]:7d} {r[3] / 1e3:9.2f} "
                  f"{r[4] / 1e3:8.2f}", file=sys.stderr)
    for t, r in enumerate(rows):
        L_t, ns = int(r[1]), int(r[3])
        if L_t < ncl // 2 or ns <= 0:
            continue
        S_t = int(rows[t + 1][1]) if t + 1 < len(rows) else 0
        b = (8 if t == 0 else 12) * L_t + 12 * S_t
        passes.append({"iter": t, "live": L_t, "written": S_t, "us": round(ns / 1e3, 2),
                       "GBps": round(b / ns, 1)})
    pts_per_step = nl * ncl
    value = ws * pts_per_step * args.steps / (total_ms / 1e3) / 1e6

    # ---- roofline of the persistent kernel (algorithmic bytes per launch:
    # every cloud's extrema and first-split reads, 16 bytes a point, and 24
    # bytes per survivor of every pass, written once and read once)
    peak, peak_kind = measured_peak()
    r0 = res[0]
    algo = 16 * pts_per_step + 24 * r0.survivor_total
    ms = statistics.mean(launch_ms)
    achieved = algo / (ms / 1e3) / 1e9
    per_cloud = [{"cloud": name, "hull": res[i].count, "status": res[i].status}
                 for i, (name, _) in enumerate(data)]
    sha = kernel_sources_sha()
    ratio = NCU_TRAFFIC.get(sha)
    traffic = round(ratio * algo) if ratio else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "frac_of_nominal_8TBps": round(achieved / 8000.0, 4),
                "traffic": traffic, "kernel": "qh2d_multi<PredF32>",
                "algo_bytes_per_launch": algo, "iterations": r0.iterations,
                "fallback_frac": r0.filter_fallbacks / max(1, r0.live_total),
                "exact_argmax_segments": r0.exact_argmax,
                "phase_us": {"pass": r0.extra[0] / 1e3, "update": r0.extra[1] / 1e3,
                             "exact": r0.extra[2] / 1e3, "other": r0.extra[3] / 1e3}}
    if passes:
        fr = sorted(p["GBps"] / peak for p in passes)
        roofline["large_passes"] = {
            "what": "passes with at least half a cloud's worth of live points: "
                    "(read + written bytes) / device time",
            "n": len(passes), "frac_min": round(fr[0], 4), "frac_median": round(fr[len(fr) // 2], 4),
            "frac_max": round(fr[-1], 4), "passes": passes}

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if ncl == N_PER_CLOUD and not args.only else
                       f"reduced: {nl} cloud(s) x {ncl} points", "points_per_step_per_gpu": pts_per_step,
                       "l2": "inputs larger than L2 (3 x 128 MB of coordinates per step)",
                       "pred": "f32-filter+exact", "loop": "persistent, one launch for all clouds"},
            "per_cloud": per_cloud, "roofline": roofline, "clocks": clocks,
            "gpu_launches": args.steps}

    # ---- the same clouds as separate single-cloud launches (context)
    sepn = max(3, args.steps // 5)
    for i, P in enumerate(dev_pts):
        qh.hull2d_async(P, None, outs[i], results[i], wss[i], opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(sepn):
        for i, P in enumerate(dev_pts):
            qh.hull2d_async(P, None, outs[i], results[i], wss[i], opts)
    e1.record(stream)
    torch.cuda.synchronize()
    sms = e0.elapsed_time(e1) / sepn
    sres = [qh.result_from_tensor(r) for r in results]
    line["separate_launches"] = {
        "value": round(pts_per_step / (sms / 1e3) / 1e6, 2), "unit": UNIT,
        "ms_per_step": round(sms, 3), "kernel": "qh2d_multi<PredF32>, one cloud per launch (qh_hull2d)",
        "same_hulls": all(sres[i].count == res[i].count and
                          torch.equal(outs[i][: sres[i].count], head_idx[i]) for i in range(nl))}

    # ---- plain GPU path: FP64 predicates, host loop with per-iteration readback
    if not args.no_plain:
        popts = qh.make_opts("f64", "host")
        ksteps = max(1, args.steps // 10)
        for i, P in enumerate(dev_pts):
            qh.hull2d_async(P, None, outs[i], results[i], wss[i], popts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ksteps):
            for i, P in enumerate(dev_pts):
                qh.hull2d_async(P, None, outs[i], results[i], wss[i], popts)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / ksteps
        pres = [qh.result_from_tensor(r) for r in results]
        same = all(pres[i].count == res[i].count and
                   torch.equal(outs[i][: pres[i].count], head_idx[i]) for i in range(nl))
        line["plain_gpu"] = {"value": round(pts_per_step / (pms / 1e3) / 1e6, 2), "unit": UNIT,
                             "ms_per_step": round(pms, 3), "pred": "f64-filter+exact",
                             "loop": "host (live count read back every iteration)",
                             "same_hulls": same,
                             "speedup_of_fast_path": round(pms / (total_ms / args.steps), 2)}

    # ---- 3D (8M points uniform in the ball, 1M points on the sphere): FP32
    # filter vs the FP64 plain path, same hulls required
    if not args.no_3d:
        line["hull3d"] = bench_3d(args, qh, dev, rank, peak, peak_kind)

    # ---- 4D (the higher-dimensional extension): 1M in the 4-ball, 100K near the 3-sphere
    if not args.no_4d:
        line["hull4d"] = bench_4d(args, qh, dev, rank, peak, peak_kind)

    # ---- batched 3D: one persistent launch per batch, CUDA graph, autotuned shape
    if not args.no_batched:
        line["batched3d"] = bench_batched(args, qh, dev, rank, peak, peak_kind)

    # ---- differentiable hulls: forward (hull + measures) and backward kernels
    if not args.no_diff:
        line["differentiable"] = bench_diff(args, qh, dev, rank)

    # ---- selection on the segmented primitives
    if not args.no_select:
        line["selection"] = bench_select(args, qh, dev, rank, peak, peak_kind)

    # ---- CPU/GPU switchover, per dimension
    if rank == 0 and not args.no_switchover:
        line["switchover"] = bench_switchover(args, qh, dev)

    # ---- end to end through the C ABI with host buffers: every step copies
    # its clouds from pinned host memory and reads its hulls back; the next
    # step's copy runs on a second stream while the synchronous
    # qh_hull2d_multi call of this step computes (two device input sets)
    if args.no_e2e:
        host_pts = []
    else:
        host_pts = [torch.from_numpy(np.stack([x, y])).pin_memory() for _, (x, y) in data]
    host_out = [torch.empty(ncl, dtype=torch.int32).pin_memory() for _ in host_pts]
    esteps = max(10, args.steps // 5) if host_pts else 0
    h2d = sum(t.numel() * 4 for t in host_pts)
    d2h = 0
    if esteps:
        # (side streams: the legacy default stream would serialise them); the
        # copies run two steps ahead through three input sets, so the link
        # (the bound: ~210 GB/s here) never waits for the host
        NB = 3
        copy_stream = torch.cuda.Stream(device=dev)
        comp = torch.cuda.Stream(device=dev)
        bufs = [[torch.empty_like(hp, device=dev) for hp in host_pts] for _ in range(NB)]
        host_res = torch.empty(nl * qh.RESULT_BYTES, dtype=torch.uint8).pin_memory()
        copied = [torch.cuda.Event() for _ in range(NB)]
        freed = [torch.cuda.Event() for _ in range(NB)]

        def issue_copy(k):
            b = k % NB
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(freed[b])
                for i, hp in enumerate(host_pts):
                    bufs[b][i].copy_(hp, non_blocking=True)
                copied[b].record(copy_stream)

        torch.cuda.synchronize()
        for b in range(NB):
            freed[b].record(comp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(min(NB - 1, esteps)):
            issue_copy(k)
        for k in range(esteps):
            if k + NB - 1 < esteps:
                issue_copy(k + NB - 1)
            b = k % NB
            with torch.cuda.stream(comp):
                comp.wait_event(copied[b])
                qh.hull2d_multi_async(bufs[b], outs, mres, mws, opts, stream=comp)
                freed[b].record(comp)
                host_res.copy_(mres, non_blocking=True)
                comp.synchronize()
                cnts = [qh.QhResult.from_buffer_copy(
                    bytes(host_res[i * qh.RESULT_BYTES:(i + 1) * qh.RESULT_BYTES].numpy())).count
                    for i in range(nl)]
                d2h = host_res.numel()
                for i in range(nl):
                    host_out[i][: cnts[i]].copy_(outs[i][: cnts[i]], non_blocking=True)
                    d2h += cnts[i] * 4
            comp.synchronize()
        torch.cuda.synchronize()
        et = (time.perf_counter() - t0) / esteps
        line["e2e"] = {"value": round(pts_per_step / et / 1e6, 2), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "how": "pinned host -> device copy of each step's clouds (overlapping the "
                              "previous step's hull on a second stream), qh_hull2d_multi_async, "
                              "result records and hull indices read back into pinned memory"}

    # ---- CPU oracle on the host cores (rank 0, bounded sample)
    if rank == 0 and not args.no_cpu_baseline:
        sample = int(os.environ.get("QH_CPU_SAMPLE", 4 * 1024 * 1024))
        p, t = oracle_step(data, sample)
        line["cpu_baseline"] = {"value": round(p / t / 1e6, 3), "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {sample} points of each of the 3 clouds"}
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, ws, rank):
    """N > 1: one hull per cloud of the 3 x 16M set, each cloud split into
    contiguous shards over the ranks (shard.ShardedHull2D: shard hulls in one
    launch, one NCCL all-gather of fixed-size rank blocks, the candidates'
    hulls in one launch).  A rank holds only its shards; the same seeded
    clouds on every rank.  value = all points of the set / max over ranks."""
    import torch
    import torch.distributed as dist

    import paper_1201_2936_gb300 as qh
    from paper_1201_2936_gb300 import build as qbuild
    from paper_1201_2936_gb300 import shard

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    multi = ws > 1

    def barrier():
        if multi:
            dist.barrier()

    def max_over_ranks(v):
        t = torch.tensor([v], device=dev)
        if multi:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    if multi:
        dist.init_process_group("nccl")
    if local == 0:
        qbuild.build()
    barrier()
    ncl = args.n
    data = clouds(0, ncl)
    lo, hi = shard.shard_range(ncl, rank, ws)
    host = [torch.from_numpy(np.stack([x[lo:hi], y[lo:hi]])).pin_memory() for _, (x, y) in data]
    dev_sh = [h.to(dev) for h in host]
    # candidate slots per rank and cloud: above these clouds' shard hulls
    # (at most ~900 vertices); a larger shard hull fails with QH_ERR_CAPACITY
    sh = shard.ShardedHull2D([(t[0], t[1]) for t in dev_sh], [lo] * len(dev_sh), ws, rank,
                             cap=4096)
    for _ in range(args.warmup):
        sh.step()
    hulls, st = sh.results()
    if any(st):
        raise SystemExit(f"sharded hull failed: {st}")
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sh.step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(e0.elapsed_time(e1))
    pts = len(data) * ncl
    value = pts * args.steps / (total_ms / 1e3) / 1e6
    # roofline of this rank's shard launch (the dominant kernel), timed alone
    lres = [qh.result_from_tensor(sh.local_res[c * qh.RESULT_BYTES:(c + 1) * qh.RESULT_BYTES])
            for c in range(len(dev_sh))]
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        sh.local_block()
    e1.record(stream)
    torch.cuda.synchronize()
    lms = e0.elapsed_time(e1) / args.steps
    algo = 16 * (hi - lo) * len(dev_sh) + 24 * lres[0].survivor_total
    peak, peak_kind = measured_peak()
    # end to end: each step copies this rank's shards from pinned host memory
    # and reads the hull records and indices back
    host_res = torch.empty(len(dev_sh) * qh.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    esteps = max(5, args.steps // 5)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(esteps):
        for h, d in zip(host, dev_sh):
            d.copy_(h, non_blocking=True)
        sh.step()
        host_res.copy_(sh.final_res, non_blocking=True)
        torch.cuda.synchronize()
        cnts = [qh.QhResult.from_buffer_copy(bytes(
            host_res[c * qh.RESULT_BYTES:(c + 1) * qh.RESULT_BYTES].numpy())).count
            for c in range(len(dev_sh))]
        idx = [sh.final_out[c][: cnts[c]].cpu() for c in range(len(dev_sh))]
        d2h = host_res.numel() + 4 * sum(cnts)
    torch.cuda.synchronize()
    et = max_over_ranks(time.perf_counter() - t0) / esteps
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + f", each cloud sharded over {ws} ranks",
                       "points_per_step_total": pts, "points_per_step_per_gpu": (hi - lo) * 3,
                       "l2": "inputs larger than L2",
                       "exchange": "one NCCL all-gather of fixed-size rank blocks per step",
                       "pred": "f32-filter+exact", "loop": "persistent"},
            "per_cloud": [{"cloud": name, "hull": int(h.numel()), "status": s}
                          for (name, _), h, s in zip(data, hulls, st)],
            "roofline": {"bound": "hbm", "kernel": "qh2d_multi<PredF32> (this rank's shards)",
                         "achieved": round(algo / (lms / 1e3) / 1e9, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(algo / (lms / 1e3) / 1e9 / peak, 4),
                         "peak_kind": peak_kind, "traffic": None,
                         "algo_bytes_per_launch": algo, "ms": round(lms, 4)},
            "clocks": clocks, "gpu_launches": 5 * args.steps,
            "e2e": {"value": round(pts / et / 1e6, 2), "unit": UNIT,
                    "h2d_bytes_per_step": sum(h.numel() * 4 for h in host),
                    "d2h_bytes_per_step": d2h,
                    "how": "each rank: pinned host -> device copy of its shards, the sharded "
                           "step, result records and hull indices read back"}}
    barrier()
    if multi:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
