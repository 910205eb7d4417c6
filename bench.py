#!/usr/bin/env python3
"""Throughput of the X-SLAM complex-step X-KinectFusion step (X-SLAM Sec. 3-4.1) on one GB300.

A step is one frame of the whole hot path (range gate, bilateral filter, pyramid, 19 ICP iterations
with the FP64 6x6 solve, TSDF update, ray cast, derivative read-out) on 1 real + K FP32 imaginary
lanes, over a seeded synthetic 640x480 depth sequence through a 256^3 x 1 cm room (K = 6: the left
twist of the first pose). Prints one JSON line (rank 0):

  value        frames/s with the depth frames resident in HBM (CUDA events on the caller's stream,
               which the library's stream is ordered against), summed over ranks;
  e2e          frames/s through the public calls with pinned host depth in and the pose + derivative
               block out every frame (host<->device copies inside the timed region): frame k + 1 is
               submitted (xslam_frame_submit) before frame k's outputs are read (xslam_frame_wait), the
               way a camera loop runs; `synchronous` is the same through xslam_frame, one frame at a
               time;
  roofline     the dominant kernel (largest device time per frame in a profiled pass over the same
               frames): algorithmic bytes per launch / its mean launch time, against the measured HBM
               copy bandwidth;
  cpu_baseline the CPU oracle (complex128, one process per lane) timed on the machine's host cores on
               frame 1 of the same sequence, which also gives the derivative error of the GPU lanes;
  plain_fp64   the plain FP64 complex path (include/xslam_plain.h: complex<double>, one run per seed,
               no lane batching) on the same frames, and the FP32 lanes' derivative error against it;
  uncomplexified_fp32  the same frames with no imaginary lanes (K = 0);
  batched      32 independent trajectories of 50-400 frames (mixed image sizes, grids and lane
               counts) advanced together through include/xslam_batch.h: aggregate frames/s and the
               per-trajectory frame latency;
  second_order relocalisation on a 512^3 map: gradient descent, nonlinear CG and Newton's method with
               the Hessian from xslam_grad order 2, the time of one Hessian evaluation, and the plain FP64
               bicomplex path beside it;
  learned_proposal  the learned pose proposal: training time and the tracking comparison.

The line carries these as compact summaries; --details PATH writes every figure to a JSON file.

--impl reference times the oracle alone on sampled steps of the same workload (see _reference).
Multi-GPU (torchrun): every rank runs its own independent sequence (replicas, no collective in the
data path; weak scaling); the timed region is bracketed by barriers and the max over ranks is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CSFD frames/s (640x480, 256³, K=6) FP32-batched vs plain FP64 at 1e-3 grad err"
H_GPU = 1e-10


# ------------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------------
def make_workload(name, seed, frames, device):
    from paper_2405_02187_gb300 import synth
    if name == "room256":
        return synth.room_walk(seed=seed, frames=frames, device=device)
    if name == "orbit64":
        return synth.small_orbit(seed=seed, frames=frames, device=device)
    raise SystemExit(f"unknown workload {name}")


def wl_desc(wl, K):
    return dict(workload=f"{wl.name}_K{K}", volume=f"{wl.dims[0]}^3 x {wl.voxel * 100:g} cm",
                image=f"{wl.intr.width}x{wl.intr.height}", lanes=K, seeds=f"POSE0 twist components 0..{K - 1}",
                icp_iters="/".join(str(i) for i in wl.icp_iters), bilateral=bool(wl.bilateral))


def xslam_cfg(wl):
    from paper_2405_02187_gb300 import xslam
    c = xslam.default_config()
    c.icp_levels = len(wl.icp_iters)
    for i, n in enumerate(wl.icp_iters):
        c.icp_iters[i] = n
    c.depth_min_m, c.depth_max_m, c.bilateral = wl.depth_min, wl.depth_max, int(wl.bilateral)
    return c


# ------------------------------------------------------------------------------------------------
# CPU oracle legs (run in spawned processes: no CUDA state is inherited)
# ------------------------------------------------------------------------------------------------
def oracle_pool(procs):
    """A pool of `procs` fresh interpreters (spawned, so no CUDA context is ever forked), each running the
    oracle on one thread: the math libraries' thread pools are set to one thread before they start."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(procs)


def _oracle_frames(task):
    """One complex lane of the oracle: frame 0 untimed, frame 1 timed. Returns (seconds, dtwist)."""
    from oracle import pipeline as P
    from oracle import se3
    wl, seed = task
    cfg = P.Config(icp_iters=tuple(wl["icp_iters"]), depth_min=wl["depth_min"], depth_max=wl["depth_max"],
                   bilateral=wl["bilateral"])
    run = P.XKinectFusion(wl["dims"], wl["voxel"], wl["trunc"], wl["origin"], wl["intr"], wl["pose0"], cfg,
                          P.Seed(seed[0], seed[1]))
    run.frame(wl["depth"][0])
    t = time.perf_counter()
    T, ok = run.frame(wl["depth"][1])
    dt = time.perf_counter() - t
    return dt, se3.readout(T, run.seed.h)[2], bool(ok)


def _oracle_shard_steps(task):
    """One complex lane of the oracle over sampled steps of frame 1. After an untimed frame 0, the
    frame's measurement (range gate, bilateral filter, pyramid, vertex and normal maps of every level)
    is computed once and timed; each step then processes shard s = i mod R of the frame's three O(N)
    stages: the 19 ICP iterations on 1/R of each level's pixels, the fusion of 1/R of the voxels and the
    ray cast of 1/R of the pixels. A step's time is its own time plus 1/R of the measurement time."""
    from oracle import fusion, icp, measure, raycast, se3
    from oracle import pipeline as P
    wl, seed, R, warm, steps = task
    cfg = P.Config(icp_iters=tuple(wl["icp_iters"]), depth_min=wl["depth_min"], depth_max=wl["depth_max"],
                   bilateral=wl["bilateral"])
    run = P.XKinectFusion(wl["dims"], wl["voxel"], wl["trunc"], wl["origin"], wl["intr"], wl["pose0"], cfg,
                          P.Seed(seed[0], seed[1]))
    run.frame(wl["depth"][0])
    intr = wl["intr"]
    n = int(np.prod(wl["dims"]))
    t = time.perf_counter()
    pyr = run.measure(wl["depth"][1])
    vns = []
    for level in range(len(cfg.icp_iters)):
        li = measure.level_intrinsics(intr, level)
        V = measure.vertex_map(pyr[level], li)
        Nm, valid = measure.normal_map(pyr[level], V)
        vns.append((V.reshape(-1, 3), Nm.reshape(-1, 3), valid.reshape(-1)))
    t_measure = time.perf_counter() - t
    out = []
    for i in range(warm + steps):
        s = i % R
        t = time.perf_counter()
        T = run.T
        for level in range(len(cfg.icp_iters) - 1, -1, -1):
            li = measure.level_intrinsics(intr, level)
            pix = np.arange(s, li[4] * li[5], R)
            for _ in range(cfg.icp_iters[level]):
                r, J, v = icp.correspondences(pyr[level], li, level, T, run.T, run.model, pix=pix, vn=vns[level])
                A, b, nv = icp.normal_equations(r, J, v)
                x = icp.solve(A, b) if nv >= 6 else None
                if x is not None:
                    T = se3.compose(se3.se3_exp(x), T)
        fusion.integrate(run.F, run.W, pyr[0], T, intr, run.dims, run.origin, run.voxel, run.mu,
                         idx=np.arange(s, n, R))
        raycast.raycast(run.F, run.W, T, intr, run.dims, run.origin, run.voxel, cfg.depth_min, cfg.depth_max,
                        pix=np.arange(s, intr.width * intr.height, R))
        if i >= warm:
            out.append(time.perf_counter() - t + t_measure / R)
    return out


def _wl_payload(wl, frames=2):
    return dict(dims=wl.dims, voxel=wl.voxel, trunc=wl.trunc, origin=wl.origin, intr=wl.intr,
                pose0=wl.poses[0], depth=wl.depth[:frames], icp_iters=wl.icp_iters, depth_min=wl.depth_min,
                depth_max=wl.depth_max, bilateral=wl.bilateral)


def cpu_model():
    """The host CPU's model name (lscpu, else the platform's processor string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------------------------------------------
# roofline bookkeeping
# ------------------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_bf16_tflops():
    """(dense bf16 TFLOP/s burst peak, "measured" | "fallback")."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


KERNEL_SRC = {"integrate": "fuse.cu", "raycast": "raycast.cu", "icp": "icp.cu"}
KERNEL_NAME = {"integrate": "k_integrate", "raycast": "k_march + k_refine", "icp": "k_icp"}


def _src_hash(stage):
    p = os.path.join(ROOT, "paper_2405_02187_gb300", "csrc", KERNEL_SRC[stage])
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def ncu_traffic(stage, workload):
    """DRAM bytes per launch of the stage's kernel from the committed ncu summary, if that summary was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{stage}")
    if not e or e.get("src_sha256_16") != _src_hash(stage):
        return None
    return e.get("dram_bytes_per_launch")


def icp_bytes_per_frame(wl, K):
    """ICP's algorithmic bytes per frame at the scope table's per-unit figure: every iteration reads,
    per pixel of its level, the pixel's own vertex and normal (24 B) and the model vertex and normal on
    1 + K lanes at its correspondence (24 (1 + K) B): 192 B per pixel-iteration at K = 6."""
    hw = wl.intr.width * wl.intr.height
    return sum(iters * (hw >> (2 * level)) * (24 + 24 * (1 + K)) for level, iters in enumerate(wl.icp_iters))


def algorithmic_bytes(stage, wl, K, per_frame, launches_per_frame=1.0):
    """Bytes a launch of the stage must move (see the kernels' headers):
    integrate: read + write of F (1 + K lanes) and W for every updated voxel, plus the depth map;
    raycast:   the model outputs (depth + vertex and normal on 1 + K lanes) plus the distinct voxels
               the march and the refinement read (per_frame["march_voxels"] of Re F, and
               per_frame["refine_voxels"] of Re F and the K imaginary planes);
    icp:       icp_bytes_per_frame / the ICP launches of a frame (one cooperative launch)."""
    L = 1 + K
    hw = wl.intr.width * wl.intr.height
    if stage == "integrate":
        return per_frame["fused"] * 2 * 4 * (L + 1) + 4 * hw
    if stage == "raycast":
        return hw * 4 * (1 + 6 * L) + per_frame["march_voxels"] * 4 + per_frame["refine_voxels"] * 4 * L
    if stage == "icp":
        return icp_bytes_per_frame(wl, K) / launches_per_frame
    raise ValueError(stage)


def raycast_voxel_reads(intr, T, hit_depth, dims, voxel, origin, step, m0, m1, chunk=2048):
    """Distinct voxels the ray cast reads at pose T (3x4) given its per-pixel hit depth (camera z,
    0 = no surface; a torch tensor H x W on any device), following the ray cast's sampling (samples at
    alpha_m = m * step, m0 <= m <= m1, within the volume's slab, each reading the 8 corners of its
    trilinear cell): the march reads every sample from the first in the volume to the second sample of
    the hit pair (to the last in the volume without a hit); the refinement reads the cells of the hit
    pair's two samples and of the six normal samples at the vertex +- one voxel per axis. Returns
    (march voxels, refine voxels), each a count of distinct voxels."""
    import torch
    dev = hit_depth.device
    nx, ny, nz = dims
    n = nx * ny * nz
    H, W = hit_depth.shape
    R = torch.tensor(np.asarray(T)[:, :3], dtype=torch.float64, device=dev)
    t = torch.tensor(np.asarray(T)[:, 3], dtype=torch.float64, device=dev)
    org = torch.tensor(origin, dtype=torch.float64, device=dev)
    nn = torch.tensor([nx, ny, nz], dtype=torch.float64, device=dev)
    v, u = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float64),
                          torch.arange(W, device=dev, dtype=torch.float64), indexing="ij")
    rc = torch.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, torch.ones_like(u)], -1).reshape(-1, 3)
    d = rc @ R.T                                  # world direction per unit camera depth
    g0 = (t - org) / voxel - 0.5                  # grid coordinate at alpha = 0
    gd = d / voxel
    # slab: 0 <= g < n - 1 on every axis
    t1 = (0.0 - g0) / gd
    t2 = ((nn - 1.0) - g0) / gd
    lo = torch.where(gd != 0, torch.minimum(t1, t2), torch.full_like(gd, -np.inf)).amax(1)
    hi = torch.where(gd != 0, torch.maximum(t1, t2), torch.full_like(gd, np.inf)).amin(1)
    inside = torch.where(gd == 0, (g0 >= 0) & (g0 < nn - 1), torch.ones_like(gd, dtype=torch.bool)).all(1)
    hd = hit_depth.reshape(-1).to(torch.float64)
    m_lo = torch.clamp(torch.floor(torch.clamp(lo, min=m0 * step) / step) - 1, min=m0)
    m_hi = torch.clamp(torch.ceil(torch.clamp(hi, max=m1 * step) / step) + 1, max=m1)
    m_end = torch.where(hd > 0, torch.floor(hd / step) + 1, m_hi)
    march = torch.zeros(n, dtype=torch.bool, device=dev)
    refine = torch.zeros(n, dtype=torch.bool, device=dev)
    off = torch.tensor([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=torch.int64, device=dev)

    def mark(bitmap, g):
        ok = ((g >= 0) & (g < nn - 1)).all(-1)
        c = torch.floor(g[ok]).to(torch.int64)[:, None, :] + off[None]
        idx = c[..., 0] + nx * (c[..., 1] + ny * c[..., 2])
        bitmap[idx.reshape(-1)] = True

    npx = H * W
    for a in range(0, npx, chunk):
        sl = slice(a, min(a + chunk, npx))
        ok = inside[sl] & (m_end[sl] >= m_lo[sl])
        if not bool(ok.any()):
            continue
        lo_c, end_c = m_lo[sl][ok], m_end[sl][ok]
        M = int((end_c - lo_c).max().item()) + 1
        m = lo_c[:, None] + torch.arange(M, device=dev, dtype=torch.float64)[None]
        keep = m <= end_c[:, None]
        g = g0 + (m * step)[..., None] * gd[sl][ok][:, None, :]
        mark(march, g[keep])
        hit = hd[sl] > 0
        if bool(hit.any()):
            a0 = hd[sl][hit]
            mh = torch.floor(a0 / step)
            gh = gd[sl][hit]
            vtx = g0 + a0[:, None] * gh
            e = torch.eye(3, dtype=torch.float64, device=dev)
            pts = [g0 + (mh * step)[:, None] * gh, g0 + ((mh + 1) * step)[:, None] * gh]
            pts += [vtx + s * e[i] for i in range(3) for s in (1.0, -1.0)]
            mark(refine, torch.cat(pts, 0))
    return int(march.sum().item()), int(refine.sum().item())


def model_voxel_reads(x, wl, dev):
    """raycast_voxel_reads of a handle's current model: its pose and the hit depth of a ray cast there."""
    import torch
    dep = torch.empty((wl.intr.height, wl.intr.width), device=dev)
    x.raycast(None, dep, None, None)
    T = x.get_pose_lanes()[0]
    step = wl.voxel * 1.0  # ray_step_vox = 1
    m0 = int(math.ceil(wl.depth_min / step - 1e-4))
    m1 = int(math.floor(wl.depth_max / step + 1e-4))
    return raycast_voxel_reads(wl.intr, T, dep, wl.dims, wl.voxel, wl.origin, step, m0, m1)


# ------------------------------------------------------------------------------------------------
# replicas: one independent sequence per rank, the slowest rank's time
# ------------------------------------------------------------------------------------------------
def replica_seed(rank):
    """Seed of rank's sequence: every replica tracks its own trajectory (no data exchange)."""
    return 2 + rank


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the default process group (x itself when there is none)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, ms_max):
    """Whole-job units/s: every rank processed units_per_rank in at most ms_max milliseconds."""
    return units_per_rank * world / (ms_max / 1000.0)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2405_02187_gb300 import xslam

    # the CPU oracle processes are spawned (fresh interpreters) before any GPU call
    pool = None
    cpu_lanes = min(args.lanes, 6)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(cpu_lanes)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W, K, L = args.warmup, args.steps, args.lanes
    nf = W + K + 1
    wl = make_workload(args.workload, replica_seed(rank), nf, dev)
    if args.workload == "room256" and nf > 300:
        print("note: more frames than the 300-frame sequence were generated", file=sys.stderr)
    cfg = xslam_cfg(wl)
    seeds = [(xslam.POSE0, j % 6, H_GPU) for j in range(L)]
    depth_dev = torch.tensor(wl.depth, device=dev)
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()

    def handle():
        x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_lanes=L)
        x.set_pose(wl.poses[0])
        return x

    # ---- timed region: device-resident depth, graphs, no host sync per frame ----
    x = handle()
    for k in range(W):
        x.frame(depth_dev[k], seeds, outputs=False)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(W, W + K):
        x.frame(depth_dev[k], seeds, outputs=False)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    _, n_fail = x.sync()
    x.close()
    ms = max_over_ranks(ms, dev)
    value = replica_throughput(K, world, ms)

    # ---- profiled pass over the same frames: per-stage device time (no graphs) ----
    x = handle()
    for k in range(W):
        x.frame(depth_dev[k], seeds, outputs=False)
    x.profile(True)
    for k in range(W, W + K):
        x.frame(depth_dev[k], seeds, outputs=False)
    stages, counters = x.profile_read()
    x.profile(False)
    nprof = counters["frames"]
    per_frame = dict(fused=counters["fused"] / nprof, hits=counters["hits"] / nprof)
    # distinct voxels the ray cast reads, counted on the last frame's model (same pose, same volume)
    per_frame["march_voxels"], per_frame["refine_voxels"] = model_voxel_reads(x, wl, dev)
    x.close()
    launches_per_frame = sum(v[1] for v in stages.values()) / nprof
    cand = {s: stages[s][0] / nprof for s in ("integrate", "raycast", "icp")}
    dom = max(cand, key=cand.get)
    # per stage: launches of its roofline kernel (a ray cast is a k_march + k_refine pair; the fusion
    # stage's tile list, the integrate kernel and the restart clear count as one update)
    n_units = dict(icp=stages["icp"][1] / nprof, integrate=1.0, raycast=1.0)
    ms_launch = stages[dom][0] / nprof / n_units[dom]
    bytes_launch = algorithmic_bytes(dom, wl, L, per_frame, launches_per_frame=n_units["icp"])
    peak, peak_src = measured_peaks()
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9
    traffic = ncu_traffic(dom, wl.name)
    roofline = dict(bound="hbm", achieved=round(achieved, 1), peak=peak, unit="GB/s",
                    frac=round(achieved / peak, 4), traffic=traffic, kernel=KERNEL_NAME[dom],
                    peak_source=f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                    bytes_per_launch=round(bytes_launch), ms_per_launch=round(ms_launch, 5))
    stage_ms = {s: round(v[0] / nprof, 4) for s, v in stages.items()}
    # the same roofline for each of the three stages (the dominant one is `roofline` itself)
    roofline_stages = {}
    for st in ("icp", "integrate", "raycast"):
        if stages[st][1] <= 0 or stages[st][0] <= 0.0:
            continue
        ms_st = stages[st][0] / nprof / n_units[st]
        b_st = algorithmic_bytes(st, wl, L, per_frame, launches_per_frame=n_units["icp"])
        a_st = b_st / (ms_st * 1e-3) / 1e9
        roofline_stages[st] = dict(kernel=KERNEL_NAME[st], achieved=round(a_st, 1), frac=round(a_st / peak, 4),
                                   traffic=ncu_traffic(st, wl.name), bytes_per_launch=round(b_st),
                                   ms_per_launch=round(ms_st, 5))

    # ---- end to end: pinned host depth in, pose + derivative block out, every frame ----
    host = torch.empty((nf,) + tuple(wl.depth.shape[1:]), dtype=torch.float32, pin_memory=True)
    host.copy_(torch.from_numpy(wl.depth))
    ms_e2e, dtw_all, dtw_frame1 = {}, {}, None
    for mode in ("synchronous", "pipelined"):
        x = handle()
        for k in range(W):
            pose, dpose, dtw, st = x.frame(host[k], seeds)
            if k == 1:
                dtw_frame1 = dtw.copy()
        torch.cuda.synchronize()
        barrier()
        e0.record()
        out = {}
        if mode == "synchronous":
            for k in range(W, W + K):
                out[k] = x.frame(host[k], seeds)[2]
        else:  # submit frame k, then read frame k - 1: every frame's depth in and outputs out, overlapped
            prev = None
            for k in range(W, W + K):
                t = x.submit(host[k], seeds)
                if prev is not None:
                    out[prev[0]] = x.wait(prev[1])[2]
                prev = (k, t)
            out[prev[0]] = x.wait(prev[1])[2]
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms_e2e[mode] = max_over_ranks(e0.elapsed_time(e1), dev)
        x.close()
        if mode == "synchronous":
            dtw_all = out
        else:
            assert all(np.array_equal(out[k], dtw_all[k]) for k in out), "pipelined frames differ"
    e2e = dict(value=round(replica_throughput(K, world, ms_e2e["pipelined"]), 2), unit="frames/s",
               h2d_bytes_per_step=int(4 * wl.intr.width * wl.intr.height), d2h_bytes_per_step=int(8 * (12 + 18 * L)),
               synchronous=round(replica_throughput(K, world, ms_e2e["synchronous"]), 2))

    # ---- beside the headline: the uncomplexified FP32 run (K = 0) and the plain FP64 complex path ----
    x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_lanes=0)
    x.set_pose(wl.poses[0])
    for k in range(W):
        x.frame(depth_dev[k], [], outputs=False)
    torch.cuda.synchronize()
    e0.record()
    for k in range(W, W + K):
        x.frame(depth_dev[k], [], outputs=False)
    e1.record()
    torch.cuda.synchronize()
    ms_real = e0.elapsed_time(e1)
    x.close()
    real32 = dict(value=round(K * world / (ms_real / 1000.0), 2), unit="frames/s", ms_per_step=round(ms_real / K, 4),
                  lanes=0)
    plain = None
    if not args.no_plain:
        # the plain path runs the same frames from frame 0 (its pose chain is its own), fewer of them
        Kp = min(K, args.plain_steps)
        xp = xslam.XSlamPlain(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_runs=L)
        xp.set_pose(wl.poses[0])
        seeds_p = [(xslam.POSE0, j % 6, 1e-20) for j in range(L)]
        for k in range(W):
            xp.frame(depth_dev[k], seeds_p)
        torch.cuda.synchronize()
        e0.record()
        for k in range(W, W + Kp):
            _, _, dtw_p, _ = xp.frame(depth_dev[k], seeds_p)
        e1.record()
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1)
        xp.close()
        last = W + Kp - 1
        err = float(np.linalg.norm(dtw_all[last] - dtw_p) / np.linalg.norm(dtw_p))
        plain = dict(value=round(Kp * world / (ms_plain / 1000.0), 3), unit="frames/s", ms_per_step=round(ms_plain / Kp, 3),
                     steps=Kp, dtype="c128", runs=L,
                     method="complex<double> AoS voxels, one complex run per seed, one thread per pixel/voxel, "
                            "no lane batching, no graphs",
                     speedup_of_value=round(value / (Kp * world / (ms_plain / 1000.0)), 2),
                     grad_rel_err_fp32_lanes_vs_plain=err, grad_err_frame=last)

    batched = None if args.no_batch else run_section("batched", run_batch, args, dev, rank)
    second = None if args.no_second_order else run_section("second_order", run_second_order, args, dev, rank)
    learned = None if args.no_learned else run_section("learned_proposal", run_learned, args, dev, rank)

    # ---- CPU oracle on the host cores (rank 0, N = 1): frame 1 of the same sequence ----
    cpu = None
    grad_err = None
    if pool is not None:
        payload = _wl_payload(wl, 2)
        lanes = [(0, j % 6) for j in range(cpu_lanes)]
        t0 = time.perf_counter()
        res = pool.map(_oracle_frames, [(payload, s) for s in lanes])
        wall = time.perf_counter() - t0
        pool.close()
        lane_s = max(r[0] for r in res)
        cpu = dict(value=round(1.0 / lane_s * cpu_lanes / L, 5), unit="frames/s", cores=cpu_lanes, kind="oracle",
                   cpu_model=cpu_model(), host_cores=os.cpu_count(),
                   sample=f"frame 1 (ICP 19 iterations, fusion, ray cast) of the same {wl.name} sequence after an "
                          f"untimed frame 0; {cpu_lanes} complex128 lanes, one process per lane, slowest lane "
                          f"{lane_s:.1f} s (wall incl. frame 0: {wall:.0f} s)")
        if dtw_frame1 is not None and W > 1:
            ref = np.stack([r[1] for r in res])
            gpu = dtw_frame1[:cpu_lanes]
            grad_err = float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref))

    # the metric's companions as top-level scalars first; the experiments beside the headline as short
    # summaries (every figure goes to --details)
    companions = dict(
        grad_rel_err_vs_oracle=grad_err,
        plain_fp64_frames_per_s=plain["value"] if plain else None,
        speedup_vs_plain_fp64=plain["speedup_of_value"] if plain else None,
        grad_rel_err_vs_plain_fp64=float(f"{plain['grad_rel_err_fp32_lanes_vs_plain']:.3g}") if plain else None,
        uncomplexified_fp32_frames_per_s=real32["value"],
        lanes_cost_vs_uncomplexified=round(real32["value"] / value, 3))
    line = dict(metric=METRIC, value=round(value, 2), unit="frames/s", n_gpus=world, steps=K, warmup=W,
                ms_per_step=round(ms / K, 4), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic", **companions,
                config=dict(wl_desc(wl, L), parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                            l2="inputs larger than L2: the TSDF state (F lanes and W) alone is "
                               f"{np.prod(wl.dims) * 4 * (L + 2) / 1e6:.0f} MB",
                            tracking_failures=int(n_fail)),
                roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(round(launches_per_frame * K)),
                clocks=clk, stage_ms_per_frame=stage_ms, roofline_stages=roofline_stages,
                per_frame=dict(fused_voxels=round(per_frame["fused"]), surface_pixels=round(per_frame["hits"]),
                               raycast_march_voxels=per_frame["march_voxels"],
                               raycast_refine_voxels=per_frame["refine_voxels"]),
                batched=_batched_summary(batched), second_order=_second_summary(second),
                learned_proposal=_learned_summary(learned))
    details = dict(line, plain_fp64=plain, uncomplexified_fp32=real32, batched=batched, second_order=second,
                   learned_proposal=learned)
    if rank == 0:
        if args.details:
            with open(args.details, "w") as f:
                json.dump(details, f, indent=1)
        print(json.dumps(line))


def run_section(name, fn, *a):
    """One of the line's companion sections (no collectives inside): an exception in it is reported in
    the line as {"error": ...} with its traceback on stderr, and the headline is still printed."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - any failure of a companion section
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{name}: {type(e).__name__}: {e}"[:300]}


def _batched_summary(b):
    if not b or "error" in b:
        return b or None
    return dict(value=b["value"], unit=b["unit"], frames=b["frames"], speedup_vs_sequential=b["speedup_vs_sequential"],
                latency_ms_median=b["latency_ms_per_frame"]["median"], roofline_frac=b["roofline"]["frac"],
                tracking_failures=b["tracking_failures"])


def _second_summary(s2):
    if not s2 or "error" in s2:
        return s2 or None
    h = s2["hessian"]
    t = s2["tsdf_loss"]
    return dict(newton_recall=s2["newton_eta"].get("recall_1cm_1deg"), newton_median_cm=s2["newton_eta"]["median_cm"],
                nlcg_median_cm=s2["nlcg"]["median_cm"], gd_median_cm=s2["gradient_descent"]["median_cm"],
                hessian_ms=h["ms_per_evaluation"], hessian_plain_fp64_ms=h["plain_fp64"]["ms_per_evaluation"],
                hessian_speedup_vs_plain_fp64=h["plain_fp64"]["speedup_of_fp32"],
                hessian_rel_err_vs_plain_fp64=h["plain_fp64"]["hess_rel_err_fp32"],
                tsdf_hessian_ms=t["hessian"]["ms_per_evaluation"],
                tsdf_hessian_plain_fp64_ms=t["plain_fp64"]["ms_per_evaluation"],
                tsdf_hessian_rel_err_vs_plain_fp64=t["plain_fp64"]["hess_rel_err_fp32"])


def _learned_summary(lp):
    if not lp or "error" in lp:
        return lp or None
    out = dict(train_ms=lp["train"]["train_ms"], pairs=lp["train"]["pairs"])
    for wname, w in lp.get("walks", {}).items():
        o = dict(start_error_sigma=w["start_error_sigma"])
        for k in ("constant_velocity", "constant_velocity_proposal", "previous_pose", "previous_pose_proposal"):
            if k in w:
                r = w[k]
                o[k] = dict(fps=r["fps"], failures=r["failures"], trans_err_cm_mean=r["trans_err_cm_mean"],
                            fallback_rate=r.get("fallback_rate"))
        out[wname] = o
    return out


# ------------------------------------------------------------------------------------------------
# batched trajectories (include/xslam_batch.h)
# ------------------------------------------------------------------------------------------------
def run_batch(args, dev, rank):
    """Many trajectories of uneven length, image size, grid and lane count, advanced together: one
    CUDA graph per step. The launch shapes are picked by the library's autotuner on the first steps; the
    timed pass then runs every trajectory from frame 0 to its end. Returns the JSON object."""
    import torch
    from paper_2405_02187_gb300 import synth, xslam

    t0 = time.perf_counter()
    trajs = synth.batch_trajectories(seed=7 + rank, n=args.batch_n, min_frames=args.batch_min, max_frames=args.batch_max,
                                     device=dev, resident=True)
    gen_s = time.perf_counter() - t0
    lens = [wl.depth.shape[0] for wl, _ in trajs]
    handles = []
    for wl, lanes in trajs:
        x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl), max_lanes=len(lanes))
        x.set_lanes([(k, j, H_GPU) for k, j in lanes])
        x.set_pose(wl.poses[0])
        handles.append(x)
    depth = [wl.depth for wl, _ in trajs]
    batch = xslam.XSlamBatch(handles)
    tune_steps = 6
    frames = [[d[k] if k < n else None for d, n in zip(depth, lens)] for k in range(tune_steps)]
    choice, tune_ms = batch.autotune(frames, tune_steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(lens)
    e0.record()
    for k in range(steps):
        batch.step([d[k] if k < n else None for d, n in zip(depth, lens)])
    e1.record()
    fails = batch.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    total = sum(lens)
    # algorithmic bytes of the whole run (the per-kernel unit counts of the single-trajectory roofline)
    moved = 0.0
    for (wl, lanes), x, n in zip(trajs, handles, lens):
        _, cnt = x.profile_read()
        L = 1 + len(lanes)
        hw = wl.intr.width * wl.intr.height
        per = dict(fused=cnt["fused"] / n, hits=cnt["hits"] / n)
        per["march_voxels"], per["refine_voxels"] = model_voxel_reads(x, wl, dev)
        moved += n * (algorithmic_bytes("integrate", wl, len(lanes), per) + algorithmic_bytes("raycast", wl, len(lanes), per))
        moved += (n - 1) * icp_bytes_per_frame(wl, len(lanes))
    # per-trajectory frame latency inside a step, from a second batch over the first steps
    batch.close()
    for (wl, lanes), x in zip(trajs, handles):
        x.reset()
        x.set_lanes([(k, j, H_GPU) for k, j in lanes])
        x.set_pose(wl.poses[0])
    batch = xslam.XSlamBatch(handles)
    batch.set_shapes(choice)
    lat = []
    for k in range(min(12, min(lens))):
        batch.step([d[k] for d in depth])
        if k >= 2:
            lat.append(batch.latency())
    # where a segmented step's time goes: one profiled step (events between the launches)
    batch.set_shapes(dict(choice, mode="segmented"))
    batch.profile(True)
    kp = min(12, min(lens))
    batch.step([d[kp] for d in depth])
    stage_ms = {}
    for stage, _, _, t in batch.profile_read():
        stage_ms[stage] = stage_ms.get(stage, 0.0) + t
    batch.close()
    lat = np.mean(np.array(lat), 0) if lat else np.zeros(len(lens))
    # the same trajectories one at a time (their own graphs, default grids): frames 2..7 of each
    seq = []
    for (wl, lanes), x, d in zip(trajs, handles, depth):
        x.reset()
        x.set_pose(wl.poses[0])
        sd = [(k, j, H_GPU) for k, j in lanes]
        for k in range(2):
            x.frame(d[k], sd, outputs=False)
        e0.record()
        for k in range(2, 8):
            x.frame(d[k], sd, outputs=False)
        e1.record()
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1) / 6)
    seq_ms = float(sum(t * n for t, n in zip(seq, lens)))
    peak, peak_src = measured_peaks()
    vox = [int(np.prod(wl.dims)) for wl, _ in trajs]
    return dict(
        workload=f"{len(trajs)} room walks of {min(lens)}-{max(lens)} frames, 320x240 or 640x480, grids "
                 f"{min(wl.dims[0] for wl, _ in trajs)}^3-{max(wl.dims[0] for wl, _ in trajs)}^3 over a 2.56 m room, "
                 f"K {min(len(l) for _, l in trajs)}-{max(len(l) for _, l in trajs)}",
        frames=total, steps=steps, value=round(total / (ms / 1000.0), 1), unit="frames/s (all trajectories)",
        ms=round(ms, 1), ms_per_step=round(ms / steps, 3), tracking_failures=int(sum(fails)),
        sequential=dict(ms=round(seq_ms, 1), value=round(total / (seq_ms / 1000.0), 1),
                        note="each trajectory alone through xslam_frame (graphs), frames 2-7 timed, times its length"),
        speedup_vs_sequential=round(seq_ms / ms, 2),
        roofline=dict(bound="hbm", achieved=round(moved / (ms * 1e-3) / 1e9, 1), peak=peak, unit="GB/s",
                      frac=round(moved / (ms * 1e-3) / 1e9 / peak, 4), algorithmic_gb=round(moved / 1e9, 2),
                      note="algorithmic bytes of every ICP, fusion and ray-cast launch of the run / its time"),
        autotune=dict(choice=choice, ms_per_step=[round(float(m), 3) for m in tune_ms],
                      candidates="mode segmented, branches; ICP grid / 1, 2, 4, 8, 16, 32; then in segmented mode fusion "
                                 "blocks per SM default, 1, 2, 4 and ray tile 32x8, 16x16, 64x4 (one coordinate at a "
                                 "time, each with the best of the ones before)"),
        segmented_step_ms_by_stage={k: round(v, 3) for k, v in stage_ms.items()},
        latency_ms_per_frame=dict(min=round(float(lat.min()), 3), median=round(float(np.median(lat)), 3),
                                  max=round(float(lat.max()), 3)),
        state_gb=round(sum(v * 4 * (2 + len(l)) for v, (_, l) in zip(vox, trajs)) / 1e9, 2),
        input_gb=round(sum(wl.depth.numel() * 4 for wl, _ in trajs) / 1e9, 2), generate_s=round(gen_s, 1))


# ------------------------------------------------------------------------------------------------
# second order: relocalisation with the Hessian (xslam_grad order 2)
# ------------------------------------------------------------------------------------------------
def run_second_order(args, dev, rank):
    """A 512^3 x 0.8 cm map of a 40-primitive scene built from a 500-frame walk; 100 query frames of
    that walk start from their true pose perturbed by up to 5 cm / 3 degrees and are relocalised by
    gradient descent, nonlinear conjugate gradients and Newton's method with the eta switch (loss,
    gradient and Hessian from the GPU), with per-iteration curves of the three optimisers (Sec. 6's ICP
    comparison). Also the time of one order-2 evaluation (21 second-order directions) and of one
    order-1."""
    import torch
    from paper_2405_02187_gb300 import reloc, synth, xslam

    t0 = time.perf_counter()
    frames = args.reloc_frames
    wl = synth.room_walk(seed=11 + rank, frames=frames, dims=512, voxel=0.008, n_prims=40, device=dev, resident=True)
    gen_s = time.perf_counter() - t0
    x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl), max_lanes=6)
    x.set_pose(wl.poses[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for k in range(frames):
        x.frame(wl.depth[k], [], outputs=False)
    e1.record()
    _, n_fail = x.sync()
    map_ms = e0.elapsed_time(e1)
    rng = np.random.Generator(np.random.PCG64(5 + rank))
    queries = []
    for _ in range(args.reloc_queries):
        k = int(rng.integers(frames // 5, frames))
        dxi = np.concatenate([rng.uniform(-1, 1, 3) * math.radians(3.0) / math.sqrt(3.0),
                              rng.uniform(-1, 1, 3) * 0.05 / math.sqrt(3.0)])
        queries.append((k, reloc.compose(reloc.se3_exp(dxi), wl.poses[k])))
    out = {}
    for method in ("gd", "nlcg", "newton"):
        errs, its, evals = [], [], 0
        t1 = time.perf_counter()
        for k, T0 in queries:
            r = reloc.relocalise(x, wl.depth[k], T0, method=method, eta=args.reloc_eta, iters=args.reloc_iters)
            errs.append(reloc.pose_error(r.T, wl.poses[k]))
            its.append(r.iterations)
            evals += r.evaluations
        wall = time.perf_counter() - t1
        e = np.array(errs)
        out[method] = dict(median_cm=round(float(np.median(e[:, 0])) * 100, 3), median_deg=round(float(np.median(e[:, 1])), 4),
                           recall_1cm_1deg=round(float(np.mean((e[:, 0] < 0.01) & (e[:, 1] < 1.0))), 3),
                           mean_iterations=round(float(np.mean(its)), 2), evaluations=evals, wall_s=round(wall, 2))
    # the paper's TSDF-difference loss (the query's surface update against the map) on the first
    # queries, Newton whenever the Hessian is positive definite (eta = inf: the loss is a sum over
    # voxels, not on the point-to-plane scale)
    out_tsdf = {}
    nq = min(len(queries), args.reloc_tsdf_queries)
    for method in ("gd", "nlcg", "newton"):
        errs, its, evals = [], [], 0
        t1 = time.perf_counter()
        for k, T0 in queries[:nq]:
            r = reloc.relocalise(x, wl.depth[k], T0, method=method, eta=float("inf"), iters=args.reloc_iters,
                                 loss="tsdf")
            errs.append(reloc.pose_error(r.T, wl.poses[k]))
            its.append(r.iterations)
            evals += r.evaluations
        wall = time.perf_counter() - t1
        e = np.array(errs)
        out_tsdf[method] = dict(median_cm=round(float(np.median(e[:, 0])) * 100, 3),
                                median_deg=round(float(np.median(e[:, 1])), 4),
                                recall_1cm_1deg=round(float(np.mean((e[:, 0] < 0.01) & (e[:, 1] < 1.0))), 3),
                                mean_iterations=round(float(np.mean(its)), 2), evaluations=evals, wall_s=round(wall, 2))
    init = np.array([reloc.pose_error(T0, wl.poses[k]) for k, T0 in queries])
    # Sec. 6's ICP optimiser comparison (translation error, rotation error and point-to-plane loss per
    # iteration for gradient descent, nonlinear CG and Newton): medians over the first 10 queries
    fig3 = {}
    n_it = 30
    for method in ("gd", "nlcg", "newton"):
        curves = []
        for k, T0 in queries[:10]:
            tr = [(T0, float(x.grad(wl.depth[k], T0, order=1)[0]))]
            reloc.relocalise(x, wl.depth[k], T0, method=method, eta=float("inf"), iters=n_it, tol=0.0, trace=tr)
            while len(tr) < n_it + 1:
                tr.append(tr[-1])
            curves.append([(*reloc.pose_error(T, wl.poses[k]), E) for T, E in tr[:n_it + 1]])
        c = np.median(np.array(curves), axis=0)
        fig3[method] = dict(trans_cm=[round(float(v) * 100, 4) for v in c[:, 0]],
                            rot_deg=[round(float(v), 4) for v in c[:, 1]],
                            loss=[float(f"{v:.4g}") for v in c[:, 2]])
    # throughput of the derivative evaluations at one query
    k, T0 = queries[0]
    for order in (1, 2):
        for _ in range(3):
            x.grad(wl.depth[k], T0, order=order)
    times = {}
    for order in (1, 2):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        n = 20
        for _ in range(n):
            x.grad(wl.depth[k], T0, order=order)
        times[order] = (time.perf_counter() - t1) / n * 1e3
    # the TSDF-difference loss at the same query
    for _ in range(3):
        x.grad_tsdf(wl.depth[k], T0, order=2)
    tsdf_times = {}
    for order in (1, 2):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        n = 20
        for _ in range(n):
            _, _, _, n_vox = x.grad_tsdf(wl.depth[k], T0, order=order)
        tsdf_times[order] = (time.perf_counter() - t1) / n * 1e3
    # the plain FP64 bicomplex path on the same query: time and the FP32 path's derivative error
    x.grad_tsdf_plain64(wl.depth[k], T0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n = 10
    for _ in range(n):
        E64, g64, H64, _ = x.grad_tsdf_plain64(wl.depth[k], T0)
    ms64 = (time.perf_counter() - t1) / n * 1e3
    E32, g32, H32, _ = x.grad_tsdf(wl.depth[k], T0, order=2)
    err_g = float(np.linalg.norm(g32 - g64) / max(np.linalg.norm(g64), 1e-300))
    err_H = float(np.linalg.norm(H32 - H64) / max(np.linalg.norm(H64), 1e-300))
    # the point-to-plane loss of xslam_grad by the plain FP64 bicomplex path (xslam_grad_plain64)
    x.grad_plain64(wl.depth[k], T0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n = 5
    for _ in range(n):
        Ep, gp, Hp = x.grad_plain64(wl.depth[k], T0)
    ms_p64 = (time.perf_counter() - t1) / n * 1e3
    Ef, gf, Hf = x.grad(wl.depth[k], T0, order=2)
    p2p64 = dict(note="Sec. 3's bicomplex step in FP64 with full products (h = 1e-20), its own FP64 march and "
                      "decisions, one thread per pixel; the FP32 truncated path's relative error against it",
                 ms_per_evaluation=round(ms_p64, 3), per_s=round(1000.0 / ms_p64, 2),
                 speedup_of_fp32=round(ms_p64 / times[2], 1),
                 grad_rel_err_fp32=float(f"{np.linalg.norm(gf - gp) / max(np.linalg.norm(gp), 1e-300):.3g}"),
                 hess_rel_err_fp32=float(f"{np.linalg.norm(Hf - Hp) / max(np.linalg.norm(Hp), 1e-300):.3g}"),
                 loss_rel_diff=float(f"{abs(Ef - Ep) / max(abs(Ep), 1e-300):.3g}"))
    x.close()
    return dict(
        workload=f"{wl.dims[0]}^3 x {wl.voxel * 100:.1f} cm map of a 40-primitive room from a {frames}-frame 640x480 walk; "
                 f"{len(queries)} queries at their true pose perturbed by up to 5 cm / 3 deg",
        map_ms_per_frame=round(map_ms / frames, 3), map_tracking_failures=int(n_fail),
        optimiser_curves=dict(note="median over 10 queries of the translation error, rotation error and loss after "
                                   "each iteration (index 0 = start); Newton without the eta switch", **fig3),
        initial=dict(median_cm=round(float(np.median(init[:, 0])) * 100, 3), median_deg=round(float(np.median(init[:, 1])), 4)),
        gradient_descent=out["gd"], nlcg=out["nlcg"], newton_eta=dict(out["newton"], eta=args.reloc_eta),
        hessian=dict(ms_per_evaluation=round(times[2], 3), per_s=round(1000.0 / times[2], 1),
                     directions=21, note="loss + gradient + 21 second-order directions over 640x480, host round trip included",
                     plain_fp64=p2p64),
        gradient=dict(ms_per_evaluation=round(times[1], 3), per_s=round(1000.0 / times[1], 1)),
        tsdf_loss=dict(note=f"the paper's TSDF-difference loss on the first {nq} queries (Newton whenever H is "
                            "positive definite); evaluation times at one query, host round trip included",
                       updated_voxels=int(n_vox), gradient_descent=out_tsdf["gd"], nlcg=out_tsdf["nlcg"],
                       newton=out_tsdf["newton"],
                       hessian=dict(ms_per_evaluation=round(tsdf_times[2], 3), per_s=round(1000.0 / tsdf_times[2], 1),
                                    voxel_direction_pairs_per_s=round(21 * n_vox / (tsdf_times[2] * 1e-3), 1)),
                       gradient=dict(ms_per_evaluation=round(tsdf_times[1], 3), per_s=round(1000.0 / tsdf_times[1], 1)),
                       plain_fp64=dict(note="Sec. 3's bicomplex step in FP64 with full products (h = 1e-20), same "
                                            "voxels; the FP32 path's relative error against it",
                                       ms_per_evaluation=round(ms64, 3), per_s=round(1000.0 / ms64, 1),
                                       speedup_of_fp32=round(ms64 / tsdf_times[2], 2),
                                       grad_rel_err_fp32=float(f"{err_g:.3g}"), hess_rel_err_fp32=float(f"{err_H:.3g}"),
                                       loss_rel_diff=float(f"{abs(E32 - E64) / max(abs(E64), 1e-300):.3g}"))),
        generate_s=round(gen_s, 1))


# ------------------------------------------------------------------------------------------------
def run_learned(args, dev, rank):
    """Train the proposal network on frame pairs of room walks tracked by the method, then track a
    1000-frame 640x480, 512^3 trajectory with K = 6 CSFD lanes from the constant-velocity start and from
    the previous pose (the paper's start), each with and without the proposal as a second judged start:
    frames/s, ICP iterations per frame (stop tolerance 1e-5), pose error against the ground truth,
    failures, the proposal's acceptance and fallback rates, and how far each start lies from the true
    motion."""
    import torch
    from paper_2405_02187_gb300 import learn, synth

    ds = learn.make_dataset(n_traj=args.learned_rooms, frames=16, reverse=True, seed=20000 + 1000 * rank, device=dev)
    P = int(ds.pairs.shape[0])
    m, losses, ms = learn.train(ds, epochs=args.learned_epochs, lr=1e-3, mirror=True)
    flops = learn.train_flops(P, 256, args.learned_epochs)
    peak, peak_kind = measured_bf16_tflops()
    tfl = flops / (ms * 1e9)
    train = dict(pairs=P, frames=ds.n_frames, rooms=args.learned_rooms, epochs=args.learned_epochs, batch=256,
                 lr=1e-3, mirror=True, data_s=round(ds.seconds, 1), train_ms=round(ms, 1),
                 loss_first=round(float(losses[0]), 4), loss_last=round(float(losses[-1]), 4),
                 gemm_tflop=round(flops / 1e12, 3), tflops_whole_steps=round(tfl, 2),
                 tensor_frac_whole_steps=round(tfl / peak, 4), peak_tflops=peak,
                 peak_note=f"whole training steps (GEMMs, reductions, loss, Adam, gather) against the {peak_kind} "
                           "bf16 burst peak")
    seeds = [(0, j, 1e-10) for j in range(6)]
    walks = {}
    # the fast walk (steps up to 4 cm and 3 deg, a fresh motion every 10 frames) and a gentle one (2 cm,
    # 1.5 deg, every 25 frames)
    for wname, step_m, step_deg, jerk in (("fast", 0.04, 3.0, 10), ("gentle", 0.02, 1.5, 25)):
        wl = synth.room_smooth(seed=31000 + rank, frames=args.learned_frames, dims=512, voxel=0.005, step_m=step_m,
                               step_deg=step_deg, jerk_every=jerk, device=dev)
        starts = learn.start_errors(m, ds.scale, wl)
        arms = {}
        for name, seed_mode, use in (("constant_velocity", 1, False), ("constant_velocity_proposal", 1, True),
                                     ("previous_pose", 0, False), ("previous_pose_proposal", 0, True)):
            r = learn.track(wl, learn.handle_config(wl, seed_mode, 1e-5), seeds, mlp=m if use else None,
                            scale=ds.scale, judge_level=2)
            dt, dr = learn.pose_errors(r["poses"], wl.poses)
            c = r["counters"]
            row = dict(fps=round(r["fps"], 1), icp_iterations_per_frame=round(c["icp_iterations"] / (len(dt) - 1), 2),
                       failures=r["failures"], trans_err_cm_mean=round(float(dt.mean()) * 100, 3),
                       trans_err_cm_max=round(float(dt.max()) * 100, 3), rot_err_deg_mean=round(float(dr.mean()), 4),
                       rot_err_deg_max=round(float(dr.max()), 4))
            if use:
                row.update(judged=c["judged"], accepted=c["accepted"],
                           fallback_rate=round(1.0 - c["accepted"] / max(c["judged"], 1), 4))
            arms[name] = row
        walks[wname] = dict(walk=dict(step_m=step_m, step_deg=step_deg, fresh_motion_every=jerk),
                            start_error_sigma=dict((k, round(float(v.mean()), 3)) for k, v in starts.items()), **arms)
        del wl
    m.close()
    return dict(workload=f"{args.learned_frames} frames of a 640x480 camera with inertia in the room (rho = 0.9; a "
                         "fast and a gentle walk), 512^3 x 0.5 cm, K = 6 (d pose / d pose0), ICP stop tolerance "
                         "1e-5, judge at the coarsest level",
                train=train, network=f"{'-'.join(str(v) for v in learn.SIZES)} BF16, tcgen05 GEMMs", walks=walks)


# ------------------------------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ------------------------------------------------------------------------------------------------
def _reference(args, rank):
    if rank != 0:
        return
    R = args.ref_shards
    L = args.lanes
    procs = min(L, 6)
    wl = make_workload(args.workload, 2, 2, "cpu")
    payload = _wl_payload(wl, 2)
    with oracle_pool(procs) as pool:
        res = pool.map(_oracle_shard_steps, [(payload, (0, j % 6), R, args.warmup, args.steps) for j in range(procs)])
    step_s = np.max(np.stack([np.asarray(r) for r in res]), 0)  # the slowest lane per step
    frame_s = step_s.mean() * R * L / procs
    value = 1.0 / frame_s
    line = dict(impl="reference", metric=METRIC, value=round(value, 6), unit="frames/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(step_s.mean() * 1000, 2),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="c128", data="synthetic",
                config=dict(wl_desc(wl, L), parallelism="host cores"),
                cpu_baseline=dict(kind="oracle", cores=procs, value=round(value, 6), unit="frames/s",
                                  cpu_model=cpu_model(), host_cores=os.cpu_count(),
                                  sample=f"each step is shard s = step mod {R} of frame 1 of {wl.name}: 1/{R} of the "
                                         f"ICP pixels (19 iterations), of the voxels and of the ray-cast pixels, plus "
                                         f"1/{R} of the once-timed measurement (filter, pyramid, vertex and normal "
                                         f"maps); {procs} complex128 lanes in parallel processes; frames/s = "
                                         f"1 / ({R} x mean step)"),
                e2e=dict(value=round(value, 6), unit="frames/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=280)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("room256", "orbit64"), default="room256")
    ap.add_argument("--lanes", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 complex path beside the headline")
    ap.add_argument("--plain-steps", type=int, default=20, help="timed frames of the plain FP64 path")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-trajectories run")
    ap.add_argument("--no-second-order", action="store_true", help="skip the relocalisation / Hessian run")
    ap.add_argument("--reloc-frames", type=int, default=500)
    ap.add_argument("--reloc-queries", type=int, default=100)
    ap.add_argument("--reloc-tsdf-queries", type=int, default=30)
    ap.add_argument("--reloc-iters", type=int, default=30)
    ap.add_argument("--reloc-eta", type=float, default=1e-3)
    ap.add_argument("--no-learned", action="store_true", help="skip training and evaluating the learned proposal")
    ap.add_argument("--learned-rooms", type=int, default=110, help="room walks of 16 frames for the training pairs")
    ap.add_argument("--learned-epochs", type=int, default=30)
    ap.add_argument("--learned-frames", type=int, default=1000)
    ap.add_argument("--batch-n", type=int, default=32)
    ap.add_argument("--batch-min", type=int, default=50)
    ap.add_argument("--batch-max", type=int, default=400)
    ap.add_argument("--ref-shards", type=int, default=32)
    ap.add_argument("--details", default=None, help="write every measured figure to this JSON file")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        _reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
