"""Training data, training and evaluation of the learned pose proposal (include/xslam_mlp.h).

Every computation runs behind the C ABI: the X-KinectFusion step tracks the training trajectories
(their ICP poses are the targets), xslam_mlp_features and xslam_mlp_pair_targets build the network's
inputs and targets, xslam_mlp_train trains on the GPU, xslam_set_proposal seeds ICP with the trained
network. This module only chooses the frames that are paired, the normalisation of the targets and
the runs to compare, and collects their results.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import synth, xslam

SIZES = (9600, 512, 512, 512, 6)


def handle_config(wl, icp_seed=0, icp_stop=0.0):
    c = xslam.default_config()
    c.icp_levels = len(wl.icp_iters)
    for i, n in enumerate(wl.icp_iters):
        c.icp_iters[i] = n
    c.depth_min_m = wl.depth_min
    c.depth_max_m = wl.depth_max
    c.bilateral = int(wl.bilateral)
    c.icp_seed = icp_seed
    c.icp_stop = icp_stop
    return c


@dataclasses.dataclass
class Dataset:
    feat: object      # CUDA bfloat16 (n_frames, 4800): every frame's features
    pairs: object     # CUDA int32 (P, 2): frame indices (earlier, later)
    targets: object   # CUDA float32 (P, 6): log(T_i^-1 T_j) / scale of the tracked poses
    scale: np.ndarray  # (6,) per-component standard deviation of the raw targets
    n_frames: int
    seconds: float    # rendering, tracking and feature time


def make_dataset(n_traj=10, frames=256, max_stride=8, seed=1000, dims=256, voxel=0.01, width=640, height=480,
                 reverse=False, device="cuda"):
    """Frame pairs (i, i + s), s = 1..max_stride, of n_traj room walks (the single-trajectory workload:
    640x480, 256^3 x 1 cm; each walk in its own random room) tracked by the X-KinectFusion step;
    targets from the tracked poses. reverse: also every pair the other way round (i + s, i)."""
    import torch
    t0 = time.perf_counter()
    feats, pairs, poses = [], [], []
    base = 0
    for t in range(n_traj):
        wl = synth.room_walk(seed=seed + t, frames=frames, dims=dims, voxel=voxel, width=width, height=height,
                             device=device, resident=True)
        x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, handle_config(wl), max_lanes=0)
        x.set_pose(wl.poses[0])
        tr = []
        for k in range(frames):
            pose, _, _, _ = x.frame(wl.depth[k])
            tr.append(pose)
        x.close()
        feats.append(xslam.features(wl.depth, wl.depth_min, wl.depth_max))
        for s in range(1, max_stride + 1):
            for i in range(frames - s):
                pairs.append((base + i, base + i + s))
                if reverse:
                    pairs.append((base + i + s, base + i))
        poses.append(np.array(tr))
        base += frames
    poses = np.concatenate(poses)
    pairs = np.array(pairs, np.int32)
    raw = xslam.pair_targets(poses, pairs, np.ones(6))
    scale = raw.std(0).astype(np.float64)
    tg = xslam.pair_targets(poses, pairs, scale)
    torch.cuda.synchronize()
    return Dataset(torch.cat(feats), torch.tensor(pairs, device=device), torch.tensor(tg, device=device), scale,
                   base, time.perf_counter() - t0)


def train(ds: Dataset, epochs=40, batch=256, lr=1e-3, seed=7, init_seed=3, mirror=True):
    """A fresh network of SIZES (He-uniform initial weights drawn on the host) trained on ds.
    Returns (mlp, per-epoch losses, training milliseconds measured with CUDA events)."""
    import torch
    rng = np.random.default_rng(init_seed)
    params = []
    for n_in, n_out in zip(SIZES[:-1], SIZES[1:]):
        bound = np.sqrt(6.0 / n_in)
        params.append((rng.uniform(-bound, bound, (n_out, n_in)), np.zeros(n_out)))
    m = xslam.Mlp(SIZES, max_batch=batch)
    m.set_params(params)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = m.train(ds.feat, ds.pairs, ds.targets, epochs=epochs, batch=batch, lr=lr, seed=seed, mirror=mirror)
    e1.record()
    torch.cuda.synchronize()
    return m, losses, e0.elapsed_time(e1)


def train_flops(n_pairs, batch, epochs):
    """Algorithmic GEMM flops of the training run: per row 2 n_in n_out per layer for the forward
    pass and the weight gradient, and again for the input gradient of every layer but the first."""
    steps = (n_pairs // batch) * epochs
    f = 0
    for l, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:])):
        f += 2 * a * b * (3 if l > 0 else 2)
    return steps * batch * f


def start_errors(m: xslam.Mlp, scale, wl):
    """Per frame k >= 2 of a workload with ground-truth poses: |start - truth| of the camera-frame
    motion T_{k-1}^-1 T_k guessed by the network, by constant velocity and by no motion, as twists
    in units of scale (the network's output units)."""
    import torch
    feat = xslam.features(wl.depth if hasattr(wl.depth, "is_cuda") else torch.tensor(wl.depth, device="cuda"),
                          wl.depth_min, wl.depth_max)
    n = feat.shape[0]
    idx = np.arange(2, n)
    x = torch.cat([feat[idx - 1], feat[idx]], 1).contiguous()
    ys = []
    for i in range(0, x.shape[0], m.max_batch):
        ys.append(m.forward(x[i:i + m.max_batch]).cpu().numpy())
    y = np.concatenate(ys)
    truth = xslam.pair_targets(wl.poses, np.stack([idx - 1, idx], 1), scale)
    cv = xslam.pair_targets(wl.poses, np.stack([idx - 2, idx - 1], 1), scale)
    e = lambda a: np.linalg.norm(a - truth, axis=1)  # noqa: E731
    return dict(network=e(y), constant_velocity=e(cv), no_motion=np.linalg.norm(truth, axis=1))


def track(wl, cfg, seeds, mlp=None, scale=None, judge_level=2, timed=True):
    """Track workload wl (depth resident on the GPU) with handle configuration cfg and the given
    seeds, optionally with the learned proposal. Returns dict: poses (n, 3, 4), frames/s of a timed
    pass (CUDA events over the whole sequence, no host reads), counters and the ICP failures."""
    import torch
    x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_lanes=len(seeds))
    if mlp is not None:
        x.set_proposal(mlp, scale, judge_level)
    out = {}
    n = wl.depth.shape[0]
    if timed:
        x.set_pose(wl.poses[0])
        x.frame(wl.depth[0], seeds, outputs=False)
        x.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(1, n):
            x.frame(wl.depth[k], seeds, outputs=False)
        e1.record()
        _, nfail = x.sync()
        out["fps"] = (n - 1) / (e0.elapsed_time(e1) / 1e3)
        x.reset()
        x.counters(reset=True)
    x.set_pose(wl.poses[0])
    poses, fails = [], 0
    for k in range(n):
        pose, _, _, st = x.frame(wl.depth[k], seeds)
        poses.append(pose)
        fails += int(st == xslam.ENOTRACK)
    out["counters"] = x.counters()
    out["failures"] = fails
    out["poses"] = np.array(poses)
    x.close()
    return out


def pose_errors(poses, truth):
    """Translation (m) and rotation (deg) error of each frame against the ground truth."""
    dt = np.linalg.norm(poses[:, :, 3] - truth[:, :, 3], axis=1)
    R = np.einsum("nij,nkj->nik", poses[:, :, :3], truth[:, :, :3])
    c = np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1)
    return dt, np.degrees(np.arccos(c))


def main(argv=None):
    """Build a training set, train, and print one JSON line (the small case the GEMM profiles use)."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train the learned pose proposal")
    ap.add_argument("--rooms", type=int, default=8)
    ap.add_argument("--frames", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--batch", type=int, default=256)
    a = ap.parse_args(argv)
    xslam.load()
    ds = make_dataset(n_traj=a.rooms, frames=a.frames, reverse=True, seed=20000)
    m, losses, ms = train(ds, epochs=a.epochs, batch=a.batch, mirror=True)
    flops = train_flops(int(ds.pairs.shape[0]), a.batch, a.epochs)
    print(json.dumps(dict(pairs=int(ds.pairs.shape[0]), epochs=a.epochs, batch=a.batch, train_ms=round(ms, 2),
                          tflops=round(flops / (ms * 1e9), 2), loss=[round(float(v), 4) for v in losses])))
    m.close()


if __name__ == "__main__":
    main()
