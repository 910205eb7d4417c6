"""Shared helpers of the GPU parity tests: conversions between the oracle's one-complex-run-per-seed
results and the CUDA path's lane layout (lane 0 real, lane j the raw imaginary part of seed j)."""
import numpy as np

from oracle import pipeline as P
from oracle import se3

H_GPU = 1e-10  # imaginary step of the FP32 lanes
H_ORA = 1e-20  # imaginary step of the complex128 oracle


def oracle_cfg(wl):
    return P.Config(icp_iters=tuple(wl.icp_iters), depth_min=wl.depth_min, depth_max=wl.depth_max,
                    bilateral=wl.bilateral)


def xslam_cfg(wl):
    from paper_2405_02187_gb300 import xslam
    c = xslam.default_config()
    c.icp_levels = len(wl.icp_iters)
    for i, n in enumerate(wl.icp_iters):
        c.icp_iters[i] = n
    c.depth_min_m = wl.depth_min
    c.depth_max_m = wl.depth_max
    c.bilateral = int(wl.bilateral)
    return c


def make_handle(wl, max_lanes=6):
    from paper_2405_02187_gb300 import xslam
    return xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl), max_lanes=max_lanes)


def gpu_seeds(seeds, h=H_GPU):
    return [(s.kind, s.index, h) for s in seeds]


def pose_lanes(T_real, complex_poses, h_ora=H_ORA, h_gpu=H_GPU):
    """(1 + K, 3, 4) GPU pose lanes from the real pose and one complex pose per seed."""
    out = [np.asarray(T_real, np.float64)]
    for Tc in complex_poses:
        out.append(np.imag(Tc) / h_ora * h_gpu)
    return np.stack(out)


def promote_seeds(T, seeds, h=H_ORA):
    """Complex initial pose of each seed's oracle run (POSE0 seeds perturb T, others keep it)."""
    out = []
    for s in seeds:
        if s.kind == P.POSE0:
            out.append(se3.promote_pose(T, s.index, h))
        else:
            out.append(np.asarray(T, np.complex128))
    return out


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def assert_lanes_close(g, o, tol=1e-3, frac=0.999, max_err=1.0, frob=1e-3, what=""):
    """Element-wise comparison of a derivative lane g (GPU) with the oracle's o over a compared set.

    The lane's scale is max |o|. At least ``frac`` of the elements must lie within ``tol`` x scale of
    the oracle, no element may be further than ``max_err`` x scale away (an element whose discrete
    decision flipped between FP32 and FP64, e.g. a voxel clamped at F_D = 1 on one side only, can
    differ by up to the lane's scale), and the Frobenius relative error stays below ``frob``."""
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    assert g.shape == o.shape and g.size > 0, what
    assert np.all(np.isfinite(g)), what
    scale = np.abs(o).max()
    if scale == 0.0:
        assert np.abs(g).max() == 0.0, what
        return
    err = np.abs(g - o) / scale
    inside = (err <= tol).mean()
    assert inside >= frac, f"{what}: {inside:.5f} of {g.size} elements within {tol} of the scale {scale:.3e}"
    assert err.max() <= max_err, f"{what}: max error {err.max():.3e} of the scale"
    fr = rel_err(g, o)
    assert fr < frob, f"{what}: Frobenius relative error {fr:.3e}"


def f32_params(wl):
    """The workload and oracle Config with every parameter rounded to float32 as the C ABI passes it
    (voxel size, truncation, origin, intrinsics, gates, depth range), for comparisons at FP64 rounding."""
    import dataclasses
    import math

    from paper_2405_02187_gb300 import synth

    f = lambda v: float(np.float32(v))  # noqa: E731
    it = wl.intr
    intr = synth.Intrinsics(f(it.fx), f(it.fy), f(it.cx), f(it.cy), it.width, it.height)
    w = dataclasses.replace(wl, voxel=f(wl.voxel), trunc=f(wl.trunc), origin=tuple(f(o) for o in wl.origin),
                            intr=intr, depth_min=f(wl.depth_min), depth_max=f(wl.depth_max))
    cfg = P.Config(icp_iters=tuple(wl.icp_iters), dist_gate=f(0.1), normal_gate_deg=20.0, disc_gate=f(0.1),
                   min_corr_frac=f(0.1), depth_min=w.depth_min, depth_max=w.depth_max, pyr_range=f(0.09),
                   bilateral=wl.bilateral)
    assert math.isinf(cfg.w_max)
    return w, cfg


def _oracle_run_worker(args):
    """One oracle run (real when seed is None) over the first `frames` frames: its pose per frame."""
    wl, seed, frames, cfg = args
    r = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, seed)
    poses, oks = [], []
    for k in range(frames):
        T, ok = r.frame(wl.depth[k])
        poses.append(np.array(T))
        oks.append(ok)
    return poses, oks


def oracle_runs_parallel(wl, seeds, frames, cfg=None):
    """The real oracle run and one complex run per seed, each in its own spawned process (started
    with `spawn`, so a process that already holds a CUDA context is never forked). Returns a dict
    like oracle.pipeline.run's: pose (F, 3, 4), ok (F,), dtwist (K, F, 6)."""
    import concurrent.futures
    import multiprocessing

    cfg = cfg or oracle_cfg(wl)
    jobs = [(wl, None, frames, cfg)] + [(wl, s, frames, cfg) for s in seeds]
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=len(jobs), mp_context=ctx) as ex:
        res = list(ex.map(_oracle_run_worker, jobs))
    pose = np.stack(res[0][0])
    dtwist = np.zeros((len(seeds), frames, 6))
    for j, s in enumerate(seeds):
        for k in range(frames):
            dtwist[j, k] = se3.readout(res[j + 1][0][k], s.h)[2]
    return dict(pose=pose, ok=np.array(res[0][1]), dtwist=dtwist)
