"""Batched trajectories (include/xslam_batch.h): every trajectory of a batch gives, bit for bit, what
its own handle gives through xslam_frame on the same frames, whatever the other trajectories are
(image size, volume, lanes, length); the autotuner restores frame 0 and keeps parity with the oracle."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import gpu_seeds, make_handle, rel_err, xslam_cfg
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _workloads():
    a = synth.tiny(frames=4)
    b = synth.small_orbit(frames=6)
    c = synth.tiny(seed=5, frames=5, n=28, width=48, height=36)
    seeds = [[P.Seed(P.POSE0, 1), P.Seed(P.POSE0, 4)], [P.Seed(P.TRUNC)], [P.Seed(P.POSE0, 2), P.Seed(P.DEPTH, -1),
                                                                          P.Seed(P.POSE0, 0)]]
    return [a, b, c], seeds


def _handle(wl, seeds):
    x = make_handle(wl, max_lanes=max(1, len(seeds)))
    x.set_lanes(gpu_seeds(seeds))
    x.set_pose(wl.poses[0])
    return x


def test_batch_matches_single_handles():
    wls, seeds = _workloads()
    lengths = [4, 6, 5]
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    # reference: each trajectory alone through xslam_frame
    ref = []
    for wl, sd, d, n in zip(wls, seeds, dev, lengths):
        x = make_handle(wl, max_lanes=max(1, len(sd)))
        x.set_pose(wl.poses[0])
        ref.append([x.frame(d[k], gpu_seeds(sd)) for k in range(n)])
    bh = [_handle(w, s) for w, s in zip(wls, seeds)]
    batch = xslam.XSlamBatch(bh)
    for k in range(max(lengths)):
        batch.step([d[k] if k < n else None for d, n in zip(dev, lengths)])
        for i, n in enumerate(lengths):
            if k < n:
                pose, dpose, dtw = batch.read(i)
                rp, rdp, rtw, _ = ref[i][k]
                assert np.array_equal(pose, rp), (i, k)
                assert np.array_equal(dpose, rdp) and np.array_equal(dtw, rtw), (i, k)
        lat = batch.latency()
        assert all((lat[i] > 0) == (k < n) for i, n in enumerate(lengths))
    assert batch.sync() == [0, 0, 0]


def test_batch_modes_agree_and_profile():
    """Branch mode (every trajectory's own chain as a graph branch) and segmented mode (one launch per
    stage) give the same bits; the segmented step's launch profile lists its stages in order."""
    wls, seeds = _workloads()
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    out = {}
    for mode in ("branches", "segmented"):
        bh = [_handle(w, s) for w, s in zip(wls, seeds)]
        batch = xslam.XSlamBatch(bh)
        batch.set_shapes(dict(icp_divisor=2, fuse_blocks_per_sm=0, ray_tile="32x8", mode=mode))
        batch.profile(True)
        for k in range(4):
            batch.step([d[k] for d in dev])
        prof = batch.profile_read()
        out[mode] = [batch.read(i) for i in range(len(wls))]
        if mode == "branches":
            assert prof == []
        else:
            stages = [p[0] for p in prof]
            assert stages[0] == "measure" and stages[-1] == "readout"
            # every trajectory tracks a 2-level pyramid with 10 + 5 iterations (tiny) or 3 levels (orbit)
            assert stages.count("icp") == max(sum(w.icp_iters) for w in wls)
            assert all(p[2] > 0 and p[3] >= 0 for p in prof) and sum(p[3] for p in prof) > 0
            assert stages.index("update") > stages.index("tiles") > stages.index("icp")
        batch.close()
    for a, b in zip(out["branches"], out["segmented"]):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


def test_batch_autotune_restores_frame0():
    wls, seeds = _workloads()
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    bh = [_handle(w, s) for w, s in zip(wls, seeds)]
    batch = xslam.XSlamBatch(bh)
    frames = [[d[k] for d in dev] for k in range(4)]
    choice, ms = batch.autotune(frames, 4)
    assert choice["icp_divisor"] in (1, 2, 4, 8, 16, 32) and choice["fuse_blocks_per_sm"] in (0, 1, 2, 4)
    assert choice["ray_tile"] in ("32x8", "16x16", "64x4") and choice["mode"] in ("segmented", "branches")
    # mode (2), divisor (6), then fusion (4) and tile (3) in segmented mode
    assert len(ms) == (15 if choice["mode"] == "segmented" else 8) and np.all(ms > 0)
    # from frame 0 again, on the chosen grids: parity with the oracle
    for k in range(4):
        batch.step([d[k] for d in dev])
    for i, (wl, sd) in enumerate(zip(wls, seeds)):
        ref = P.run(wl, sd, frames=4)
        pose, _, dtw = batch.read(i)
        assert np.abs(pose - ref["pose"][3]).max() < 1e-5
        for j, s in enumerate(sd):
            if s.kind == P.POSE0:
                assert rel_err(dtw[j], ref["dtwist"][j, 3]) < 1e-3


def test_batch_gives_the_handles_back():
    """After the autotuner changed their ICP grids, a destroyed batch leaves its handles as they were: a
    reset handle gives a fresh handle's bits; a handle in a live batch cannot join a second one."""
    wls, seeds = _workloads()
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    bh = [_handle(w, s) for w, s in zip(wls, seeds)]
    batch = xslam.XSlamBatch(bh)
    with pytest.raises(xslam.XSlamError):
        xslam.XSlamBatch(bh[:1])
    batch.set_shapes(dict(icp_divisor=8, fuse_blocks_per_sm=0, ray_tile="32x8", mode="segmented"))
    for k in range(3):
        batch.step([d[k] for d in dev])
    batch.close()
    for wl, sd, d, x in zip(wls, seeds, dev, bh):
        x.reset()
        x.set_pose(wl.poses[0])
        y = make_handle(wl, max_lanes=max(1, len(sd)))
        y.set_pose(wl.poses[0])
        for k in range(3):
            a = x.frame(d[k], gpu_seeds(sd))
            b = y.frame(d[k], gpu_seeds(sd))
            assert all(np.array_equal(u, v) for u, v in zip(a[:3], b[:3])), k


def test_batch_of_own_chains_matches_single_handles():
    """A handle outside the plain frame chain (here a constant-velocity ICP start) makes the batch run
    every trajectory's own chain as a graph branch; each still equals its handle bit for bit."""
    wls, seeds = _workloads()
    lengths = [4, 5, 5]
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]

    def handle(wl, sd):
        c = xslam_cfg(wl)
        c.icp_seed = 1
        x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, c, max_lanes=max(1, len(sd)))
        return x

    ref = []
    for wl, sd, d, n in zip(wls, seeds, dev, lengths):
        x = handle(wl, sd)
        x.set_pose(wl.poses[0])
        ref.append([x.frame(d[k], gpu_seeds(sd)) for k in range(n)])
    bh = []
    for wl, sd in zip(wls, seeds):
        x = handle(wl, sd)
        x.set_lanes(gpu_seeds(sd))
        x.set_pose(wl.poses[0])
        bh.append(x)
    batch = xslam.XSlamBatch(bh)
    for k in range(max(lengths)):
        batch.step([d[k] if k < n else None for d, n in zip(dev, lengths)])
        for i, n in enumerate(lengths):
            if k < n:
                pose, dpose, dtw = batch.read(i)
                rp, rdp, rtw, _ = ref[i][k]
                assert np.array_equal(pose, rp) and np.array_equal(dtw, rtw), (i, k)


def test_batch_errors():
    wl = synth.tiny(frames=2)
    x = _handle(wl, [P.Seed(P.POSE0, 0)])
    with pytest.raises(xslam.XSlamError):
        xslam.XSlamBatch([x, x])
    batch = xslam.XSlamBatch([x])
    with pytest.raises(xslam.XSlamError) as e:
        batch.step([None])
    assert e.value.status == xslam.EINVAL
    batch.step([torch.tensor(wl.depth[0], device="cuda")])
    batch.sync()
    y = _handle(wl, [P.Seed(P.POSE0, 0)])
    y.frame(torch.tensor(wl.depth[0], device="cuda"), [(xslam.POSE0, 0, 1e-10)])
    with pytest.raises(xslam.XSlamError):  # past frame 0
        xslam.XSlamBatch([y])
