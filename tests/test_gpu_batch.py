"""Batched trajectories (include/xslam_batch.h): every trajectory of a batch gives, bit for bit, what
its own handle gives through xslam_frame on the same frames, whatever the other trajectories are
(image size, volume, lanes, length); the autotuner restores frame 0 and keeps parity with the oracle."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import gpu_seeds, make_handle, rel_err
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


def test_batch_matches_single_handles(monkeypatch):
    wls, seeds = _workloads()
    lengths = [4, 6, 5]
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    # reference: each trajectory alone through xslam_frame, with the ICP kernel a batch runs (one
    # launch per iteration; XSLAM_ICP_RUN=0 selects it for a handle created alone)
    monkeypatch.setenv("XSLAM_ICP_RUN", "0")
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


def test_batch_autotune_restores_frame0():
    wls, seeds = _workloads()
    dev = [torch.tensor(w.depth, device="cuda") for w in wls]
    bh = [_handle(w, s) for w, s in zip(wls, seeds)]
    batch = xslam.XSlamBatch(bh)
    frames = [[d[k] for d in dev] for k in range(4)]
    div, ms = batch.autotune(frames, 4)
    assert div in (1, 2, 4, 8, 16) and np.all(ms > 0)
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
