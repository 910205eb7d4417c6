"""End to end at the headline configuration: frames 0-2 of the 640x480 room walk in the 256^3 x 1 cm
volume, bilateral filter on, through xslam_frame, against whole oracle frames (X-SLAM Sec. 4.1).

Lanes: two POSE0 directions and the all-pixel DEPTH seed (the oracle runs one complex run per lane,
each in its own process). This pins the real pose, its derivatives and the 6x6 solve at the
conditioning of the full-size frames: pose within 1e-5 m / rad of the oracle, twist blocks within 1e-3
relative."""
import numpy as np
import pytest

from gpu_helpers import gpu_seeds, make_handle, oracle_runs_parallel, rel_err
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAMES = 3


def test_headline_frames_match_oracle():
    wl = synth.room_walk(frames=FRAMES)
    assert wl.bilateral and wl.dims == (256, 256, 256) and wl.intr.width == 640
    seeds = [P.Seed(P.POSE0, 1), P.Seed(P.POSE0, 3), P.Seed(P.DEPTH, -1)]
    ref = oracle_runs_parallel(wl, seeds, FRAMES)
    assert ref["ok"].all()
    x = make_handle(wl, max_lanes=6)
    x.set_pose(wl.poses[0])
    dev = torch.tensor(wl.depth, device="cuda")
    for k in range(FRAMES):
        pose, _, dtw, st = x.frame(dev[k], gpu_seeds(seeds))
        assert st == xslam.OK
        assert np.abs(pose - ref["pose"][k]).max() < 1e-5, k
        for j in range(len(seeds)):
            assert rel_err(dtw[j], ref["dtwist"][j, k]) < 1e-3, (k, j, dtw[j], ref["dtwist"][j, k])
