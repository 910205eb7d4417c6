"""The plain FP64 complex path (include/xslam_plain.h) against the oracle: both evaluate the same
complex<double> pipeline, one complex run per seed, so given the same float32-rounded parameters
(the C ABI passes voxel size, truncation, origin, intrinsics and gates as float) they agree to FP64
rounding; and against the batched FP32 lanes, which must agree with it to the derivative tolerance."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import H_ORA, f32_params, gpu_seeds, make_handle, rel_err, xslam_cfg
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f32(wl):
    w, cfg = f32_params(wl)
    return w, cfg


def _plain(wl, seeds, frames, max_runs=None, h=H_ORA):
    x = xslam.XSlamPlain(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl),
                         max_runs=max_runs or max(1, len(seeds)))
    x.set_pose(wl.poses[0])
    out = [x.frame(torch.tensor(wl.depth[k], device="cuda"), gpu_seeds(seeds, h)) for k in range(frames)]
    return x, out


@pytest.mark.parametrize("bilateral", [False, True])
def test_plain_matches_oracle_tiny(bilateral):
    wl = dataclasses.replace(synth.tiny(frames=3), bilateral=bilateral)
    seeds = [P.Seed(P.POSE0, 0), P.Seed(P.POSE0, 4), P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)]
    x, out = _plain(wl, seeds, 3)
    w32, c32 = _f32(wl)
    ref = P.run(w32, seeds, frames=3, cfg=c32)
    for k in range(3):
        pose, dpose, dtw, st = out[k]
        assert st == xslam.OK
        assert np.abs(pose - ref["pose"][k]).max() < 1e-10
        for j in range(len(seeds)):
            # relative to the derivative's scale, with a floor of 1: d pose / d mu vanishes (to 1e-17)
            # once ICP has converged on the noise-free scene
            for a, b in ((dpose[j], ref["dpose"][j, k]), (dtw[j], ref["dtwist"][j, k])):
                assert np.abs(a - b).max() <= 1e-8 * max(1.0, np.abs(b).max()), (k, j)
    # the TSDF of every run: real part and derivative
    buf = torch.empty(x.n_vox, device="cuda", dtype=torch.float64)
    for j in range(len(seeds)):
        r = ref["runs"][j + 1]
        F = x.read_tsdf(j, 0, buf).cpu().numpy()
        W = x.read_tsdf(j, 2, buf).cpu().numpy()
        dF = x.read_tsdf(j, 1, buf).cpu().numpy()
        assert np.array_equal(W, r.W)
        assert np.abs(F - r.F.real).max() < 1e-10
        assert rel_err(dF, r.F.imag / H_ORA) < 1e-8


def test_plain_sequence_and_fp32_lanes():
    """6 POSE0 runs over 6 frames of the 64^3 orbit: oracle to FP64 rounding; the batched FP32 lanes
    to the derivative tolerance."""
    wl = synth.small_orbit(frames=6)
    seeds = [P.Seed(P.POSE0, j) for j in range(6)]
    _, out = _plain(wl, seeds, 6)
    w32, c32 = _f32(wl)
    ref = P.run(w32, seeds, frames=6, cfg=c32)
    g = make_handle(wl, max_lanes=6)
    g.set_pose(wl.poses[0])
    for k in range(6):
        pose, _, dtw, st = out[k]
        assert st == xslam.OK
        assert np.abs(pose - ref["pose"][k]).max() < 1e-10
        assert rel_err(dtw, ref["dtwist"][:, k]) < 1e-8
        gp, _, gtw, gst = g.frame(torch.tensor(wl.depth[k], device="cuda"), gpu_seeds(seeds))
        assert np.abs(gp - pose).max() < 1e-5
        if k > 0:
            assert rel_err(gtw, dtw) < 1e-3


def test_plain_without_seeds_is_the_real_pipeline():
    wl = synth.small_orbit(frames=4)
    _, out = _plain(wl, [], 4, max_runs=1)
    w32, c32 = _f32(wl)
    ref = P.run(w32, [], frames=4, cfg=c32)
    for k in range(4):
        assert np.abs(out[k][0] - ref["pose"][k]).max() < 1e-10
        assert out[k][1].shape == (0, 3, 4)


def test_plain_argument_errors():
    wl = synth.tiny(frames=2)
    x = xslam.XSlamPlain(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl), max_runs=2)
    d = torch.tensor(wl.depth[0], device="cuda")
    for bad in ([(xslam.POSE0, 0, H_ORA)] * 3, [(xslam.POSE, 0, H_ORA)], [(xslam.DEPTH, 3, H_ORA)],
                [(xslam.POSE0, 6, H_ORA)], [(xslam.POSE0, 0, 0.0)]):
        with pytest.raises(xslam.XSlamError) as e:
            x.frame(d, bad)
        assert e.value.status == xslam.EINVAL
    x.frame(d, [(xslam.TRUNC, 0, H_ORA)])
    with pytest.raises(xslam.XSlamError) as e:
        x.frame(d, [(xslam.TRUNC, 0, 2 * H_ORA)])
    assert e.value.status == xslam.ESTATE
    with pytest.raises(xslam.XSlamError) as e:
        x.set_pose(wl.poses[0])
    assert e.value.status == xslam.ESTATE
    with pytest.raises(xslam.XSlamError):
        xslam.XSlamPlain(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, xslam_cfg(wl), max_runs=17)
