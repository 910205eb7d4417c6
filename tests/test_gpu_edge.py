"""Edge cases of the CUDA path against the oracle: the maximum lane count, no lanes, ragged volume and
image sizes, the relocalisation gradient (xslam_grad), argument and state errors, and reset."""
import numpy as np
import pytest

from gpu_helpers import H_GPU, gpu_seeds, make_handle, rel_err
from oracle import pipeline as P
from oracle import measure, reloc, se3
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sequence(wl, seeds, frames, max_lanes=None):
    x = make_handle(wl, max_lanes=max(1, len(seeds)) if max_lanes is None else max_lanes)
    x.set_pose(wl.poses[0])
    out = [x.frame(torch.tensor(wl.depth[k], device="cuda"), gpu_seeds(seeds)) for k in range(frames)]
    return x, out


def _check(wl, seeds, frames, out):
    ref = P.run(wl, seeds, frames=frames)
    assert ref["ok"].all()
    for k in range(frames):
        pose, dpose, dtw, st = out[k]
        assert st == xslam.OK
        assert np.abs(pose - ref["pose"][k]).max() < 1e-5, k
        for j, s in enumerate(seeds):
            if s.kind == P.POSE0:
                assert rel_err(dtw[j], ref["dtwist"][j, k]) < 1e-3, (k, j)
            else:
                assert np.abs(dtw[j] - ref["dtwist"][j, k]).max() < 1e-3 * max(1.0, np.abs(ref["dtwist"][j, k]).max())


def test_maximum_lanes():
    """15 imaginary lanes (the C ABI's maximum): every lane matches its own oracle run."""
    wl = synth.tiny(frames=3)
    seeds = [P.Seed(P.POSE0, j % 6) for j in range(12)] + [P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1), P.Seed(P.POSE0, 5)]
    assert len(seeds) == 15
    _, out = _sequence(wl, seeds, 3)
    _check(wl, seeds, 3, out)


def test_no_lanes_is_the_real_pipeline():
    wl = synth.small_orbit(frames=6)
    _, out = _sequence(wl, [], 6, max_lanes=0)
    ref = P.run(wl, [], frames=6)
    for k in range(6):
        assert np.abs(out[k][0] - ref["pose"][k]).max() < 1e-5


def test_ragged_sizes():
    """Volume dims that are not multiples of any block size and a 44x36 image (last chunk partial)."""
    base = synth.tiny(frames=3, n=28, width=44, height=36)
    dims = (28, 26, 25)
    origin = tuple(-d * base.voxel / 2 for d in dims)
    wl = synth.Workload(base.name + "_ragged", base.intr, dims, base.voxel, base.trunc, origin, base.poses,
                        base.depth, base.scene, base.seed, icp_iters=base.icp_iters)
    seeds = [P.Seed(P.POSE0, 1), P.Seed(P.POSE0, 3)]
    _, out = _sequence(wl, seeds, 3)
    _check(wl, seeds, 3, out)


def test_relocalisation_gradient():
    """xslam_grad (order 1) against the oracle's complex-step gradient on the GPU's own volume."""
    wl = synth.small_orbit(frames=4)
    x, _ = _sequence(wl, [], 3, max_lanes=6)  # xslam_grad needs room for 6 lanes and no sequence lanes
    n = x.n_vox
    buf = torch.empty(n, device="cuda")
    F = x.read_tsdf(0, buf).cpu().numpy().astype(np.float64)
    W = x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64)
    T = se3.compose(se3.se3_exp(np.array([0.01, -0.006, 0.004, 0.008, 0.004, -0.006])), wl.poses[3])
    q = torch.tensor(wl.depth[3], device="cuda")
    Eg, gg = x.grad(q, T)
    D = measure.range_gate(wl.depth[3].astype(np.float64), wl.depth_min, wl.depth_max)
    Eo, go, n = reloc.gradient(F, W, T, D, wl.intr, wl.dims, wl.origin, wl.voxel, depth_min=wl.depth_min,
                               depth_max=wl.depth_max)
    assert n > 1000
    assert abs(Eg - Eo) <= 1e-3 * Eo
    assert rel_err(gg, go) < 1e-3


def test_argument_and_state_errors():
    wl = synth.tiny(frames=2)
    x = make_handle(wl, max_lanes=2)
    d = torch.tensor(wl.depth[0], device="cuda")
    for bad in ([(xslam.POSE, 6, H_GPU)], [(xslam.DEPTH, 10 ** 8, H_GPU)], [(xslam.POSE0, 0, 0.0)],
                [(xslam.POSE0, 7, H_GPU)], [(xslam.POSE0, 0, H_GPU)] * 3):
        with pytest.raises(xslam.XSlamError) as e:
            x.frame(d, bad)
        assert e.value.status == xslam.EINVAL
    x.frame(d, [(xslam.POSE0, 0, H_GPU)])
    with pytest.raises(xslam.XSlamError) as e:
        x.set_pose(wl.poses[0])
    assert e.value.status == xslam.ESTATE
    with pytest.raises(xslam.XSlamError) as e:
        x.grad(d, wl.poses[0])  # sequence lanes in use
    assert e.value.status in (xslam.ESTATE, xslam.EINVAL)


def test_reset_restarts_the_sequence():
    wl = synth.tiny(frames=3)
    seeds = [P.Seed(P.POSE0, 2)]
    x, a = _sequence(wl, seeds, 3)
    x.reset()
    x.set_pose(wl.poses[0])
    b = [x.frame(torch.tensor(wl.depth[k], device="cuda"), gpu_seeds(seeds)) for k in range(3)]
    for ra, rb in zip(a, b):
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[2], rb[2])
