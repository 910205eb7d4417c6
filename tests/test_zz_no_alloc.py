"""xslam_icp_system_noalloc against xslam_icp_system through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory where they need the
ICP normal equations (framework-owned memory pools, real-time loops, plug-ins restricted to the
buffers their host hands them). It keeps its scratch in a fixed file-scope device array, so this test
also checks that two calls in a row, sharing that array, both reproduce the handle-based call.
This file is collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _seed_set(n):
    from oracle import pipeline as P
    if n == 3:
        return [P.Seed(P.POSE0, 0), P.Seed(P.POSE0, 3), P.Seed(P.DEPTH, -1)]
    # 15 lanes: the largest lane count, whose partial sums use the largest stride of the fixed array
    s = [P.Seed(P.POSE0, j) for j in range(6)] + [P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)]
    s += [P.Seed(P.POSE0, j, h=2e-20) for j in range(6)] + [P.Seed(P.TRUNC, h=3e-20)]
    assert len(s) == 15
    return s


@pytest.mark.parametrize("n_seeds,levels", [(3, (0, 2)), (15, (0,))], ids=["4_lanes", "16_lanes"])
def test_icp_system_noalloc_matches_handle_call(n_seeds, levels):
    from gpu_helpers import H_GPU, gpu_seeds, make_handle, rel_err, xslam_cfg
    from oracle import se3
    from paper_2405_02187_gb300 import synth, xslam

    wl = synth.small_orbit(frames=5)
    seeds = _seed_set(n_seeds)
    L = 1 + len(seeds)
    x = make_handle(wl, max_lanes=max(6, len(seeds)))
    x.set_pose(wl.poses[0])
    dev = [torch.tensor(wl.depth[k], device="cuda") for k in range(5)]
    for k in range(3):
        x.frame(dev[k], gpu_seeds(seeds))
    T_prev = x.get_pose_lanes()
    H, W = wl.intr.height, wl.intr.width
    dep = torch.empty((H, W), device="cuda")
    vm = torch.empty((3 * L, H, W), device="cuda")
    nm = torch.empty((3 * L, H, W), device="cuda")
    x.raycast(T_prev, dep, vm, nm)
    x.set_model(dep, vm, nm, T_prev)
    model = torch.cat([dep[None], vm, nm], 0).contiguous()
    # a pose estimate away from the model pose on every lane
    Tj = T_prev.copy()
    Tj[0] = se3.compose(se3.se3_exp(np.array([0.004, -0.002, 0.003, 0.005, 0.002, -0.004])), T_prev[0])
    cfg = xslam_cfg(wl)
    for level in levels:
        lvl = torch.empty((H >> level, W >> level), device="cuda")
        x.measure(dev[3], level, lvl)
        ref, n_ref = x.icp_system(level, Tj)
        assert n_ref > 100
        outs = []
        for _ in range(2):  # two calls in a row share the scratch array
            out, n = xslam.icp_system_noalloc(lvl, level, wl.intr, model, Tj, T_prev, gpu_seeds(seeds), cfg)
            assert n == n_ref
            assert rel_err(out[0], ref[0]) < 1e-5
            for j in range(1, L):
                assert rel_err(out[j] / H_GPU, ref[j] / H_GPU) < 1e-4, (level, j)
            outs.append(out)
        assert np.array_equal(outs[0], outs[1])


def test_icp_system_noalloc_rejects_too_many_lanes():
    from paper_2405_02187_gb300 import synth, xslam

    wl = synth.small_orbit(frames=1)
    H, W = wl.intr.height, wl.intr.width
    d = torch.zeros((H, W), device="cuda")
    m = torch.zeros((1 + 6 * 17, H, W), device="cuda")
    T = np.zeros((17, 3, 4))
    seeds = [(xslam.POSE0, 0, 1e-10)] * 16
    with pytest.raises(xslam.XSlamError) as e:
        xslam.icp_system_noalloc(d, 0, wl.intr, m, T, T, seeds)
    assert e.value.status == xslam.EINVAL and "0..15" in str(e.value)
