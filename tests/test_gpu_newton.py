"""Newton ICP (xslam_config.icp_newton) on the GPU against the oracle's Newton tracker: the real
trajectory of the same sequence, frame by frame; and the lane restriction."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import make_handle, oracle_cfg, xslam_cfg
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _newton_handle(wl, eta=1e-4):
    cfg = xslam_cfg(wl)
    cfg.icp_newton = 1
    cfg.icp_newton_eta = eta
    return xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_lanes=2)


@pytest.mark.parametrize("which,eta", [("tiny", float("inf")), ("orbit", float("inf")), ("orbit", 1e-4)])
def test_newton_sequence_matches_oracle(which, eta):
    """eta = inf: Newton steps only; 1e-4: the switch to Gauss-Newton steps above it."""
    wl = synth.tiny(frames=3) if which == "tiny" else synth.small_orbit(frames=8)
    n = wl.depth.shape[0]
    x = _newton_handle(wl, eta)
    x.set_pose(wl.poses[0])
    out = [x.frame(torch.tensor(wl.depth[k], device="cuda"), []) for k in range(n)]
    ref = P.run(wl, [], frames=n, cfg=dataclasses.replace(oracle_cfg(wl), icp_newton=True, icp_newton_eta=eta))
    assert ref["ok"].all()
    for k in range(n):
        assert out[k][3] == xslam.OK
        assert np.abs(out[k][0] - ref["pose"][k]).max() < 1e-5, k
    # and close to the Gauss-Newton trajectory on this easy sequence
    g = make_handle(wl, max_lanes=0)
    g.set_pose(wl.poses[0])
    gn = [g.frame(torch.tensor(wl.depth[k], device="cuda"), []) for k in range(n)]
    assert max(np.abs(a[0][:, 3] - b[0][:, 3]).max() for a, b in zip(out, gn)) < 5e-3


def test_newton_rejects_lanes():
    wl = synth.tiny(frames=1)
    x = _newton_handle(wl)
    with pytest.raises(xslam.XSlamError) as e:
        x.frame(torch.tensor(wl.depth[0], device="cuda"), [(xslam.POSE0, 0, 1e-10)])
    assert e.value.status == xslam.EINVAL
