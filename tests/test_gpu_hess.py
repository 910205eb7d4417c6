"""xslam_grad order 2 (truncated-bicomplex FP32 lanes on the GPU) against the oracle's bicomplex
Hessian of the relocalisation loss, evaluated on the GPU's own volume; and against order 1."""
import numpy as np
import pytest

from gpu_helpers import gpu_seeds, make_handle, rel_err
from oracle import measure, reloc, se3
from paper_2405_02187_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OFFSETS = [np.array([0.01, -0.006, 0.004, 0.008, 0.004, -0.006]), np.array([-0.004, 0.002, 0.006, -0.01, 0.003, 0.002]),
           np.zeros(6)]


@pytest.fixture(scope="module")
def mapped():
    wl = synth.small_orbit(frames=5)
    x = make_handle(wl, max_lanes=6)
    x.set_pose(wl.poses[0])
    for k in range(4):
        x.frame(torch.tensor(wl.depth[k], device="cuda"), [])
    buf = torch.empty(x.n_vox, device="cuda")
    F = x.read_tsdf(0, buf).cpu().numpy().astype(np.float64)
    W = x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64)
    return wl, x, F, W


@pytest.mark.parametrize("off", range(len(OFFSETS)))
def test_hessian_matches_oracle(mapped, off):
    wl, x, F, W = mapped
    T = se3.compose(se3.se3_exp(OFFSETS[off]), wl.poses[4])
    q = torch.tensor(wl.depth[4], device="cuda")
    E, g, H = x.grad(q, T, order=2)
    D = measure.range_gate(wl.depth[4].astype(np.float64), wl.depth_min, wl.depth_max)
    Eo, go, Ho = reloc.hessian_bicomplex(F, W, T, D, wl.intr, wl.dims, wl.origin, wl.voxel, depth_min=wl.depth_min,
                                         depth_max=wl.depth_max)
    assert abs(E - Eo) <= 1e-3 * Eo
    assert rel_err(g, go) < 1e-3
    assert rel_err(H, Ho) < 2e-3
    assert np.abs(H - H.T).max() == 0.0
    # order 1 (six first-order lanes through the model maps) gives the same loss and gradient
    E1, g1 = x.grad(q, T, order=1)
    assert abs(E1 - E) <= 1e-4 * E and rel_err(g1, g) < 1e-3


def test_newton_step_from_the_hessian(mapped):
    """A Newton step -H^-1 g from a displaced pose lands closer to the pose the frame was taken at than
    the displacement (the loss is near-quadratic in the twist around the optimum)."""
    wl, x, _, _ = mapped
    q = torch.tensor(wl.depth[4], device="cuda")
    T = se3.compose(se3.se3_exp(0.5 * OFFSETS[0]), wl.poses[4])
    E, g, H = x.grad(q, T, order=2)
    step = -np.linalg.solve(H, g)
    T1 = se3.compose(se3.se3_exp(step), T)
    d0 = np.linalg.norm(T[:, 3] - wl.poses[4][:, 3])
    d1 = np.linalg.norm(T1[:, 3] - wl.poses[4][:, 3])
    E1, _ = x.grad(q, T1, order=1)
    assert E1 < E and d1 < 0.5 * d0


@pytest.mark.parametrize("off", [0, 1])
def test_plain64_hessian_matches_oracle_and_fp32(mapped, off):
    """xslam_grad_plain64: the paper's bicomplex arithmetic in FP64 (full products, h = 1e-20, its own
    FP64 march and decisions) against the oracle's bicomplex Hessian on the same volume (1e-5), and the
    FP32 truncated path against it (2e-3)."""
    wl, x, F, W = mapped
    T = se3.compose(se3.se3_exp(OFFSETS[off]), wl.poses[4])
    q = torch.tensor(wl.depth[4], device="cuda")
    E64, g64, H64 = x.grad_plain64(q, T)
    D = measure.range_gate(wl.depth[4].astype(np.float64), wl.depth_min, wl.depth_max)
    Eo, go, Ho = reloc.hessian_bicomplex(F, W, T, D, wl.intr, wl.dims, wl.origin, wl.voxel, depth_min=wl.depth_min,
                                         depth_max=wl.depth_max)
    assert abs(E64 - Eo) <= 1e-5 * Eo
    assert rel_err(g64, go) < 1e-5 and rel_err(H64, Ho) < 1e-5
    E, g, H = x.grad(q, T, order=2)
    assert rel_err(g, g64) < 1e-3 and rel_err(H, H64) < 2e-3
