"""xslam_grad_tsdf (the paper's TSDF-difference relocalisation loss, Sec. 5.2, with its gradient and
truncated-bicomplex Hessian on the GPU) against the oracle's complex-step gradient and bicomplex
Hessian (oracle/reloc.py tsdf_*), evaluated on the GPU's own volume; and the properties that hold at
any size: zero loss and gradient where the query repeats the frame the volume was fused from, a
Gauss-Newton (positive semi-definite) Hessian there, order 1 agreeing with order 2, and the volume
left unchanged."""
import numpy as np
import pytest

from gpu_helpers import make_handle, rel_err
from oracle import measure, reloc, se3
from paper_2405_02187_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

START = np.array([0.0, 0.004, 0.0, 0.01, 0.0, 0.0])  # 1 cm and 0.23 degrees off
OFFSETS = [np.array([0.01, -0.006, 0.004, 0.008, 0.004, -0.006]), np.array([-0.004, 0.002, 0.006, -0.01, 0.003, 0.002]),
           np.zeros(6)]


@pytest.fixture(scope="module")
def mapped():
    wl = synth.small_orbit(frames=5)
    x = make_handle(wl, max_lanes=0)
    x.set_pose(wl.poses[0])
    for k in range(4):
        x.frame(torch.tensor(wl.depth[k], device="cuda"), [])
    buf = torch.empty(x.n_vox, device="cuda")
    F = x.read_tsdf(0, buf).cpu().numpy().astype(np.float64)
    W = x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64)
    return wl, x, F, W


def _oracle(wl, F, W, T, depth):
    D = measure.range_gate(depth.astype(np.float64), wl.depth_min, wl.depth_max)
    E, g, H = reloc.tsdf_hessian_bicomplex(F, W, T, D, wl.intr, wl.dims, wl.origin, wl.voxel, wl.trunc)
    keep = reloc.tsdf_decisions(F, W, T, D, wl.intr, wl.dims, wl.origin, wl.voxel, wl.trunc)[0]
    n = int(np.count_nonzero(keep & (W > 0)))
    return E, g, H, n


@pytest.mark.parametrize("off", range(len(OFFSETS)))
def test_matches_oracle(mapped, off):
    wl, x, F, W = mapped
    T = se3.compose(se3.se3_exp(OFFSETS[off]), wl.poses[4])
    q = torch.tensor(wl.depth[4], device="cuda")
    E, g, H, n = x.grad_tsdf(q, T, order=2)
    Eo, go, Ho, no = _oracle(wl, F, W, T, wl.depth[4])
    print(off, E, Eo, n, no, rel_err(g, go), rel_err(H, Ho))
    # a voxel whose update decision sits on a boundary may fall either way in FP32
    assert abs(n - no) <= max(2, 1e-4 * no)
    assert abs(E - Eo) <= 2e-3 * Eo
    assert rel_err(g, go) < 2e-3
    assert rel_err(H, Ho) < 2e-3
    assert np.abs(H - H.T).max() == 0.0
    E1, g1, H1, n1 = x.grad_tsdf(q, T, order=1)
    assert n1 == n and abs(E1 - E) <= 1e-6 * E and rel_err(g1, g) < 1e-6
    assert H1 is None


def test_volume_unchanged(mapped):
    wl, x, F, W = mapped
    q = torch.tensor(wl.depth[4], device="cuda")
    x.grad_tsdf(q, wl.poses[4], order=2)
    buf = torch.empty(x.n_vox, device="cuda")
    assert np.array_equal(x.read_tsdf(0, buf).cpu().numpy().astype(np.float64), F)
    assert np.array_equal(x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64), W)


@pytest.mark.parametrize("which", ["small", "room256"])
def test_zero_at_the_fusing_pose(which):
    """A volume holding one frame: the same frame at the same pose changes nothing (E = 0 and g = 0
    exactly, the update rounds F_D as the fusion did), and the Hessian is the Gauss-Newton form."""
    if which == "small":
        wl = synth.small_orbit(frames=2)
    else:
        wl = synth.room_walk(seed=7, frames=2, device="cuda", resident=True)
    x = make_handle(wl, max_lanes=0)
    x.set_pose(wl.poses[0])
    d0 = torch.as_tensor(wl.depth[0], device="cuda")
    x.frame(d0, [])
    E, g, H, n = x.grad_tsdf(d0, wl.poses[0], order=2)
    assert n > 1000
    assert E == 0.0 and np.abs(g).max() == 0.0
    ev = np.linalg.eigvalsh(H)
    assert ev.min() >= -1e-5 * ev.max() and ev.max() > 0
    # off the fusing pose the loss grows, and a Newton step brings it back down
    T = se3.compose(se3.se3_exp(START), wl.poses[0])
    E1, g1, H1, _ = x.grad_tsdf(d0, T, order=2)
    assert E1 > 0
    step = -np.linalg.solve(H1, g1)
    E2, _, _, _ = x.grad_tsdf(d0, se3.compose(se3.se3_exp(step), T), order=1)
    assert E2 < 0.1 * E1
    x.close()


def test_rejects(mapped):
    from paper_2405_02187_gb300 import xslam
    wl, x, _, _ = mapped
    q = torch.tensor(wl.depth[4], device="cuda")
    with pytest.raises(xslam.XSlamError):
        x.grad_tsdf(q, wl.poses[4], order=3)
    T = np.array(wl.poses[4], np.float64)
    T[0, 3] = np.nan
    with pytest.raises(xslam.XSlamError):
        x.grad_tsdf(q, T, order=2)


@pytest.mark.parametrize("method", ["gd", "nlcg", "newton"])
def test_relocalise_with_the_tsdf_loss(method):
    """A map holding one frame and that frame as the query, 1 cm and 0.23 degrees off: the three
    optimisers never raise the loss; Newton lands on the frame's pose in a few steps, nonlinear CG close
    to it, gradient descent at least halfway (Sec. 5.2, the optimisers of Sec. 6)."""
    from paper_2405_02187_gb300 import reloc as R
    wl = synth.small_orbit(frames=2)
    x = make_handle(wl, max_lanes=0)
    x.set_pose(wl.poses[0])
    d0 = torch.as_tensor(wl.depth[0], device="cuda")
    x.frame(d0, [])
    T0 = se3.compose(se3.se3_exp(START), wl.poses[0])
    tr = [(T0, x.grad_tsdf(d0, T0, order=1)[0])]
    r = R.relocalise(x, d0, T0, method=method, eta=float("inf"), iters=30, trace=tr, loss="tsdf")
    x.close()
    assert all(b[1] <= a[1] for a, b in zip(tr, tr[1:]))
    d0_m = R.pose_error(T0, wl.poses[0])[0]
    d1, r1 = R.pose_error(r.T, wl.poses[0])
    print(method, d0_m, d1, r1, r.iterations, r.loss)
    bound = {"gd": 0.5 * d0_m, "nlcg": 1e-3, "newton": 1e-4}[method]
    assert d1 < bound
    if method == "newton":
        assert r.newton_steps >= 1 and r1 < 0.01


@pytest.mark.parametrize("off", range(len(OFFSETS)))
def test_plain_fp64_path(mapped, off):
    """The plain FP64 bicomplex path (full products, h = 1e-20) against the oracle, and the FP32
    truncated path against it within the 1e-3 derivative error."""
    wl, x, F, W = mapped
    T = se3.compose(se3.se3_exp(OFFSETS[off]), wl.poses[4])
    q = torch.tensor(wl.depth[4], device="cuda")
    E64, g64, H64, n64 = x.grad_tsdf_plain64(q, T)
    Eo, go, Ho, no = _oracle(wl, F, W, T, wl.depth[4])
    print(off, E64, Eo, n64, no, rel_err(g64, go), rel_err(H64, Ho))
    assert abs(n64 - no) <= 2
    assert abs(E64 - Eo) <= 1e-4 * Eo
    assert rel_err(g64, go) < 1e-4 and rel_err(H64, Ho) < 1e-4
    E, g, H, n = x.grad_tsdf(q, T, order=2)
    assert rel_err(g, g64) < 1e-3 and rel_err(H, H64) < 1e-3


def test_ragged_volume_matches_oracle():
    """A volume whose sides are not multiples of the 8^3 brick and a 44x36 image: partial bricks at
    every face, the last pixel row and column."""
    base = synth.tiny(frames=3, n=28, width=44, height=36)
    dims = (28, 26, 25)
    origin = tuple(-d * base.voxel / 2 for d in dims)
    wl = synth.Workload(base.name + "_ragged", base.intr, dims, base.voxel, base.trunc, origin, base.poses,
                        base.depth, base.scene, base.seed, icp_iters=base.icp_iters)
    x = make_handle(wl, max_lanes=0)
    x.set_pose(wl.poses[0])
    for k in range(2):
        x.frame(torch.tensor(wl.depth[k], device="cuda"), [])
    buf = torch.empty(x.n_vox, device="cuda")
    F = x.read_tsdf(0, buf).cpu().numpy().astype(np.float64)
    W = x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64)
    q = torch.tensor(wl.depth[2], device="cuda")
    T = se3.compose(se3.se3_exp(0.5 * OFFSETS[0]), wl.poses[2])
    E, g, H, n = x.grad_tsdf(q, T, order=2)
    E64, g64, H64, n64 = x.grad_tsdf_plain64(q, T)
    x.close()
    Eo, go, Ho, no = _oracle(wl, F, W, T, wl.depth[2])
    print(E, Eo, n, no, rel_err(g, go), rel_err(H, Ho))
    assert no > 100 and abs(n - no) <= 2 and abs(n64 - no) <= 2
    assert abs(E - Eo) <= 2e-3 * Eo and rel_err(g, go) < 2e-3 and rel_err(H, Ho) < 2e-3
    assert abs(E64 - Eo) <= 1e-4 * Eo and rel_err(g64, go) < 1e-4 and rel_err(H64, Ho) < 1e-4


def test_degenerate_queries(mapped):
    """A query with no valid depth, and a pose looking away from the map: nothing is updated, so the
    loss, gradient and Hessian are exactly zero on both paths; the handle stays usable."""
    wl, x, _, _ = mapped
    empty = torch.zeros_like(torch.tensor(wl.depth[4], device="cuda"))
    E, g, H, n = x.grad_tsdf(empty, wl.poses[4], order=2)
    assert n == 0 and E == 0.0 and not g.any() and not H.any()
    E64, g64, H64, n64 = x.grad_tsdf_plain64(empty, wl.poses[4])
    assert n64 == 0 and E64 == 0.0 and not g64.any() and not H64.any()
    # turned half a revolution about the vertical axis through the camera
    away = se3.compose(wl.poses[4], np.concatenate([se3.se3_exp(np.array([0.0, np.pi, 0.0, 0.0, 0.0, 0.0]))[:, :3],
                                                    np.zeros((3, 1))], 1))
    q = torch.tensor(wl.depth[4], device="cuda")
    E, g, H, n = x.grad_tsdf(q, away, order=2)
    Ea, _, _, na = x.grad_tsdf(q, wl.poses[4], order=2)
    assert na > 1000
    assert n < 0.01 * na
    # the handle is unchanged; blocks take tiles by work stealing, so FP32 sums may differ in rounding order
    E2, g2, H2, n2 = x.grad_tsdf(q, wl.poses[4], order=2)
    assert n2 == na and abs(E2 - Ea) <= 1e-6 * Ea
