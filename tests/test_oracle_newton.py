"""Pins of the oracle's Newton ICP (X-SLAM Sec. 4.1, second-order ICP with the Hessian of Eq.
csfd_hessian): the bicomplex gradient of an iteration's energy against the complex step through the
Gauss-Newton correspondence code, the Hessian against central differences of that gradient (every
decision identical over the stencil), the Gauss-Newton matrix where the residuals vanish, and
convergence of the multi-level Newton tracker to the true pose."""
import numpy as np
import pytest

from oracle import icp, measure, se3
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth


@pytest.fixture(scope="module")
def setup():
    wl = synth.tiny(frames=3)
    cfg = P.Config(icp_iters=tuple(wl.icp_iters), depth_min=wl.depth_min, depth_max=wl.depth_max)
    r = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, None)
    r.frame(wl.depth[0])
    r.frame(wl.depth[1])
    pyr = r.measure(wl.depth[2])
    return wl, r, pyr


def _E(pyr, lintr, level, T, Tprev, model):
    rr, J, valid = icp.correspondences(pyr[level], lintr, level, T, Tprev, model)
    return np.sum(rr[valid] ** 2), valid


def test_newton_energy_derivatives(setup):
    wl, r, pyr = setup
    level = 0
    lintr = measure.level_intrinsics(wl.intr, level)
    Tprev = r.T
    Tj = se3.compose(se3.se3_exp(np.array([0.003, -0.002, 0.002, 0.004, -0.003, 0.002])), Tprev)
    E, g, H, n, A = icp.newton_energy(pyr[level], lintr, level, Tj, Tprev, r.model)
    assert n > 300
    E0, valid0 = _E(pyr, lintr, level, Tj, Tprev, r.model)
    assert abs(E - E0) <= 1e-12 * E0
    h = 1e-20
    gc = np.array([np.imag(_E(pyr, lintr, level, se3.promote_pose(Tj, j, h), Tprev, r.model)[0]) / h for j in range(6)])
    assert np.abs(g - gc).max() <= 1e-10 * np.abs(gc).max()
    # Hessian: central differences (global twist) of the complex-step gradient, decisions identical
    d = 1e-7

    def grad_at(xi):
        out = np.zeros(6)
        for j in range(6):
            x = np.asarray(xi, np.complex128).copy()
            x[j] += 1j * h
            Ec, v = _E(pyr, lintr, level, se3.compose(se3.se3_exp(x), Tj), Tprev, r.model)
            assert np.array_equal(v, valid0)
            out[j] = np.imag(Ec) / h
        return out

    Hfd = np.stack([(grad_at(d * np.eye(6)[k]) - grad_at(-d * np.eye(6)[k])) / (2 * d) for k in range(6)], 1)
    assert np.abs(H - Hfd).max() <= 1e-6 * np.abs(H).max()
    # A is 2 J~ J~^T of the exact first derivatives (the complex step of each residual)
    rr0, _, v0 = icp.correspondences(pyr[level], lintr, level, Tj, Tprev, r.model)
    Jt = np.stack([icp.correspondences(pyr[level], lintr, level, se3.promote_pose(Tj, j, h), Tprev, r.model)[0].imag[v0] / h
                   for j in range(6)], 1)
    assert np.abs(A - 2.0 * Jt.T @ Jt).max() <= 1e-9 * np.abs(A).max()


def test_newton_hessian_is_gauss_newton_at_zero_residual(setup):
    wl, r, pyr = setup
    level = 1
    lintr = measure.level_intrinsics(wl.intr, level)
    T_true = r.T  # frame 1's tracked pose; the noise-free frame 1 seen again has near-zero residuals
    pyr1 = r.measure(wl.depth[1])
    E, g, H, n, _ = icp.newton_energy(pyr1[level], lintr, level, T_true, T_true, r.model)
    rr, J, valid = icp.correspondences(pyr1[level], lintr, level, T_true, T_true, r.model)
    A = 2.0 * J[valid].T @ J[valid]
    assert np.median(np.abs(rr[valid])) < 2e-3
    assert np.linalg.norm(H - A) <= 0.1 * np.linalg.norm(A)


def test_newton_tracker_converges(setup):
    wl, r, pyr = setup
    T, ok = icp.track_newton(pyr, wl.intr, r.T, r.T, r.model, iters=wl.icp_iters)
    assert ok
    Tg, okg = icp.track(pyr, wl.intr, r.T, r.T, r.model, iters=wl.icp_iters)
    assert np.abs(T[:, 3] - wl.poses[2][:, 3]).max() < 2e-3
    assert np.abs(T - Tg).max() < 2e-3


def test_newton_solve_damping():
    H = np.diag([1.0, 2.0, 3.0, -0.5, 1.0, 1.0])
    g = np.ones(6)
    x = icp.newton_solve(H, g)
    mu = 10.0 ** (-3) * np.trace(H) / 6.0  # k = 1 is not enough (-0.5 + 0.0013), the first that is PD
    ks = [k for k in range(1, 7) if np.all(np.linalg.eigvalsh(H + 10.0 ** (k - 4) * np.trace(H) / 6.0 * np.eye(6)) > 0)]
    mu = 10.0 ** (ks[0] - 4) * np.trace(H) / 6.0
    assert np.allclose(x, -np.linalg.solve(H + mu * np.eye(6), g))
    assert icp.newton_solve(np.diag([1.0, 1, 1, 1, 1, -1e9]), g) is None
