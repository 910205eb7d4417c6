"""Pins of the oracle's relocalisation loss derivatives (X-SLAM Sec. 5.2 point-to-plane reading;
second order by the bicomplex step of Sec. 3): bicomplex arithmetic against closed forms; the
bicomplex Hessian against central differences of the complex-step gradient (every discrete decision
identical over the stencil), its symmetry, its gradient part against the complex step, and the
Gauss-Newton form where the residuals vanish."""
import numpy as np
import pytest

from oracle import measure, reloc, se3
from oracle import pipeline as P
from oracle.bicomplex import Bicomplex, sqrt
from paper_2405_02187_gb300 import synth

H_STEP = 1e-20


@pytest.fixture(scope="module")
def mapped():
    wl = synth.tiny(frames=3)
    cfg = P.Config(icp_iters=tuple(wl.icp_iters), depth_min=wl.depth_min, depth_max=wl.depth_max)
    r = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, None)
    for k in range(3):
        r.frame(wl.depth[k])
    D = measure.range_gate(wl.depth[2].astype(np.float64), wl.depth_min, wl.depth_max)
    return wl, r, D


def _args(wl):
    return (wl.intr, wl.dims, wl.origin, wl.voxel)


T_OFF = np.array([0.004, -0.003, 0.002, 0.003, 0.002, -0.002])


def test_bicomplex_arithmetic_closed_forms():
    x = Bicomplex(0.7 + 1j * H_STEP, 0.0)
    y = Bicomplex(1.3, H_STEP + 0j)
    f = x * x * y * y * y / (1 + x)  # d2/dxdy = (x^2/(1+x))' * 3 y^2
    ref = (2 * 0.7 * 1.7 - 0.49) / 1.7 ** 2 * 3 * 1.3 ** 2
    assert abs(f.i1i2() / H_STEP ** 2 - ref) < 1e-13 * abs(ref)
    assert abs(f.i1() / H_STEP - (2 * 0.7 * 1.7 - 0.49) / 1.7 ** 2 * 1.3 ** 3) < 1e-13
    g = sqrt(x * y + 2.0)
    s = np.sqrt(0.7 * 1.3 + 2)
    assert abs(g.i1i2() / H_STEP ** 2 - (1 / (2 * s) - 0.7 * 1.3 / (4 * s ** 3))) < 1e-14
    assert abs(g.real - s) < 1e-15


def test_bicomplex_pose_is_the_second_order_exponential():
    T0 = se3.se3_exp(np.array([0.1, -0.2, 0.3, 0.5, -0.1, 0.2]))
    for j, k in ((0, 0), (1, 4), (5, 2)):
        T = reloc.bicomplex_pose(T0, j, k, H_STEP)
        # i1 part: G_j T0; i2 part: G_k T0 (the complex steps of se3.promote_pose)
        assert np.allclose(T.i1() / H_STEP, se3.promote_pose(T0, j, H_STEP).imag / H_STEP, atol=1e-12)
        assert np.allclose(T.i2() / H_STEP, se3.promote_pose(T0, k, H_STEP).imag / H_STEP, atol=1e-12)
        # i1 i2 part: (G_j G_k + G_k G_j) T0 / 2, from the exponential series with two steps
        d = 1e-5
        fd = (se3.perturb_pose(se3.perturb_pose(T0, k, d), j, d) - se3.perturb_pose(se3.perturb_pose(T0, k, -d), j, d)
              - se3.perturb_pose(se3.perturb_pose(T0, k, d), j, -d) + se3.perturb_pose(se3.perturb_pose(T0, k, -d), j, -d))
        # the mixed second difference of exp(a e_j) exp(b e_k) T0 is G_j G_k T0; symmetrised with the other order
        fd2 = (se3.perturb_pose(se3.perturb_pose(T0, j, d), k, d) - se3.perturb_pose(se3.perturb_pose(T0, j, d), k, -d)
               - se3.perturb_pose(se3.perturb_pose(T0, j, -d), k, d) + se3.perturb_pose(se3.perturb_pose(T0, j, -d), k, -d))
        assert np.allclose(T.i1i2() / H_STEP ** 2, (fd + fd2) / (8 * d * d), atol=1e-6)


def _stable(r, wl, D, T0, d):
    """Whether every discrete decision of the loss is the same at exp(+-d e_k) T0, k = 0..5."""
    ref = reloc.decisions(r.F, r.W, T0, D, *_args(wl))
    for k in range(6):
        for s in (-1, 1):
            dk = reloc.decisions(r.F, r.W, se3.compose(se3.se3_exp(s * d * np.eye(6)[k]), T0), D, *_args(wl))
            if not all(np.array_equal(a, b) for a, b in zip(ref, dk)):
                return False
    return True


def test_bicomplex_hessian_matches_gradient_differences(mapped):
    wl, r, D = mapped
    d = 1e-7
    # a pose whose stencil crosses no cell face of any sample (one in a few poses has a sample within
    # 1e-7 of a face, where the loss is only continuous)
    for scale in (1.0, 0.9, 1.1, 0.8, 1.2, 0.7):
        T0 = se3.compose(se3.se3_exp(scale * T_OFF), wl.poses[2])
        if _stable(r, wl, D, T0, d):
            break
    else:
        pytest.fail("no pose with a stable stencil")
    E, g, H = reloc.hessian_bicomplex(r.F, r.W, T0, D, *_args(wl))
    Hfd = reloc.hessian(r.F, r.W, T0, D, *_args(wl), delta=d)
    assert np.abs(H - Hfd).max() <= 1e-7 * np.abs(H).max()
    E1, g1, n = reloc.gradient(r.F, r.W, T0, D, *_args(wl))
    assert n > 200 and abs(E - E1) <= 1e-13 * E1
    assert np.abs(g - g1).max() <= 1e-12 * np.abs(g1).max()
    assert np.linalg.eigvalsh(H).min() > 0  # near the optimum


def test_bicomplex_hessian_symmetry(mapped):
    wl, r, D = mapped
    T0 = se3.compose(se3.se3_exp(-0.7 * T_OFF), wl.poses[2])
    _, _, H = reloc.hessian_bicomplex(r.F, r.W, T0, D, *_args(wl), full=True)
    assert np.abs(H - H.T).max() <= 1e-10 * np.abs(H).max()


def test_hessian_is_gauss_newton_where_residuals_vanish(mapped):
    """E = mean r^2 has H = 2/n sum (dr dr^T + r d2r): at the pose the map was built from, on the
    noise-free scene, the residuals are at the TSDF's discretisation level and H is the Gauss-Newton
    term up to that."""
    wl, r, D = mapped
    T0 = wl.poses[2]
    _, _, H = reloc.hessian_bicomplex(r.F, r.W, T0, D, *_args(wl))
    res, valid = reloc.residuals(r.F, r.W, T0, D, *_args(wl))
    assert np.median(np.abs(res[valid])) < 1e-3  # a few silhouette pixels reach a centimetre
    J = np.zeros((int(valid.sum()), 6))
    for j in range(6):
        rc, vc = reloc.residuals(r.F, r.W, se3.promote_pose(T0, j, H_STEP), D, *_args(wl))
        assert np.array_equal(vc, valid)
        J[:, j] = rc.imag[valid] / H_STEP
    Hgn = 2.0 * J.T @ J / valid.sum()
    assert np.linalg.norm(H - Hgn) <= 0.03 * np.linalg.norm(Hgn)
    # and a wrong factor or a dropped first-order term would not pass
    assert np.linalg.norm(H - 0.5 * Hgn) > 0.3 * np.linalg.norm(Hgn)
