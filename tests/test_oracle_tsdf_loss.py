"""Pins of the paper's relocalisation loss (Sec. 5.2), E(T) = sum_p (F_r(p) - F_q(p))^2 with F_q the
reference volume after the surface update by the query frame at T (oracle/reloc.py tsdf_*): zero with
a zero gradient where the query repeats the frame the reference was fused from; there the bicomplex
Hessian equals the Gauss-Newton form 2 sum_p grad e_p grad e_p^T built from independent complex steps of
the surface update; elsewhere the complex-step gradient matches central differences, and the
bicomplex Hessian matches central differences of the complex-step gradient, on stencils whose every
discrete decision is asserted identical."""
import numpy as np
import pytest

from oracle import fusion, measure, reloc, se3
from paper_2405_02187_gb300 import synth

H = 1e-20


@pytest.fixture(scope="module")
def setup():
    wl = synth.tiny(frames=2)
    n = int(np.prod(wl.dims))
    F, W = np.ones(n), np.zeros(n)
    D0 = measure.range_gate(wl.depth[0].astype(np.float64), wl.depth_min, wl.depth_max)
    fusion.integrate(F, W, D0, wl.poses[0], wl.intr, wl.dims, wl.origin, wl.voxel, wl.trunc)
    return wl, F, W, D0


def _args(wl):
    return wl.intr, wl.dims, wl.origin, wl.voxel, wl.trunc


def test_zero_at_the_fusing_pose(setup):
    wl, F, W, D0 = setup
    T = wl.poses[0]
    assert reloc.tsdf_loss(F, W, T, D0, *_args(wl)) == 0.0
    E, g = reloc.tsdf_gradient(F, W, T, D0, *_args(wl))
    assert E == 0.0 and np.abs(g).max() < 1e-9
    # Gauss-Newton form at zero residual, from per-voxel complex steps of the surface update
    e = []
    for j in range(6):
        Fq = np.array(F, np.complex128)
        fusion.integrate(Fq, np.array(W), D0, se3.promote_pose(T, j, H), *_args(wl))
        e.append(np.imag(F - Fq)[W > 0] / H)
    e = np.array(e)
    GN = 2.0 * e @ e.T
    _, gb, Hb = reloc.tsdf_hessian_bicomplex(F, W, T, D0, *_args(wl))
    assert np.abs(gb).max() < 1e-9
    np.testing.assert_allclose(Hb, GN, rtol=1e-8, atol=1e-8 * np.abs(GN).max())
    assert np.linalg.eigvalsh(Hb).min() > 0


def _stable_pose(wl, F, W, D, base, delta):
    """A pose near base whose surface-update decisions are the same at exp(+-delta e_j) pose, all j."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        xi = np.concatenate([rng.normal(0, 0.01, 3), rng.normal(0, 0.005, 3)])
        T = se3.compose(se3.se3_exp(xi), base)
        ref = reloc.tsdf_decisions(F, W, T, D, *_args(wl))
        ok = True
        for j in range(6):
            for s in (1, -1):
                dec = reloc.tsdf_decisions(F, W, se3.perturb_pose(T, j, s * delta), D, *_args(wl))
                ok &= all(np.array_equal(a, b) for a, b in zip(ref, dec))
        if ok:
            return T
    raise AssertionError("no stable pose found")


def test_gradient_matches_central_differences(setup):
    wl, F, W, _ = setup
    D1 = measure.range_gate(wl.depth[1].astype(np.float64), wl.depth_min, wl.depth_max)
    delta = 1e-7
    T = _stable_pose(wl, F, W, D1, wl.poses[1], delta)
    E, g = reloc.tsdf_gradient(F, W, T, D1, *_args(wl))
    assert E > 0
    fd = np.zeros(6)
    for j in range(6):
        Ep = reloc.tsdf_loss(F, W, se3.perturb_pose(T, j, delta), D1, *_args(wl))
        Em = reloc.tsdf_loss(F, W, se3.perturb_pose(T, j, -delta), D1, *_args(wl))
        fd[j] = (Ep - Em) / (2 * delta)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_bicomplex_hessian_matches_differences_of_the_gradient(setup):
    wl, F, W, _ = setup
    D1 = measure.range_gate(wl.depth[1].astype(np.float64), wl.depth_min, wl.depth_max)
    delta = 1e-6
    T = _stable_pose(wl, F, W, D1, wl.poses[1], delta)
    E, g, Hb = reloc.tsdf_hessian_bicomplex(F, W, T, D1, *_args(wl))
    Ec, gc = reloc.tsdf_gradient(F, W, T, D1, *_args(wl))
    assert E == pytest.approx(Ec, rel=1e-12)
    np.testing.assert_allclose(g, gc, rtol=1e-10, atol=1e-12 * np.abs(gc).max())
    Hfd = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = delta
        gp = reloc.tsdf_gradient_at(F, W, T, e, D1, *_args(wl))
        gm = reloc.tsdf_gradient_at(F, W, T, -e, D1, *_args(wl))
        Hfd[:, k] = (gp - gm) / (2 * delta)
    np.testing.assert_allclose(Hb, Hfd, rtol=1e-4, atol=1e-5 * np.abs(Hfd).max())
    np.testing.assert_allclose(Hb, Hb.T, rtol=1e-12, atol=1e-12 * np.abs(Hb).max())


def test_unobserved_voxels_do_not_count(setup):
    """The sum runs over the voxels the reference has observed: whatever an unobserved voxel stores
    leaves E, g and H unchanged, and forgetting observed voxels removes exactly their terms."""
    wl, F, W, _ = setup
    D1 = measure.range_gate(wl.depth[1].astype(np.float64), wl.depth_min, wl.depth_max)
    T = wl.poses[1]
    E, g, Hb = reloc.tsdf_hessian_bicomplex(F, W, T, D1, *_args(wl))
    F2 = F.copy()
    F2[W == 0] = -0.3
    E2, g2, H2 = reloc.tsdf_hessian_bicomplex(F2, W, T, D1, *_args(wl))
    assert E2 == E and np.array_equal(g2, g) and np.array_equal(H2, Hb)
    # forget every other observed voxel: E drops by the forgotten voxels' squared changes
    keep, clamp, xc, yc = reloc.tsdf_decisions(F, W, T, D1, *_args(wl))
    Fq, Wq = F.copy(), W.copy()
    fusion.integrate(Fq, Wq, D1, T, *_args(wl))
    obs = np.nonzero(W > 0)[0]
    W3 = W.copy()
    W3[obs[::2]] = 0.0
    E3 = reloc.tsdf_loss(F, W3, T, D1, *_args(wl))
    d = (F - Fq)[obs[::2]]
    assert E3 == pytest.approx(E - np.sum(d * d), rel=1e-12)
    assert 0 < E3 < E
