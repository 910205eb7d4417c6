"""Pins of the oracle's pipeline stages against closed forms (X-SLAM Sec. 4.1).

Each test builds its inputs analytically (exact plane/sphere renders, analytic TSDF fields) so that
a dropped term, a wrong sign or a transposed operand in the oracle fails a comparison with a value
that does not come from the oracle."""
import math

import numpy as np
import pytest

from oracle import fusion, icp, measure, raycast, se3
from paper_2405_02187_gb300 import synth

INTR = synth.Intrinsics(60.0, 60.0, 31.5, 23.5, 64, 48)


# ---------------------------------------------------------------------------------------------
# surface measurement
# ---------------------------------------------------------------------------------------------
def test_vertex_depth_derivative_is_backprojection():
    """Eq. pvnpd: Im V*(u) / h = K^-1 u_dot exactly when D* = D + h i."""
    rng = np.random.default_rng(0)
    D = rng.uniform(0.5, 3.0, (INTR.height, INTR.width))
    li = measure.level_intrinsics(INTR, 0)
    V = measure.vertex_map(D + 1e-20j, li)
    ref = synth.pixel_rays(INTR)
    assert np.abs(V.imag / 1e-20 - ref).max() < 1e-15
    assert np.abs(V.real - D[..., None] * ref).max() < 1e-15


@pytest.mark.parametrize("level", [0, 1, 2])
def test_normals_of_rendered_plane(level):
    """Eq. normal on an exactly rendered tilted plane gives the plane normal (pointing away from the
    camera) at every valid pixel; pyramid levels see the rays of level-0 pixel 2^l u."""
    n = np.array([0.2, -0.3, -1.0])
    n /= np.linalg.norm(n)
    plane = synth.Plane(tuple(n), -2.0)
    D = synth.render_depth([plane], INTR, np.eye(3, 4))
    li = measure.level_intrinsics(INTR, level)
    Dl = D[::2 ** level, ::2 ** level]
    V = measure.vertex_map(Dl, li)
    # every vertex is on the plane
    assert np.abs(V @ n + 2.0).max() < 1e-12
    N, valid = measure.normal_map(Dl, V)
    assert valid[:-1, :-1].all() and not valid[-1].any() and not valid[:, -1].any()
    assert np.abs(N[valid] - (-n)).max() < 1e-10  # -n points away from the camera at the origin


def test_pyramid_linear_ramp_and_masks():
    """The symmetric 5x5 binomial reproduces a linear ramp at the centre tap; invalid and
    out-of-range taps are excluded from the normalised average; the perturbation is averaged too."""
    H, W = 24, 32
    v, u = np.mgrid[0:H, 0:W].astype(float)
    D = 1.0 + 0.01 * u + 0.02 * v
    D1 = measure.pyramid_down(D, 10.0)
    inner = (slice(1, H // 2 - 1), slice(1, W // 2 - 1))
    assert np.abs(D1[inner] - D[::2, ::2][inner]).max() < 1e-14
    # a step edge wider than the range gate: each side averages only its own side
    S = np.where(u < 15, 1.0, 2.0)
    S1 = measure.pyramid_down(S, 0.09)
    assert set(np.unique(S1)) <= {1.0, 2.0}
    # invalid centre -> invalid; invalid neighbours do not pull the average towards 0
    Z = np.full((H, W), 1.5)
    Z[10, 10] = 0.0
    Z[6, 7] = 0.0
    Z1 = measure.pyramid_down(Z, 0.09)
    assert Z1[5, 5] == 0.0
    assert np.all(Z1[Z1 > 0] == 1.5)
    # D + h i: the imaginary part is averaged with the same normalised weights -> h everywhere valid
    Zc = measure.pyramid_down(np.where(Z > 0, Z + 1e-20j, 0), 0.09)
    assert np.all(np.abs(Zc.imag[Z1 > 0] / 1e-20 - 1.0) < 1e-14)


# ---------------------------------------------------------------------------------------------
# surface update (fusion)
# ---------------------------------------------------------------------------------------------
DIMS = (24, 24, 24)
VOX = 0.05
ORIGIN = (-0.6, -0.6, 0.4)
MU = 0.2


def _camera_z(T):
    idx = np.arange(np.prod(DIMS))
    p = fusion.voxel_centres(idx, DIMS, ORIGIN, VOX)
    return se3.transform(se3.inverse(T), p)


def test_fusion_fronto_parallel_plane_closed_form():
    """A plane at camera depth Z gives F = min(1, (Z - z_p) / mu) where not null, null where
    z_p > Z + mu or outside the image (Sec. 4.1, Psi with the reading sdf = L(x) - z)."""
    Z = 1.1
    T = np.eye(3, 4)
    D = synth.render_depth([synth.Plane((0, 0, 1), Z)], INTR, T)
    F = np.ones(np.prod(DIMS))
    Wt = np.zeros(np.prod(DIMS))
    upd = fusion.integrate(F, Wt, D, T, INTR, DIMS, ORIGIN, VOX, MU)
    pc = _camera_z(T)
    z = pc[:, 2]
    x = INTR.fx * pc[:, 0] / z + INTR.cx
    y = INTR.fy * pc[:, 1] / z + INTR.cy
    inside = (x >= 0) & (x < INTR.width - 1) & (y >= 0) & (y < INTR.height - 1)
    expect_upd = inside & (Z - z >= -MU)
    assert np.array_equal(upd, expect_upd)
    ref = np.minimum(1.0, (Z - z) / MU)
    assert np.abs(F[upd] - ref[upd]).max() < 1e-12
    assert np.all(Wt[upd] == 1) and np.all(Wt[~upd] == 0) and np.all(F[~upd] == 1)


def test_fusion_trunc_derivative_and_running_average():
    """mu* = mu + h i gives Im F / h = -sdf / mu^2 where unclamped and 0 where clamped; three frames
    give the running average (W F + F_D) / (W + 1) = mean of the three F_D."""
    T = np.eye(3, 4)
    pc = _camera_z(T)
    z = pc[:, 2]
    F = np.ones(np.prod(DIMS), complex)
    Wt = np.zeros(np.prod(DIMS))
    Zs = [1.1, 1.12, 1.07]
    masks = []
    for Z in Zs:
        D = synth.render_depth([synth.Plane((0, 0, 1), Z)], INTR, T)
        masks.append(fusion.integrate(F, Wt, D, T, INTR, DIMS, ORIGIN, VOX, MU + 1e-20j))
    m = masks[0] & masks[1] & masks[2]
    sdf = np.stack([Z - z for Z in Zs])
    FD = np.minimum(1.0, sdf / MU)
    dFD = np.where(sdf < MU, -sdf / MU ** 2, 0.0)
    assert np.abs(F.real[m] - FD.mean(0)[m]).max() < 1e-12
    assert np.abs(F.imag[m] / 1e-20 - dFD.mean(0)[m]).max() < 1e-10
    assert np.all(Wt[m] == 3)


def test_fusion_sphere_projective_sdf():
    """A sphere: F * mu equals the exact projective distance (depth of the sphere along the ray of
    the voxel's projection minus the voxel's depth) up to the bilinear interpolation error of L(x)."""
    T = se3.se3_exp(np.array([0.02, -0.03, 0.01, 0.05, 0.0, -0.02]))
    sph = synth.Sphere((0.0, 0.0, 1.2), 0.35)
    D = synth.render_depth([sph], INTR, T)
    F = np.ones(np.prod(DIMS))
    Wt = np.zeros(np.prod(DIMS))
    upd = fusion.integrate(F, Wt, D, T, INTR, DIMS, ORIGIN, VOX, MU)
    pc = _camera_z(T)
    z = pc[:, 2]
    x = INTR.fx * pc[:, 0] / z + INTR.cx
    y = INTR.fy * pc[:, 1] / z + INTR.cy
    # exact depth of the sphere along the continuous ray through (x, y)
    ray = np.stack([(x - INTR.cx) / INTR.fx, (y - INTR.cy) / INTR.fy, np.ones_like(x)], -1) @ T[:, :3].T
    o = T[:, 3]
    c = np.array(sph.center)
    A = (ray * ray).sum(-1)
    B = 2 * ray @ (o - c)
    C = (o - c) @ (o - c) - sph.radius ** 2
    disc = B * B - 4 * A * C
    a = (-B - np.sqrt(np.maximum(disc, 0))) / (2 * A)
    sdf = a - z
    core = upd & (disc > 0.05 * B * B) & (sdf < MU)  # away from the silhouette, unclamped
    assert core.sum() > 200
    assert np.abs(F[core] * MU - sdf[core]).max() < 2e-3


# ---------------------------------------------------------------------------------------------
# ray casting
# ---------------------------------------------------------------------------------------------
def _linear_tsdf(n, d, mu):
    """F(p) = clamp((d - n.p) / mu, -1, 1), observed everywhere: the TSDF of the plane n.p = d with
    free space on the side n.p < d."""
    idx = np.arange(np.prod(DIMS))
    p = fusion.voxel_centres(idx, DIMS, ORIGIN, VOX)
    return np.clip((d - p @ n) / mu, -1.0, 1.0), np.ones(idx.shape[0])


def test_raycast_plane_exact_vertices_normals():
    """Trilinear interpolation reproduces a linear field, so the zero crossing lands exactly on the
    plane and grad F / |grad F| is exactly the plane's normal towards free space."""
    n = np.array([0.1, 0.2, 1.0])
    n /= np.linalg.norm(n)
    d = 1.3
    F, Wt = _linear_tsdf(n, d, MU)
    T = se3.se3_exp(np.array([0.03, -0.02, 0.01, 0.02, -0.01, 0.0]))
    depth, V, N = raycast.raycast(F, Wt, T, INTR, DIMS, ORIGIN, VOX, 0.2, 4.0)
    valid = depth > 0
    assert valid.mean() > 0.5
    assert np.abs(V[valid] @ n - d).max() < 1e-12
    assert np.abs(N[valid] + n).max() < 1e-12
    # depth is the camera-z of the vertex: exact ray/plane intersection
    ref = synth.render_depth([synth.Plane(tuple(n), d)], INTR, T)
    assert np.abs(depth[valid] - ref[valid]).max() < 1e-12


def test_raycast_pose_derivative_equals_ray_plane_derivative():
    """POSE lane through the ray caster: Im V / h equals the derivative of the exact ray/plane
    intersection with respect to a left twist of the pose (closed form, differentiated by hand)."""
    n = np.array([0.1, -0.1, 1.0])
    n /= np.linalg.norm(n)
    d = 1.25
    F, Wt = _linear_tsdf(n, d, MU)
    T0 = se3.se3_exp(np.array([0.01, 0.02, -0.01, 0.0, 0.03, 0.01]))
    rays = synth.pixel_rays(INTR).reshape(-1, 3)
    for j in range(6):
        Tc = se3.promote_pose(T0, j, 1e-20)
        depth, V, _ = raycast.raycast(F.astype(complex), Wt, Tc, INTR, DIMS, ORIGIN, VOX, 0.2, 4.0)
        valid = (depth > 0).reshape(-1)
        # vertex(T) = t + alpha R r with alpha = (d - n.t) / (n.R r);  d/dxi for T -> exp(xi) T:
        # dR = [w] R, dt = [w] t + v
        e = np.zeros(6)
        e[j] = 1.0
        w, vv = e[:3], e[3:]
        R, t = T0[:, :3], T0[:, 3]
        Rr = rays @ R.T
        dRr = np.cross(w, Rr)
        dt = np.cross(w, t) + vv
        nr = Rr @ n
        alpha = (d - n @ t) / nr
        dalpha = (-(n @ dt) * nr - (d - n @ t) * (dRr @ n)) / nr ** 2
        dV = dt + dalpha[:, None] * Rr + alpha[:, None] * dRr
        got = V.reshape(-1, 3).imag / 1e-20
        assert np.abs(got[valid] - dV[valid]).max() < 1e-9


def test_raycast_trunc_derivative_vanishes():
    """Scaling F by 1/mu moves no zero crossing: with mu* = mu + h i the vertex has Im V = 0."""
    n = np.array([0.0, 0.0, 1.0])
    F, Wt = _linear_tsdf(n, 1.2, MU)
    idx = np.arange(np.prod(DIMS))
    p = fusion.voxel_centres(idx, DIMS, ORIGIN, VOX)
    sdf = 1.2 - p @ n
    mu = MU + 1e-20j
    Fc = np.where(np.abs(sdf) < MU, sdf / mu, np.clip(sdf / MU, -1, 1))
    depth, V, N = raycast.raycast(Fc, Wt, np.eye(3, 4), INTR, DIMS, ORIGIN, VOX, 0.2, 4.0)
    valid = depth > 0
    assert valid.mean() > 0.5
    assert np.abs(V.imag[valid]).max() < 1e-32
    assert np.abs(N.imag[valid]).max() < 1e-32


# ---------------------------------------------------------------------------------------------
# ICP
# ---------------------------------------------------------------------------------------------
def _model_at(scene, intr, T):
    """Model maps of an exact render at pose T (world-frame vertices and normals)."""
    D = synth.render_depth(scene, intr, T)
    D = measure.range_gate(D, 0.2, 4.0)
    li = measure.level_intrinsics(intr, 0)
    V = measure.vertex_map(D, li)
    N, valid = measure.normal_map(D, V)
    Vw = se3.transform(T, V)
    Nw = N @ T[:, :3].T
    depth = np.where(valid, D, 0.0)
    return dict(depth=depth, V=np.where(valid[..., None], Vw, 0), N=np.where(valid[..., None], Nw, 0)), D


def _corner_scene():
    return [synth.Room((-1.2, -0.8, -1.0), (1.0, 1.1, 1.3)),
            synth.Box((-0.3, -0.8, 0.5), (0.2, -0.4, 0.9)),
            synth.Sphere((0.4, -0.5, 0.7), 0.25)]


def test_icp_jacobian_is_residual_derivative():
    """J = [(p' x n)^T, n^T] is d r / d x for p' -> exp(x) p' with q, n held fixed (Eq. icp)."""
    scene = _corner_scene()
    T = synth.look_at((0.1, 0.2, -0.5), (0.0, -0.3, 0.8))
    model, D = _model_at(scene, INTR, T)
    Tj = se3.compose(se3.se3_exp(np.array([0.01, -0.005, 0.002, 0.01, 0.0, -0.005])), T)
    r, J, valid = icp.correspondences(D, measure.level_intrinsics(INTR, 0), 0, Tj, T, model)
    assert valid.sum() > 500
    # recompute r along a complex twist with the correspondences frozen
    li = measure.level_intrinsics(INTR, 0)
    V = measure.vertex_map(D, li).reshape(-1, 3)
    pp = se3.transform(Tj, V)[valid]
    q_minus_p = -r[valid]  # only used for the shape check below
    assert q_minus_p.shape[0] == pp.shape[0]
    for j in range(6):
        x = np.zeros(6, complex)
        x[j] = 1e-20j
        ppc = se3.transform(se3.se3_exp(x), pp)
        # r(x) - r(0) = (p'(x) - p') . n  with n fixed
        n = J[valid][:, 3:]
        dr = np.sum((ppc - pp) * n, -1).imag / 1e-20
        assert np.abs(dr - J[valid][:, j]).max() < 1e-12


def test_icp_fixed_point_and_convergence():
    """Noise-free renders: the true pose is an exact zero-residual fixed point of the Gauss-Newton
    iteration, and ICP started 2 cm / 2 degrees away converges back to it."""
    scene = _corner_scene()
    intr = synth.Intrinsics(120.0, 120.0, 79.5, 59.5, 160, 120)
    T = synth.look_at((0.1, 0.2, -0.5), (0.0, -0.3, 0.8))
    model, D = _model_at(scene, intr, T)
    pyr = measure.pyramid(D, 3, 0.09)
    r, J, valid = icp.correspondences(pyr[0], measure.level_intrinsics(intr, 0), 0, T, T, model)
    assert valid.mean() > 0.8
    assert np.abs(r[valid]).max() < 1e-12
    A, b, _ = icp.normal_equations(r, J, valid)
    assert np.abs(icp.solve(A, b)).max() < 1e-12
    off = np.array([math.radians(2) / math.sqrt(3)] * 3 + [0.02 / math.sqrt(3)] * 3) * np.array([1, -1, 1, 1, 1, -1])
    T0 = se3.compose(se3.se3_exp(off), T)
    Tk, ok = icp.track(pyr, intr, T0, T, model, iters=(10, 5, 4))
    assert ok
    assert np.abs(Tk - T).max() < 1e-9
    # the converged pose does not depend on the starting guess: its derivative w.r.t. the start is 0
    T0c = se3.compose(se3.se3_exp(off + 1e-20j * np.eye(6)[2]), T.astype(complex))
    Tkc, ok = icp.track(pyr, intr, T0c, T, model, iters=(10, 5, 4))
    assert ok
    assert np.abs(Tkc.imag / 1e-20).max() < 1e-6


def test_icp_rejects_too_few_correspondences():
    """Fewer than min_corr_frac valid correspondences fails the frame and returns the initial pose."""
    scene = _corner_scene()
    intr = synth.Intrinsics(120.0, 120.0, 79.5, 59.5, 160, 120)
    T = synth.look_at((0.1, 0.2, -0.5), (0.0, -0.3, 0.8))
    model, D = _model_at(scene, intr, T)
    model["depth"][:, 8:] = 0.0  # almost no model left
    pyr = measure.pyramid(D, 3, 0.09)
    Tk, ok = icp.track(pyr, intr, T, T, model, iters=(10, 5, 4))
    assert not ok and np.array_equal(Tk, T)
