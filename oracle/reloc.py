"""Relocalisation loss of a query depth frame against the TSDF map (X-SLAM Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper optimises the query pose T_q with the gradient and Hessian of a loss computed by X-KF. Read
here (as for the second-order workload) as the point-to-plane form: the model maps V_g, N_g are ray
cast from the volume at T_q itself, so the correspondence of pixel u is u, and
  E(T_q) = mean over pixels u of r_u^2,   r_u = (T_q V_q(u) - V_g(u)) . N_g(u),
with V_q = D_q K^-1 u (Eq. vertex) from the range-gated (and, for the 640x480 workload, bilaterally
filtered) query depth; a pixel counts if its query depth and model are valid and |T_q V_q - V_g| is at
most the ICP distance gate. The derivative with respect to a left twist of T_q is Im E(exp(h i e_j) T_q) / h
(Eq. csfd), one complex run per twist component; the volume is taken as real. The second-order
derivatives follow the paper's bicomplex step (Sec. 3): E(exp(h i1 e_j + h i2 e_k) T_q) in bicomplex
arithmetic (oracle/bicomplex.py) with the real pose's discrete decisions (``hessian_bicomplex``);
``hessian`` is an independent check by central differences of the complex-step gradient with respect
to the global twist xi of exp(xi) T_q.
"""
from __future__ import annotations

import numpy as np

from . import measure, raycast, se3


def residuals(F, Wt, T, Dq, intr, dims, origin, voxel, depth_min=0.2, depth_max=4.0, dist_gate=0.1):
    """r_u for every pixel (real or complex with T) and the mask of pixels that count."""
    dg, Vg, Ng = raycast.raycast(F, Wt, T, intr, dims, origin, voxel, depth_min, depth_max)
    V = measure.vertex_map(Dq, measure.level_intrinsics(intr, 0))
    p = se3.transform(np.asarray(T), V.reshape(-1, 3))
    diff = p - Vg.reshape(-1, 3)
    dre = np.real(diff)
    valid = (Dq.reshape(-1) > 0) & (dg.reshape(-1) > 0) & (np.sum(dre * dre, -1) <= dist_gate ** 2)
    return np.sum(diff * Ng.reshape(-1, 3), -1), valid


def loss(F, Wt, T, Dq, intr, dims, origin, voxel, depth_min=0.2, depth_max=4.0, dist_gate=0.1):
    """E(T) for a real or complex pose T (the volume F, Wt is real)."""
    dg, Vg, Ng = raycast.raycast(F, Wt, T, intr, dims, origin, voxel, depth_min, depth_max)
    V = measure.vertex_map(Dq, measure.level_intrinsics(intr, 0))
    p = se3.transform(np.asarray(T), V.reshape(-1, 3))
    diff = p - Vg.reshape(-1, 3)
    dre = np.real(diff)
    valid = (Dq.reshape(-1) > 0) & (dg.reshape(-1) > 0) & (np.sum(dre * dre, -1) <= dist_gate ** 2)
    r = np.sum(diff * Ng.reshape(-1, 3), -1)[valid]
    return np.sum(r * r) / max(int(valid.sum()), 1), int(valid.sum())


def gradient(F, Wt, T, Dq, intr, dims, origin, voxel, h=1e-20, **kw):
    """(E, dE/dxi) with xi a left twist of T (phi then rho), by six complex runs."""
    E, n = loss(F, Wt, np.asarray(T, np.float64), Dq, intr, dims, origin, voxel, **kw)
    g = np.zeros(6)
    for j in range(6):
        Ec, _ = loss(F, Wt, se3.promote_pose(T, j, h), Dq, intr, dims, origin, voxel, **kw)
        g[j] = np.imag(Ec) / h
    return E, g, n


def gradient_at(F, Wt, T0, xi, Dq, intr, dims, origin, voxel, h=1e-20, **kw):
    """dE(exp(xi + s e_j) T0) / ds at s = 0, j = 0..5: the gradient with respect to the global twist xi
    of exp(xi) T0 (a complex step on each component of xi; for xi = 0 this is ``gradient``)."""
    g = np.zeros(6)
    for j in range(6):
        x = np.asarray(xi, np.complex128).copy()
        x[j] += 1j * h
        Ec, _ = loss(F, Wt, se3.compose(se3.se3_exp(x), T0), Dq, intr, dims, origin, voxel, **kw)
        g[j] = np.imag(Ec) / h
    return g


def hessian(F, Wt, T0, Dq, intr, dims, origin, voxel, delta=1e-5, h=1e-20, **kw):
    """H_jk = d^2 E(exp(xi) T0) / dxi_j dxi_k at xi = 0 (the second-order derivative that X-SLAM Sec. 3
    obtains from bicomplex steps, here as a reference): central differences with step delta along xi_k
    of the complex-step gradient. Truncation O(delta^2), rounding O(eps / delta); valid when no discrete
    decision of the loss changes within +-delta."""
    H = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = delta
        gp = gradient_at(F, Wt, T0, e, Dq, intr, dims, origin, voxel, h=h, **kw)
        gm = gradient_at(F, Wt, T0, -e, Dq, intr, dims, origin, voxel, h=h, **kw)
        H[:, k] = (gp - gm) / (2 * delta)
    return H


def decisions(F, Wt, T, Dq, intr, dims, origin, voxel, depth_min=0.2, depth_max=4.0, dist_gate=0.1):
    """The discrete decisions of loss at pose T (ray-cast hit samples, pixel validity and cells, the
    accepted pixels), to check that a finite-difference stencil does not cross one."""
    log = []
    dg, Vg, _ = raycast.raycast(F, Wt, np.real(T), intr, dims, origin, voxel, depth_min, depth_max, log=log)
    V = measure.vertex_map(Dq, measure.level_intrinsics(intr, 0))
    p = se3.transform(np.real(T), V.reshape(-1, 3))
    diff = p - Vg.reshape(-1, 3)
    ok = (Dq.reshape(-1) > 0) & (dg.reshape(-1) > 0) & (np.sum(diff * diff, -1) <= dist_gate ** 2)
    return log + [ok]


def _generator(j):
    """4x4 generator of the left twist component j (phi then rho)."""
    G = np.zeros((4, 4))
    if j < 3:
        w = np.zeros(3)
        w[j] = 1.0
        G[:3, :3] = se3.hat(w)
    else:
        G[j - 3, 3] = 1.0
    return G


def bicomplex_pose(T0, j, k, h):
    """exp(h i1 e_j + h i2 e_k) T0 to O(h^3) (Sec. 3 second-order step on a left twist): with
    X = h i1 G_j + h i2 G_k, exp(X) = I + X + X^2 / 2 + O(h^3) and
    X^2 = -h^2 (G_j^2 + G_k^2) + h^2 i1 i2 (G_j G_k + G_k G_j)."""
    from .bicomplex import Bicomplex
    Gj, Gk = _generator(j), _generator(k)
    T4 = np.eye(4)
    T4[:3] = np.asarray(T0, np.float64)
    M1 = np.eye(4) - 0.5 * h * h * (Gj @ Gj + Gk @ Gk) + 1j * h * Gj
    M2 = h * Gk + 0.5j * h * h * (Gj @ Gk + Gk @ Gj)
    return Bicomplex((M1 @ T4)[:3], (M2 @ T4)[:3])


def _tri_bc(F, dims, g):
    """Trilinear F (real volume) at bicomplex voxel coordinates g (list of 3 arrays); cells from the
    real parts, as in the ray cast."""
    from .bicomplex import Bicomplex
    nx, ny, _ = dims
    i0 = [np.floor(c.real).astype(np.int64) for c in g]
    f = [c - i for c, i in zip(g, i0)]
    val = Bicomplex(np.zeros(g[0].shape, np.complex128))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                lin = (i0[0] + dx) + nx * ((i0[1] + dy) + ny * (i0[2] + dz))
                w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                val = val + w * F[lin]
    return val


def hessian_bicomplex(F, Wt, T0, Dq, intr, dims, origin, voxel, depth_min=0.2, depth_max=4.0, dist_gate=0.1,
                      ray_step_vox=1.0, h=1e-20, full=False):
    """(E, g, H) at T0: the loss, its gradient and its Hessian with respect to a left twist, H_jk the
    i1 i2 part / h^2 of E(exp(h i1 e_j + h i2 e_k) T0) (bicomplex step, Sec. 3), for j <= k (H is
    filled symmetrically; full=True evaluates every (j, k) separately). The discrete decisions (the ray-cast hit sample, pixel validity, the cells,
    the accepted pixels) are those of the real pose; the ray-cast refinement and the residual are
    evaluated in bicomplex arithmetic, step by step as in raycast.raycast and loss."""
    from . import bicomplex as bc
    T0 = np.asarray(T0, np.float64)
    log = []
    dg, Vg, _ = raycast.raycast(F, Wt, T0, intr, dims, origin, voxel, depth_min, depth_max, ray_step_vox, log=log)
    m_hit = log[0]
    V = measure.vertex_map(Dq, measure.level_intrinsics(intr, 0)).reshape(-1, 3)
    diff0 = se3.transform(T0, V) - Vg.reshape(-1, 3)
    ok = (Dq.reshape(-1) > 0) & (dg.reshape(-1) > 0) & (np.sum(diff0 * diff0, -1) <= dist_gate ** 2)
    idx = np.nonzero(ok)[0]
    n = idx.size
    H, g = np.zeros((6, 6)), np.zeros(6)
    if n == 0:
        return 0.0, g, H
    uu, vv = idx % intr.width, idx // intr.width
    ray = [(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones(n)]
    step = ray_step_vox * voxel
    org = np.asarray(origin, np.float64)
    a_m = m_hit[idx] * step
    Vq = V[idx]
    E = 0.0
    for j in range(6):
        for k in range(0 if full else j, 6):
            T = bicomplex_pose(T0, j, k, h)
            dirs = [T[r, 0] * ray[0] + T[r, 1] * ray[1] + T[r, 2] * ray[2] for r in range(3)]
            t = [T[r, 3] for r in range(3)]
            samples = []
            for a in (a_m, a_m + step):
                gco = [(t[r] + a * dirs[r] - org[r]) / voxel - 0.5 for r in range(3)]
                samples.append(_tri_bc(F, dims, gco))
            Fm, Fn = samples
            alpha0 = a_m - step * Fm / (Fn - Fm)
            v0 = [alpha0 * dirs[r] + t[r] for r in range(3)]
            grad = []
            for ax in range(3):
                vals = []
                for sgn in (1.0, -1.0):
                    gco = [(v0[r] + (sgn * voxel if r == ax else 0.0) - org[r]) / voxel - 0.5 for r in range(3)]
                    vals.append(_tri_bc(F, dims, gco))
                grad.append((vals[0] - vals[1]) / (2 * voxel))
            g2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]
            nrm = bc.sqrt(g2)
            N = [gr / nrm for gr in grad]
            p = [T[r, 0] * Vq[:, 0] + T[r, 1] * Vq[:, 1] + T[r, 2] * Vq[:, 2] + T[r, 3] for r in range(3)]
            res = (p[0] - v0[0]) * N[0] + (p[1] - v0[1]) * N[1] + (p[2] - v0[2]) * N[2]
            r2 = res * res
            Es = bc.Bicomplex(np.sum(r2.z1) / n, np.sum(r2.z2) / n)
            H[j, k] = float(Es.i1i2()) / (h * h)
            if not full:
                H[k, j] = H[j, k]
            if j == k:
                g[j] = float(Es.i1()) / h
                E = float(Es.real)
    return E, g, H


# ---------------------------------------------------------------------------------------------------
# The paper's relocalisation loss (Sec. 5.2): the query frame fused into the reference volume at the
# query pose, E(T) = sum_p (F_r(p) - F_q(p))^2 with (F_q, W_q) = surface_update(M_r, T, D_q). Only the
# voxels the query updates differ. The sum runs over the voxels the reference has observed (W_r > 0):
# an unobserved voxel has no TSDF value to compare (its stored F = 1 is a convention of fusion.py), and
# counting it would reward poses that see less of the map. The derivatives with respect to a left
# twist of T follow the update's discrete decisions (which voxels are updated, which are clamped at
# F_D = 1, the pixel cells) at the real pose.
# ---------------------------------------------------------------------------------------------------
def tsdf_loss(F, Wt, T, Dq, intr, dims, origin, voxel, mu, disc_gate=0.1):
    """E(T) for a real or complex pose T (the reference volume F, Wt is real)."""
    from . import fusion
    T = np.asarray(T)
    Fq = np.array(F, np.complex128 if np.iscomplexobj(T) else np.float64)
    Wq = np.array(Wt, np.float64)
    fusion.integrate(Fq, Wq, Dq, T, intr, dims, origin, voxel, mu, disc_gate)
    d = (np.asarray(F, np.float64) - Fq)[np.asarray(Wt) > 0]
    return np.sum(d * d)


def tsdf_gradient(F, Wt, T, Dq, intr, dims, origin, voxel, mu, h=1e-20, **kw):
    """(E, dE/dxi), xi a left twist of T, by six complex runs."""
    E = tsdf_loss(F, Wt, np.asarray(T, np.float64), Dq, intr, dims, origin, voxel, mu, **kw)
    g = np.zeros(6)
    for j in range(6):
        g[j] = np.imag(tsdf_loss(F, Wt, se3.promote_pose(T, j, h), Dq, intr, dims, origin, voxel, mu, **kw)) / h
    return float(E), g


def tsdf_gradient_at(F, Wt, T0, xi, Dq, intr, dims, origin, voxel, mu, h=1e-20, **kw):
    """The gradient with respect to the global twist xi of exp(xi) T0 (complex steps on xi)."""
    g = np.zeros(6)
    for j in range(6):
        x = np.asarray(xi, np.complex128).copy()
        x[j] += 1j * h
        g[j] = np.imag(tsdf_loss(F, Wt, se3.compose(se3.se3_exp(x), T0), Dq, intr, dims, origin, voxel, mu,
                                 **kw)) / h
    return g


def tsdf_decisions(F, Wt, T, Dq, intr, dims, origin, voxel, mu, disc_gate=0.1):
    """The surface update's discrete decisions at the real pose T (update mask, clamp mask, cells)."""
    from . import fusion
    log = []
    fusion.integrate(np.array(F, np.float64), np.array(Wt, np.float64), Dq, np.real(T), intr, dims, origin, voxel,
                     mu, disc_gate, log=log)
    return log


def tsdf_hessian_bicomplex(F, Wt, T0, Dq, intr, dims, origin, voxel, mu, disc_gate=0.1, h=1e-20):
    """(E, g, H) at T0 by the bicomplex step (Sec. 3): E(exp(h i1 e_j + h i2 e_k) T0) with the surface
    update's decisions at the real pose, evaluated step by step as in fusion.integrate
    (p_c = R^T (p - t), x = pi(K p_c), L(x) bilinear, sdf = L - |t - p| / |K^-1 x_dot|, F_D = sdf / mu
    unless clamped, F_q = (W F_r + F_D) / (W + 1)); H_jk = the i1 i2 part / h^2, g_j the i1 part / h."""
    from . import bicomplex as bc
    from . import fusion
    T0 = np.asarray(T0, np.float64)
    keep, clamp, xc, yc = tsdf_decisions(F, Wt, T0, Dq, intr, dims, origin, voxel, mu, disc_gate)
    E = float(tsdf_loss(F, Wt, T0, Dq, intr, dims, origin, voxel, mu, disc_gate))
    g, H = np.zeros(6), np.zeros((6, 6))
    # clamped voxels take F_D = 1 at every pose near T0: no derivative; unobserved ones are not summed
    sel = keep & ~clamp & (np.asarray(Wt) > 0)
    idx = np.nonzero(sel)[0]
    if idx.size == 0:
        return E, g, H
    p = fusion.voxel_centres(idx, dims, origin, voxel)
    i0, j0 = xc[sel].astype(np.int64), yc[sel].astype(np.int64)
    D = np.asarray(Dq, np.float64)
    d00, d10, d01, d11 = D[j0, i0], D[j0, i0 + 1], D[j0 + 1, i0], D[j0 + 1, i0 + 1]
    Fr = np.asarray(F, np.float64)[idx]
    w = np.asarray(Wt, np.float64)[idx]
    for j in range(6):
        for k in range(j, 6):
            T = bicomplex_pose(T0, j, k, h)
            dv = [p[:, r] - T[r, 3] for r in range(3)]
            pc = [T[0, c] * dv[0] + T[1, c] * dv[1] + T[2, c] * dv[2] for c in range(3)]
            x = intr.fx * pc[0] / pc[2] + intr.cx
            y = intr.fy * pc[1] / pc[2] + intr.cy
            a, b = x - i0, y - j0
            L = (1 - a) * (1 - b) * d00 + a * (1 - b) * d10 + (1 - a) * b * d01 + a * b * d11
            lam = bc.sqrt(((x - intr.cx) / intr.fx) * ((x - intr.cx) / intr.fx)
                          + ((y - intr.cy) / intr.fy) * ((y - intr.cy) / intr.fy) + 1.0)
            dist = bc.sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2])
            FD = (L - dist / lam) / mu
            e = Fr - (w * Fr + FD) / (w + 1.0)
            s = e * e
            Es = bc.Bicomplex(np.sum(s.z1), np.sum(s.z2))
            H[j, k] = H[k, j] = float(Es.i1i2()) / (h * h)
            if j == k:
                g[j] = float(Es.i1()) / h
    return E, g, H
