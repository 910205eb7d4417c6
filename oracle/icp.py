"""Differentiable projective point-to-plane ICP (X-SLAM Sec. 4.1, "Differentiable ICP" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Energy (Eq. icp): E = sum_u ((T_j V_k(u) - V_g(u_hat))^T N_g(u_hat))^2 with
u_hat = pi(K T_{k-1}^-1 T_j V_k(u)); V_g, N_g are the model maps ray-cast at the previous pose T_{k-1},
sampled at the real-valued u_hat by bilinear interpolation (Sec. 4.1, "we generalize the domain of
integer-value pixel index to R^2 by bilinear interpolation"). Linearising the pose update (Eq. "icp
approx") turns each iteration into the linear least-squares problem A x = b, solved through its
normal equations; complex inputs give a complex A and b and the complex solve carries the derivative.

Readings of the paper used here:
  * the norm in Eq. icp is the squared residual (Gauss-Newton / normal equations);
  * u_hat's lost pi(.) is restored: u_hat = pi(K_l T_{k-1}^-1 T_j V_k(u));
  * the update is a left-multiplied twist x = (omega, v): T_{j+1} = exp(x) T_j, with residual
    r = (p' - q).n and Jacobian J = [(p' x n)^T, n^T] at p' = T_j V_k(u);
  * pyramid level l reads the level-0 model maps at pixel 2^l u (K_l = K / 2^l);
  * a correspondence needs: p' in front of the previous camera, the bilinear cell inside the level
    image (0 <= cell <= size - 2), its 4 model taps valid with |d10-d00|+|d01-d00|+|d11-d00| < disc_gate on the model
    depth, |p' - q| <= dist_gate, and |(R_j N_k(u)) . n| >= cos(normal_gate) |n| (orientation-free,
    because the measured and the ray-cast normals point opposite ways); all decided on real parts;
  * the bilinear normal is not re-normalised;
  * the bilinear cell of u_hat is chosen as floor(u_hat + CELL_BIAS) with CELL_BIAS = 2^-6 pixel
    (the weights a = u_hat - cell then lie in [-2^-6, 1 - 2^-6)): at the first iteration
    T_j = T_{k-1}, so u_hat equals the integer pixel u up to rounding, and an unbiased floor would
    pick the cell on either side of u depending on the last bit; the bias removes that tie;
  * iterations run coarse to fine, a fixed number per level (no early exit unless a stop tolerance is
    given); an iteration with fewer than min_corr_frac of the level's pixels as correspondences, or
    whose real A is not positive definite, fails the frame: the pose falls back to T_{k-1}.
"""
from __future__ import annotations

import math

import numpy as np

from . import measure, se3

CELL_BIAS = 2.0 ** -6


def correspondences(D, lintr, level, Tj, Tprev, model, dist_gate=0.1, normal_gate_deg=20.0,
                    disc_gate=0.1, log=None, pix=None, vn=None):
    """Per-pixel residual r, Jacobian J (N, 6) and validity mask at one pyramid level.
    ``log``, if a list, receives the discrete decisions (validity, bilinear cells); ``pix`` restricts
    the result to those linear pixel indices (each pixel is independent); ``vn`` = (V, N, valid) of
    D's vertex and normal maps if already computed."""
    fx, fy, cx, cy, W, H = lintr
    if vn is None:
        V = measure.vertex_map(D, lintr)
        Nm, vvalid = measure.normal_map(D, V)
    else:
        V, Nm, vvalid = vn
    V = V.reshape(-1, 3)
    Nm = Nm.reshape(-1, 3)
    valid = vvalid.reshape(-1)
    if pix is not None:
        V, Nm, valid = V[pix], Nm[pix], valid[pix]
    Tj = np.asarray(Tj)
    pp = se3.transform(Tj, V)                          # p' = T_j V_k(u)
    pc = se3.transform(se3.inverse(Tprev), pp)         # previous camera frame
    z = pc[:, 2]
    valid &= np.real(z) > 0
    zs = np.where(valid, z, 1.0)
    ux = fx * pc[:, 0] / zs + cx
    uy = fy * pc[:, 1] / zs + cy
    ci = np.floor(np.real(ux) + CELL_BIAS)
    cj = np.floor(np.real(uy) + CELL_BIAS)
    valid &= (ci >= 0) & (ci <= W - 2) & (cj >= 0) & (cj <= H - 2)
    i0 = np.where(valid, ci, 0).astype(np.int64)
    j0 = np.where(valid, cj, 0).astype(np.int64)
    a = ux - i0
    b = uy - j0
    s = 2 ** level
    dg = model["depth"]
    taps = [(j0 * s, i0 * s), (j0 * s, (i0 + 1) * s), ((j0 + 1) * s, i0 * s), ((j0 + 1) * s, (i0 + 1) * s)]
    d = [dg[r, c] for r, c in taps]
    valid &= (d[0] > 0) & (d[1] > 0) & (d[2] > 0) & (d[3] > 0)
    valid &= (np.abs(d[1] - d[0]) + np.abs(d[2] - d[0]) + np.abs(d[3] - d[0])) < disc_gate
    w = [(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b]
    q = sum(w[i][:, None] * model["V"][taps[i]] for i in range(4))
    n = sum(w[i][:, None] * model["N"][taps[i]] for i in range(4))
    diff = pp - q
    dre = np.real(diff)
    valid &= np.sum(dre * dre, -1) <= dist_gate ** 2
    nw = np.real(Nm) @ np.real(Tj[:, :3]).T
    nre = np.real(n)
    cosang = np.abs(np.sum(nw * nre, -1))
    valid &= cosang >= math.cos(math.radians(normal_gate_deg)) * np.sqrt(np.sum(nre * nre, -1))
    r = np.sum(diff * n, -1)
    J = np.concatenate([np.cross(pp, n), n], -1)
    if log is not None:
        log += [valid, np.where(valid, i0, -1), np.where(valid, j0, -1)]
    return r, J, valid


def normal_equations(r, J, valid):
    """A = sum J J^T, b = -sum J r over valid pixels (Eq. "icp approx" posed as A x = b)."""
    Jv = J[valid]
    rv = r[valid]
    A = Jv.T @ Jv
    b = -(Jv.T @ rv)
    return A, b, int(valid.sum())


def solve(A, b):
    """x = A^-1 b (complex LU; the real part decides positive definiteness)."""
    try:
        np.linalg.cholesky(np.real(A))
    except np.linalg.LinAlgError:
        return None
    return np.linalg.solve(A, b)


def track(pyr, intr, T_init, T_prev, model, iters=(10, 5, 4), min_corr_frac=0.1, log=None, stop_tol=0.0,
          levels=None, stats=None, **gates):
    """Multi-level ICP from coarse to fine; returns (T_k, ok). On a failure the pose falls back to
    T_prev, the pose the model was ray cast at.

    stop_tol > 0: a level ends early after an iteration whose real step |x| is below stop_tol (the
    step itself is applied); 0 runs the fixed counts. levels: (first, last) pyramid levels to run,
    first >= last (default: all, coarsest first). stats: a dict whose "iterations" entry counts the
    iterations run."""
    T = np.asarray(T_init)
    first, last = (len(iters) - 1, 0) if levels is None else levels
    for level in range(first, last - 1, -1):
        lintr = measure.level_intrinsics(intr, level)
        npx = lintr[4] * lintr[5]
        for _ in range(iters[level]):
            if stats is not None:
                stats["iterations"] = stats.get("iterations", 0) + 1
            r, J, valid = correspondences(pyr[level], lintr, level, T, T_prev, model, log=log, **gates)
            A, b, nv = normal_equations(r, J, valid)
            if nv < min_corr_frac * npx:
                return np.asarray(T_prev), False
            x = solve(A, b)
            if x is None:
                return np.asarray(T_prev), False
            T = se3.compose(se3.se3_exp(x), T)
            if stop_tol > 0 and np.linalg.norm(np.real(x)) < stop_tol:
                break
    return T, True


# ---------------------------------------------------------------------------------------------------
# Newton ICP (Sec. 4.1: "a second-order ICP procedure using Newton's method at each ICP step", the
# Hessian from Eq. csfd_hessian). Readings: the energy of an iteration is E(xi) = sum_u r_u(exp(xi) T_j)^2
# with the correspondences' bilinear cells, validity and gates fixed at the real T_j (as in the
# Gauss-Newton iteration); r, q and n follow xi through p', u_hat and the bilinear weights exactly (no
# linearisation). When the mean squared residual is at most eta and H is positive definite, the step is
# the Newton step xi = -H^-1 g; otherwise it is the point-to-plane Gauss-Newton step of the same iteration
# (A x = b with the correspondences held fixed, ``normal_equations``). This is the switch the paper
# applies to relocalisation (Sec. 5.2: a first-order direction while the loss exceeds eta, Newton's
# below it). eta = inf gives Newton steps only, a singular H damped as H + mu I with
# mu = 10^(k-4) trace(H) / 6 for the first k = 1..6 that makes it positive definite (none: the frame
# fails).
# ---------------------------------------------------------------------------------------------------
def newton_energy(D, lintr, level, Tj, Tprev, model, h=1e-20, **gates):
    """(E, g, H, n_valid, A) of the iteration energy at Tj by the bicomplex step (oracle/bicomplex.py);
    A = 2 sum dr dr^T, the Gauss-Newton part of H, from the same pairs' first-order parts."""
    from . import reloc
    from .bicomplex import Bicomplex
    fx, fy, cx, cy, W, H_ = lintr
    log = []
    correspondences(D, lintr, level, Tj, Tprev, model, log=log, **gates)
    valid, ci, cj = log[0], log[1], log[2]
    idx = np.nonzero(valid)[0]
    n = idx.size
    H = np.zeros((6, 6))
    A = np.zeros((6, 6))
    g = np.zeros(6)
    if n == 0:
        return 0.0, g, H, 0, A
    V = measure.vertex_map(D, lintr).reshape(-1, 3)[idx]
    i0, j0 = ci[idx], cj[idx]
    s = 2 ** level
    taps = [(j0 * s, i0 * s), (j0 * s, (i0 + 1) * s), ((j0 + 1) * s, i0 * s), ((j0 + 1) * s, (i0 + 1) * s)]
    mV = [model["V"][t] for t in taps]
    mN = [model["N"][t] for t in taps]
    Pinv = se3.inverse(np.asarray(Tprev, np.float64))
    E = 0.0
    for j in range(6):
        for k in range(j, 6):
            T = reloc.bicomplex_pose(Tj, j, k, h)
            pp = [T[r, 0] * V[:, 0] + T[r, 1] * V[:, 1] + T[r, 2] * V[:, 2] + T[r, 3] for r in range(3)]
            pc = [pp[0] * Pinv[r, 0] + pp[1] * Pinv[r, 1] + pp[2] * Pinv[r, 2] + Pinv[r, 3] for r in range(3)]
            ux = fx * pc[0] / pc[2] + cx
            uy = fy * pc[1] / pc[2] + cy
            a = ux - i0
            b = uy - j0
            w = [(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b]
            q = [w[0] * mV[0][:, r] + w[1] * mV[1][:, r] + w[2] * mV[2][:, r] + w[3] * mV[3][:, r] for r in range(3)]
            nn = [w[0] * mN[0][:, r] + w[1] * mN[1][:, r] + w[2] * mN[2][:, r] + w[3] * mN[3][:, r] for r in range(3)]
            res = (pp[0] - q[0]) * nn[0] + (pp[1] - q[1]) * nn[1] + (pp[2] - q[2]) * nn[2]
            r2 = res * res
            Es = Bicomplex(np.sum(r2.z1), np.sum(r2.z2))
            H[j, k] = H[k, j] = float(Es.i1i2()) / (h * h)
            A[j, k] = A[k, j] = 2.0 * float(np.sum(res.i1() * res.i2())) / (h * h)
            if j == k:
                g[j] = float(Es.i1()) / h
                E = float(Es.real)
    return E, g, H, n, A


def newton_solve(H, g):
    """x = -(H + mu I)^-1 g with the damping reading above; None if no damping makes H positive definite."""
    tr = np.trace(H) / 6.0
    for k in range(7):
        mu = 0.0 if k == 0 else 10.0 ** (k - 4) * tr
        try:
            L = np.linalg.cholesky(H + mu * np.eye(6))
        except np.linalg.LinAlgError:
            continue
        return -np.linalg.solve(L.T, np.linalg.solve(L, g))
    return None


def track_newton(pyr, intr, T_init, T_prev, model, iters=(10, 5, 4), min_corr_frac=0.1, eta=1e-4, **gates):
    """Multi-level ICP from coarse to fine with Newton steps (real poses) and the eta switch above;
    returns (T_k, ok)."""
    T = np.asarray(T_init, np.float64)
    for level in range(len(iters) - 1, -1, -1):
        lintr = measure.level_intrinsics(intr, level)
        npx = lintr[4] * lintr[5]
        for _ in range(iters[level]):
            E, g, H, nv, _ = newton_energy(pyr[level], lintr, level, T, T_prev, model, **gates)
            if nv < min_corr_frac * npx:
                return np.asarray(T_init), False
            if not np.isfinite(eta):
                x = newton_solve(H, g)
            elif E <= eta * nv and np.all(np.linalg.eigvalsh(H) > 0):
                x = -np.linalg.solve(H, g)
            else:
                r, J, valid = correspondences(pyr[level], lintr, level, T, T_prev, model, **gates)
                A, b, _ = normal_equations(r, J, valid)
                x = solve(A, b)
            if x is None:
                return np.asarray(T_init), False
            T = se3.compose(se3.se3_exp(x), T)
    return T, True
