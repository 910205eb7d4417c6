"""ICP start poses and the judge of the learned proposal (not part of X-SLAM, which starts ICP at the
previous pose, Sec. 4.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Start poses of frame k, with T_1 = T_{k-1} and T_2 = T_{k-2} (T_2 = T_1 at k = 1):
  constant velocity  T_1 T_2^-1 T_1 (the last camera motion repeated, in the camera frame), its rotation
                     block R then taken through one Newton step of the polar decomposition,
                     1.5 R - 0.5 R R^T R (the nearest rotation to second order): the extrapolation
                     otherwise multiplies a pose's deviation from SO(3) by about 2.4 per frame;
  proposal           T_1 exp(xi), xi = scale * y the network's output (oracle/mlp.py).
Both carry the CSFD lanes of T_1 and T_2 (xi is real: the depth frames carry no perturbation in the
runs that use the proposal).

The judge of a candidate pose T at pyramid level l: with g the ICP distance gate, each pixel u of the
level with a depth D(u) > 0 contributes c_u = min(r_u^2, g^2), where r_u = (p - V)^T N is the
point-to-plane residual of p = T V_k(u) against the model vertex V and normal N at the nearest pixel
of the projection pi(K_l T_{k-1}^-1 p) (read at 2^l times that pixel in the level-0 model maps); a
pixel without such a model point, or with |p - V| > g, contributes g^2. J(T) = mean_u c_u (g^2 for a
level without depth). Lower is better; a pose that loses its correspondences is charged for every
pixel it loses, so J cannot be lowered by drifting off the model.
"""
from __future__ import annotations

import numpy as np

from . import se3


def polar_step(T):
    """T with its rotation block R replaced by 1.5 R - 0.5 R R^T R (plain transpose: on complex lanes
    the step's derivative, which keeps a tangent of SO(3) at R as it is)."""
    T = np.array(T)
    R = T[:, :3]
    T[:, :3] = 1.5 * R - 0.5 * R @ R.T @ R
    return T


def cv_seed(T1, T2):
    """T_1 T_2^-1 T_1, its rotation taken to SO(3) by polar_step."""
    return polar_step(se3.compose(T1, se3.compose(se3.inverse(T2), T1)))


def proposal_seed(T1, xi):
    """T_1 exp(xi) for a real twist xi = (phi, rho)."""
    E = se3.se3_exp(np.asarray(xi, np.float64))
    return se3.compose(T1, E.astype(np.asarray(T1).dtype))


def judge(D, lintr, level, T, T_prev, model, dist_gate):
    """J(T) at one pyramid level (real parts only)."""
    fx, fy, cx, cy, W, H = lintr
    D = np.real(np.asarray(D))
    T = np.real(np.asarray(T))
    Tp = np.real(np.asarray(T_prev))
    g2 = dist_gate ** 2
    vv, uu = np.nonzero(D > 0)
    n = vv.size
    if n == 0:
        return g2
    d = D[vv, uu]
    V = np.stack([d * (uu - cx) / fx, d * (vv - cy) / fy, d], -1)
    p = se3.transform(T, V)
    pc = se3.transform(se3.inverse(Tp), p)
    z = pc[:, 2]
    ok = z > 0
    zs = np.where(ok, z, 1.0)
    ui = np.floor(fx * pc[:, 0] / zs + cx + 0.5)
    vi = np.floor(fy * pc[:, 1] / zs + cy + 0.5)
    ok &= (ui >= 0) & (ui <= W - 1) & (vi >= 0) & (vi <= H - 1)
    s = 2 ** level
    r0 = np.where(ok, vi, 0).astype(np.int64) * s
    c0 = np.where(ok, ui, 0).astype(np.int64) * s
    ok &= np.real(model["depth"][r0, c0]) > 0
    Vm = np.real(model["V"][r0, c0])
    Nm = np.real(model["N"][r0, c0])
    diff = p - Vm
    ok &= np.sum(diff * diff, -1) <= g2
    r = np.sum(diff * Nm, -1)
    c = np.where(ok, np.minimum(r * r, g2), g2)
    return float(c.sum() / n)
