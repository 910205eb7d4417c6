"""Relocalisation loss of a query depth frame against the TSDF map (X-SLAM Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper optimises the query pose T_q with the gradient and Hessian of a loss computed by X-KF. Read
here (as for the second-order workload) as the point-to-plane form: the model maps V_g, N_g are ray
cast from the volume at T_q itself, so the correspondence of pixel u is u, and
  E(T_q) = mean over pixels u of r_u^2,   r_u = (T_q V_q(u) - V_g(u)) . N_g(u),
with V_q = D_q K^-1 u (Eq. vertex) from the range-gated (and, for the 640x480 workload, bilaterally
filtered) query depth; a pixel counts if its query depth and model are valid and |T_q V_q - V_g| is at
most the ICP distance gate. The derivative with respect to a left twist of T_q is Im E(exp(h i e_j) T_q) / h
(Eq. csfd), one complex run per twist component; the volume is taken as real.
"""
from __future__ import annotations

import numpy as np

from . import measure, raycast, se3


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
