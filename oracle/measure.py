"""Surface measurement (X-SLAM Sec. 4.1, "Surface measurement" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Functions accept real (float64) or complex (complex128) depth; every validity decision is taken on
real parts, the imaginary part follows the chosen branch.

Readings of the paper used here (it names the operations but not their parameters):
  * the bilateral filter of the raw depth is off (all workloads are synthetic);
  * depth outside [depth_min, depth_max] counts as invalid (0);
  * the pyramid has 3 levels; level l+1 at pixel u is the 5x5 binomial ([1 4 6 4 1]/16 per axis)
    average of level l around pixel 2u over the taps that are valid and within ``range_m`` of the
    centre depth, and is invalid where the centre is invalid; the perturbation is averaged with the
    same weights ("The perturbed hi is also Gaussian smoothed");
  * level l uses intrinsics fx/2^l, fy/2^l, cx/2^l, cy/2^l, so its pixel u sees the ray of level-0
    pixel 2^l u;
  * a vertex has a normal only if it and its +x and +y neighbours are valid (last column and last
    row have none).
"""
from __future__ import annotations

import numpy as np

BINOMIAL5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def level_intrinsics(intr, level: int):
    """(fx, fy, cx, cy, width, height) of pyramid level ``level``."""
    s = 2 ** level
    return (intr.fx / s, intr.fy / s, intr.cx / s, intr.cy / s, intr.width // s, intr.height // s)


def range_gate(D, depth_min: float, depth_max: float):
    """Depth outside the sensor range becomes invalid (0)."""
    Dr = np.real(D)
    return np.where((Dr >= depth_min) & (Dr <= depth_max), D, 0)


def pyramid_down(D, range_m: float):
    """One coarser level (Sec. 4.1: "A coarser level depth is computed by applying Gaussian
    smoothing"), centred at (2u, 2v) of the finer level."""
    H, W = D.shape
    h2, w2 = H // 2, W // 2
    P = np.zeros((H + 4, W + 4), D.dtype)
    P[2:-2, 2:-2] = D
    C = D[0:2 * h2:2, 0:2 * w2:2]
    Cr = np.real(C)
    acc = np.zeros((h2, w2), D.dtype)
    wsum = np.zeros((h2, w2))
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            tap = P[2 + dy:2 + dy + 2 * h2:2, 2 + dx:2 + dx + 2 * w2:2]
            tr = np.real(tap)
            ok = (tr > 0) & (np.abs(tr - Cr) < range_m)
            w = BINOMIAL5[dy + 2] * BINOMIAL5[dx + 2] * ok
            acc = acc + w * tap
            wsum = wsum + w
    out = np.where(Cr > 0, acc / np.where(wsum > 0, wsum, 1.0), 0)
    return out.astype(D.dtype)


def pyramid(D0, levels: int, range_m: float):
    out = [D0]
    for _ in range(1, levels):
        out.append(pyramid_down(out[-1], range_m))
    return out


def vertex_map(D, lintr):
    """V_k(u) = D_k(u) K^-1 u_dot (Eq. vertex), shape (H, W, 3)."""
    fx, fy, cx, cy, W, H = lintr
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    return np.stack([D * ((u - cx) / fx), D * ((v - cy) / fy), D * np.ones((H, W))], -1)


def normal_map(D, V):
    """N_k(u) = [V(u^x+) - V(u)] x [V(u^y+) - V(u)] / |...| (Eq. normal); returns (N, valid)."""
    H, W = D.shape
    Dr = np.real(D)
    valid = np.zeros((H, W), bool)
    valid[:-1, :-1] = (Dr[:-1, :-1] > 0) & (Dr[:-1, 1:] > 0) & (Dr[1:, :-1] > 0)
    ex = np.zeros_like(V)
    ey = np.zeros_like(V)
    ex[:, :-1] = V[:, 1:] - V[:, :-1]
    ey[:-1, :] = V[1:, :] - V[:-1, :]
    c = np.cross(ex, ey)
    n2 = np.sum(c * c, -1)
    valid &= np.real(n2) > 0
    norm = np.sqrt(np.where(valid, n2, 1.0) + (0j if np.iscomplexobj(n2) else 0.0))
    N = np.where(valid[..., None], c / norm[..., None], 0)
    return N, valid
