"""Surface measurement (X-SLAM Sec. 4.1, "Surface measurement" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Functions accept real (float64) or complex (complex128) depth; every validity decision is taken on
real parts, the imaginary part follows the chosen branch.

Readings of the paper used here (it names the operations but not their parameters):
  * depth outside [depth_min, depth_max] counts as invalid (0), before any filtering;
  * the bilateral filter of the raw depth (Sec. 4.1, "applying a bilateral filter to the raw depth map
    for noise reduction") is optional: a 7x7 window, spatial sigma 4.5 pixels, range sigma 0.03 m,
    over valid taps only, invalid where the centre is invalid; it is on where the depth noise exceeds
    the pixel footprint (the 640x480 workload), off otherwise;
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


def bilateral(D, sigma_s: float = 4.5, sigma_r: float = 0.03, radius: int = 3):
    """Edge-preserving smoothing of the raw depth (Sec. 4.1, surface measurement): the normalised sum
    of w_s(u - u') w_r(D(u) - D(u')) D(u') over the valid taps u' of the (2 radius + 1)^2 window, with
    Gaussian w_s and w_r; tap validity is decided on real parts, the range weight is evaluated on the
    complex depths (it is a smooth function of them)."""
    H, W = D.shape
    P = np.zeros((H + 2 * radius, W + 2 * radius), D.dtype)
    P[radius:-radius, radius:-radius] = D
    Cr = np.real(D)
    acc = np.zeros((H, W), D.dtype)
    wsum = np.zeros((H, W), D.dtype)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            tap = P[radius + dy:radius + dy + H, radius + dx:radius + dx + W]
            tr = np.real(tap)
            w = np.exp(-(dx * dx + dy * dy) / (2 * sigma_s ** 2) - (tap - D) ** 2 / (2 * sigma_r ** 2)) * (tr > 0)
            acc = acc + w * tap
            wsum = wsum + w
    return np.where(Cr > 0, acc / np.where(np.real(wsum) > 0, wsum, 1.0), 0).astype(D.dtype)


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
