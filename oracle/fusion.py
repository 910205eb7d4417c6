"""Surface update: projective TSDF fusion (X-SLAM Sec. 4.1, "Surface Update" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For a voxel p (Sec. 4.1):
  x = pi(K T^-1 p),
  eta = |K^-1 x_dot|^-1 |t - p| - L(x)    (Eq. bi_interpolate; L = bilinear depth at x),
  F_D = Psi(eta), W_D = 1,
  F <- (W F + W_D F_D) / (W + W_D),  W <- W + W_D.

Readings of the paper used here:
  * sign: the garbled Psi is read as the KinectFusion TSDF, positive in free space:
    sdf = L(x) - |K^-1 x_dot|^-1 |t - p| (the paper's eta with its sign flipped), null if
    sdf < -mu, otherwise F_D = min(1, sdf / mu) (no extra sgn). |K^-1 x_dot|^-1 |t - p| equals the
    camera-frame depth of p because p lies on the ray of its own projection;
  * voxel centres are p = origin + (i + 0.5) * voxel, linear index x + nx * (y + ny * z);
  * an unobserved voxel holds F = 1, W = 0;
  * L(x) needs its four taps valid and |D10-D00| + |D01-D00| + |D11-D00| < disc_gate (the
    depth-discontinuity rule of Sec. 4.1 "derivative w.r.t. pixel coordinate", with N(u) the other
    three corners of the bilinear cell); otherwise the voxel is not updated; the pixel centre is at
    the integer coordinate (no -0.5 shift);
  * x must satisfy 0 <= x < W-1, 0 <= y < H-1 and p must be in front of the camera;
  * W_D = 1 makes Im W identically zero, so W stays real; an optional cap w_max (default none)
    limits W after the average.
"""
from __future__ import annotations

import numpy as np

from . import se3


def voxel_centres(idx, dims, origin, voxel):
    nx, ny, _ = dims
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    return np.asarray(origin, np.float64) + (np.stack([i, j, k], -1) + 0.5) * voxel


def bilinear_depth(D, x, y, disc_gate):
    """L(x): bilinear depth at real-valued pixel coordinates, with validity (Sec. 4.1)."""
    H, W = D.shape
    xr, yr = np.real(x), np.real(y)
    inside = (xr >= 0) & (xr < W - 1) & (yr >= 0) & (yr < H - 1)
    i0 = np.where(inside, np.floor(xr), 0).astype(np.int64)
    j0 = np.where(inside, np.floor(yr), 0).astype(np.int64)
    a = x - i0
    b = y - j0
    d00, d10 = D[j0, i0], D[j0, i0 + 1]
    d01, d11 = D[j0 + 1, i0], D[j0 + 1, i0 + 1]
    r00, r10, r01, r11 = (np.real(d) for d in (d00, d10, d01, d11))
    ok = inside & (r00 > 0) & (r10 > 0) & (r01 > 0) & (r11 > 0)
    ok &= (np.abs(r10 - r00) + np.abs(r01 - r00) + np.abs(r11 - r00)) < disc_gate
    L = (1 - a) * (1 - b) * d00 + a * (1 - b) * d10 + (1 - a) * b * d01 + a * b * d11
    return L, ok


def integrate(F, Wt, D, T, intr, dims, origin, voxel, mu, disc_gate=0.1, w_max=np.inf,
              idx=None, chunk=1 << 20, log=None):
    """Fuse depth D at camera pose T into (F, Wt) in place; returns the mask of updated voxels.

    F: flat (nx*ny*nz,) real or complex TSDF; Wt: flat real weights; T: 3x4 real or complex pose;
    mu: real or complex truncation. ``idx`` restricts the update to those linear voxel indices.
    ``log``, if a list, receives the discrete decisions (update mask, clamp mask, pixel cells)."""
    if idx is None:
        idx = np.arange(F.shape[0])
    Tinv = se3.inverse(T)
    t = np.asarray(T)[:, 3]
    mu_re = np.real(mu)
    updated = np.zeros(idx.shape[0], bool)
    for s in range(0, idx.shape[0], chunk):
        ii = idx[s:s + chunk]
        p = voxel_centres(ii, dims, origin, voxel)
        pc = se3.transform(Tinv, p)
        z = pc[:, 2]
        front = np.real(z) > 0
        zs = np.where(front, z, 1.0)
        x = intr.fx * pc[:, 0] / zs + intr.cx
        y = intr.fy * pc[:, 1] / zs + intr.cy
        L, ok = bilinear_depth(D, x, y, disc_gate)
        lam = np.sqrt(((x - intr.cx) / intr.fx) ** 2 + ((y - intr.cy) / intr.fy) ** 2 + 1.0)
        dvec = t - p
        dist = np.sqrt(np.sum(dvec * dvec, -1))
        sdf = L - dist / lam
        keep = front & ok & (np.real(sdf) >= -mu_re)
        FD = np.where(np.real(sdf) >= mu_re, 1.0, sdf / mu)
        k = ii[keep]
        w = Wt[k]
        F[k] = (w * F[k] + FD[keep]) / (w + 1.0)
        Wt[k] = np.minimum(w + 1.0, w_max)
        updated[s:s + chunk] = keep
        if log is not None:
            log += [keep, keep & (np.real(sdf) >= mu_re), np.where(keep, np.floor(np.real(x)), -1),
                    np.where(keep, np.floor(np.real(y)), -1)]
    return updated
