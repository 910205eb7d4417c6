"""Ray casting of the TSDF volume (X-SLAM Sec. 4.1, "Ray casting" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For pixel u the ray is r(alpha, u) = alpha R K^-1 u_dot + t; alpha advances by a fixed step; F at a
sample is the trilinear interpolation of the volume; a zero crossing F(v_m) > 0, F(v_{m+1}) < 0
gives alpha0 = alpha_m - dalpha F(v_m) / (F(v_{m+1}) - F(v_m)) and the vertex r(alpha0, u); the
normal is grad F / |grad F| at that vertex (Eq. surface_prediction).

Readings of the paper used here (it leaves these open):
  * alpha is the camera-frame depth (K^-1 u_dot has z = 1); samples sit at alpha_m = m * dalpha for
    every integer m with depth_min <= alpha_m <= depth_max; dalpha = ray_step_vox * voxel;
  * a sample is valid only if its trilinear cell lies inside the volume and all 8 corners have W > 0;
    only consecutive valid samples form a pair; the first pair with F_m > 0 and F_{m+1} <= 0 is the
    hit (an exact zero counts as negative); a pair with F_m <= 0 and F_{m+1} > 0 ends the ray with
    no hit;
  * the march decides on real parts with the real pose; the two samples of the hit are then
    re-evaluated with the complex pose and complex TSDF (same cells), which carries the
    imaginary part into alpha0, the vertex and the normal;
  * grad F uses central differences of the trilinear F at the vertex +- one voxel along each axis;
    the pixel is invalid if any of those six samples is invalid;
  * outputs are the global-frame vertex and normal maps plus the real depth Re(alpha0) of the
    vertex (0 where invalid).
"""
from __future__ import annotations

import math

import numpy as np


def _cell(g_real, dims):
    n = np.asarray(dims)
    inside = np.all((g_real >= 0) & (g_real < n - 1), -1)
    i0 = np.where(inside[:, None], np.floor(g_real), 0).astype(np.int64)
    return i0, inside


def trilinear(F, Wt, g, i0, inside, dims):
    """Trilinear interpolation at continuous voxel coordinates g (voxel centres at integers) using
    the cell with min corner i0; returns (value, valid)."""
    nx, ny, _ = dims
    f = g - i0
    val = 0
    ok = inside.copy()
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                lin = (i0[:, 0] + dx) + nx * ((i0[:, 1] + dy) + ny * (i0[:, 2] + dz))
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                val = val + w * F[lin]
                ok &= Wt[lin] > 0
    return val, ok


def raycast(F, Wt, T, intr, dims, origin, voxel, depth_min=0.2, depth_max=4.0, ray_step_vox=1.0, log=None,
            pix=None):
    """Predict (depth, V_g, N_g) at pose T from the volume (F, Wt). Shapes (H, W), (H, W, 3) x2, or
    (P,), (P, 3), (P, 3) for the linear pixel indices ``pix`` if given (each ray is independent).
    ``log``, if a list, receives the discrete decisions (hit sample, pixel validity, trilinear cells)."""
    H, W = intr.height, intr.width
    T = np.asarray(T)
    origin = np.asarray(origin, np.float64)
    uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones_like(uu)], -1).reshape(-1, 3)
    if pix is not None:
        ray = ray[np.asarray(pix)]
    n = ray.shape[0]
    dirs = ray @ T[:, :3].T          # complex if T is
    t = T[:, 3]
    dir_re, t_re = np.real(dirs), np.real(t)
    Fre = np.real(F)
    step = ray_step_vox * voxel
    m0 = math.ceil(depth_min / step - 1e-4)
    m1 = math.floor(depth_max / step + 1e-4)

    prev_valid = np.zeros(n, bool)
    prev_pos = np.zeros(n, bool)
    done = np.zeros(n, bool)
    hit = np.zeros(n, bool)
    m_hit = np.zeros(n, np.int64)
    active = np.arange(n)
    for m in range(m0, m1 + 1):
        if active.size == 0:
            break
        a = m * step
        g = (t_re + a * dir_re[active] - origin) / voxel - 0.5
        i0, inside = _cell(g, dims)
        val, ok = trilinear(Fre, Wt, g, i0, inside, dims)
        pv, pp = prev_valid[active], prev_pos[active]
        both = pv & ok
        pos = val > 0
        hit_now = both & pp & ~pos
        stop_now = both & ~pp & pos
        hit[active[hit_now]] = True
        m_hit[active[hit_now]] = m - 1
        done[active[hit_now | stop_now]] = True
        prev_valid[active] = ok
        prev_pos[active] = pos
        active = active[~(hit_now | stop_now)]

    depth = np.zeros(n)
    dt = np.result_type(dirs, F)
    V = np.zeros((n, 3), dt)
    N = np.zeros((n, 3), dt)
    idx = np.nonzero(hit)[0]
    if idx.size:
        a_m = m_hit[idx] * step
        a_n = (m_hit[idx] + 1) * step
        samples = []
        cells = []
        for a in (a_m, a_n):
            g_re = (t_re + a[:, None] * dir_re[idx] - origin) / voxel - 0.5
            i0, inside = _cell(g_re, dims)
            cells.append(i0)
            g = (t + a[:, None] * dirs[idx] - origin) / voxel - 0.5
            samples.append(trilinear(F, Wt, g, i0, inside, dims)[0])
        Fm, Fn = samples
        alpha0 = a_m - step * Fm / (Fn - Fm)
        v0 = alpha0[:, None] * dirs[idx] + t
        grad = []
        ok = np.ones(idx.size, bool)
        for axis in range(3):
            e = np.zeros(3)
            e[axis] = voxel
            vals = []
            for sgn in (1.0, -1.0):
                g = (v0 + sgn * e - origin) / voxel - 0.5
                i0, inside = _cell(np.real(g), dims)
                cells.append(np.where(inside[:, None], i0, -1))
                val, vok = trilinear(F, Wt, g, i0, inside, dims)
                vals.append(val)
                ok &= vok
            grad.append((vals[0] - vals[1]) / (2 * voxel))
        grad = np.stack(grad, -1)
        g2 = np.sum(grad * grad, -1)
        ok &= np.real(g2) > 0
        norm = np.sqrt(np.where(ok, g2, 1.0) + (0j if np.iscomplexobj(g2) else 0.0))
        good = idx[ok]
        depth[good] = np.real(alpha0[ok])
        V[good] = v0[ok]
        N[good] = (grad / norm[:, None])[ok]
    if log is not None:
        log += [np.where(hit, m_hit, -1), depth > 0] + (cells if idx.size else [])
    if pix is not None:
        return depth, V, N
    return depth.reshape(H, W), V.reshape(H, W, 3), N.reshape(H, W, 3)
