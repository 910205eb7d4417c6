"""Complex SE(3) exponential and pose algebra (X-SLAM Sec. 4.1, "Ray casting" paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Poses are 3x4 arrays [R | t] (camera to world), real or complex. A twist is xi = (phi, rho), rotation
first (Eq. lie). Readings of the paper used here:
  * the "conjugate transpose" a^H in Eq. rotvector and Eq. rotation_jacobi is read as the plain
    transpose a^T: conjugation is not holomorphic and would destroy the imaginary part;
  * theta is taken as the principal square root of phi^T phi (no conjugate), not from arccos of the
    trace (that definition is circular);
  * at theta = 0 the closed forms divide by zero, so for |theta^2| < 1e-4 both R and the rotation
    Jacobian are evaluated from their exponential power series (exact limits, truncation < 1e-24).
"""
from __future__ import annotations

import math

import numpy as np

_SERIES_THETA2 = 1e-4
_SERIES_TERMS = 12


def hat(v):
    """[v]: the skew-symmetric matrix with [v] w = v x w."""
    v = np.asarray(v)
    z = np.zeros((), v.dtype)
    return np.array([[z, -v[2], v[1]], [v[2], z, -v[0]], [-v[1], v[0], z]])


def vee(M):
    """Inverse of hat for a skew-symmetric matrix."""
    return np.array([M[2, 1], M[0, 2], M[1, 0]])


def so3_exp(phi):
    """R = exp(phi) = cos(theta) Id + (1 - cos(theta)) a a^T + sin(theta) [a],  a = phi / theta
    (Eq. rotvector)."""
    phi = np.asarray(phi)
    theta2 = phi @ phi
    if abs(theta2) < _SERIES_THETA2:
        return _series(hat(phi), first=0)
    theta = np.sqrt(theta2 + 0j) if np.iscomplexobj(phi) else math.sqrt(theta2)
    a = phi / theta
    c, s = np.cos(theta), np.sin(theta)
    return c * np.eye(3) + (1 - c) * np.outer(a, a) + s * hat(a)


def rotation_jacobian(phi):
    """R~ = sin(theta)/theta Id + (1 - sin(theta)/theta) a a^T + (1 - cos(theta))/theta [a]
    (Eq. rotation_jacobi)."""
    phi = np.asarray(phi)
    theta2 = phi @ phi
    if abs(theta2) < _SERIES_THETA2:
        return _series(hat(phi), first=1)
    theta = np.sqrt(theta2 + 0j) if np.iscomplexobj(phi) else math.sqrt(theta2)
    a = phi / theta
    c, s = np.cos(theta), np.sin(theta)
    return (s / theta) * np.eye(3) + (1 - s / theta) * np.outer(a, a) + ((1 - c) / theta) * hat(a)


def _series(P, first):
    """sum_n P^n / (n + first)!  (first = 0: exp(P); first = 1: the left Jacobian of SO(3))."""
    out = np.eye(3, dtype=P.dtype)
    term = np.eye(3, dtype=P.dtype)
    for n in range(1, _SERIES_TERMS):
        term = term @ P
        out = out + term / math.factorial(n + first)
    return out


def se3_exp(xi):
    """T = exp(xi) = [exp(phi), R~ rho] (Eq. lie), as a 3x4 array."""
    xi = np.asarray(xi)
    R = so3_exp(xi[:3])
    t = rotation_jacobian(xi[:3]) @ xi[3:]
    return np.concatenate([R, t[:, None]], 1)


def compose(A, B):
    """A * B for 3x4 rigid transforms."""
    A = np.asarray(A)
    B = np.asarray(B)
    return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], 1)


def inverse(T):
    """T^-1 = [R^T | -R^T t] (plain transpose; see module docstring)."""
    T = np.asarray(T)
    Rt = T[:, :3].T
    return np.concatenate([Rt, (-Rt @ T[:, 3])[:, None]], 1)


def transform(T, p):
    """T p for points p of shape (..., 3)."""
    return p @ T[:, :3].T + T[:, 3]


def promote_pose(T, j: int, h: float):
    """Left twist seed: T* = exp(h i e_j) T, j = 0..5 indexing (phi, rho) (Eq. lie, eq. pvnpxi)."""
    return perturb_pose(T, j, 1j * h)


def perturb_pose(T, j: int, delta):
    """exp(delta e_j) T for a complex (CSFD) or real (finite-difference) step delta."""
    dt = np.complex128 if isinstance(delta, complex) else np.float64
    xi = np.zeros(6, dt)
    xi[j] = delta
    return compose(se3_exp(xi), np.asarray(T, dt))


def readout(T_star, h: float):
    """Derivative read-out of a complex pose (Eq. csfd applied to T, eq. pvnpxi):
    dT = Im(T*) / h (12 values, row-major 3x4) and the same derivative as a left twist
    (omega, v) with [omega] = dR R^T and v = dt - omega x t."""
    T_star = np.asarray(T_star)
    T = T_star.real
    dT = T_star.imag / h
    W = dT[:, :3] @ T[:, :3].T
    omega = 0.5 * (vee(W) - vee(W.T))
    v = dT[:, 3] - np.cross(omega, T[:, 3])
    return T, dT, np.concatenate([omega, v])
