"""Camera relocalisation against a TSDF map (X-SLAM Sec. 5.2): minimise the point-to-plane loss E of
a query depth frame over its pose, by gradient descent or by Newton's method with the paper's switch
(gradient direction while E exceeds a threshold eta, Newton direction -H^-1 g below it).

Every loss, gradient and Hessian comes from xslam_grad (orders 1 and 2, computed on the GPU); this
module holds only the host-side iteration: 6x6 solves, the SE(3) exponential of the step, and the
step-size control.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """exp of a left twist (phi then rho) as a 3x4 pose (Rodrigues and the left Jacobian)."""
    xi = np.asarray(xi, np.float64)
    phi, rho = xi[:3], xi[3:]
    th = math.sqrt(float(phi @ phi))
    W = _hat(phi)
    if th < 1e-8:
        R = np.eye(3) + W + 0.5 * W @ W
        V = np.eye(3) + 0.5 * W + W @ W / 6.0
    else:
        a, b = math.sin(th) / th, (1.0 - math.cos(th)) / (th * th)
        c = (th - math.sin(th)) / (th ** 3)
        R = np.eye(3) + a * W + b * W @ W
        V = np.eye(3) + b * W + c * W @ W
    return np.concatenate([R, (V @ rho)[:, None]], 1)


def compose(A, B):
    return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], 1)


def pose_error(T, T_ref):
    """(translation error in metres, rotation error in degrees)."""
    dR = T[:, :3] @ T_ref[:, :3].T
    c = max(-1.0, min(1.0, (np.trace(dR) - 1.0) / 2.0))
    return float(np.linalg.norm(T[:, 3] - T_ref[:, 3])), math.degrees(math.acos(c))


@dataclasses.dataclass
class Result:
    T: np.ndarray
    iterations: int
    loss: float
    newton_steps: int
    evaluations: int


def relocalise(handle, depth, T_init, method="newton", eta=1e-3, iters=30, tol=1e-6, step0=0.01):
    """Minimise E(T) from T_init. handle: an XSlam holding the map; depth: the query's CUDA depth.
    method "gd": steps -a g with a backtracking/expanding step size (a g at most step0 at first);
    method "newton": -H^-1 g when E <= eta and H is positive definite (halved until E decreases),
    otherwise the gradient step. Stops when a step's norm falls below tol."""
    T = np.asarray(T_init, np.float64)
    evals = 0
    if method == "newton":
        E, g, H = handle.grad(depth, T, order=2)
    else:
        E, g = handle.grad(depth, T, order=1)
    evals += 1
    alpha = step0 / max(np.linalg.norm(g), 1e-30)
    n_newton = 0
    it = 0
    for it in range(1, iters + 1):
        direction = None
        if method == "newton" and E <= eta:
            try:
                np.linalg.cholesky(H)
                direction = -np.linalg.solve(H, g)
            except np.linalg.LinAlgError:
                direction = None
        accepted = False
        if direction is not None:
            s = 1.0
            for _ in range(6):
                T1 = compose(se3_exp(s * direction), T)
                E1, g1, H1 = handle.grad(depth, T1, order=2)
                evals += 1
                if E1 <= E:
                    step = s * direction
                    T, E, g, H = T1, E1, g1, H1
                    accepted = True
                    n_newton += 1
                    break
                s *= 0.5
        if not accepted:
            for _ in range(12):
                step = -alpha * g
                T1 = compose(se3_exp(step), T)
                if method == "newton":
                    E1, g1, H1 = handle.grad(depth, T1, order=2)
                else:
                    E1, g1 = handle.grad(depth, T1, order=1)
                evals += 1
                if E1 <= E:
                    T, E, g = T1, E1, g1
                    if method == "newton":
                        H = H1
                    alpha *= 2.0
                    accepted = True
                    break
                alpha *= 0.5
        if not accepted or np.linalg.norm(step) < tol:
            break
    return Result(T, it, float(E), n_newton, evals)
