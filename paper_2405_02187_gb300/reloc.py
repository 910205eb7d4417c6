"""Camera relocalisation against a TSDF map (X-SLAM Sec. 5.2): minimise the point-to-plane loss E of
a query depth frame over its pose, by gradient descent, by nonlinear conjugate gradients (the three
optimisers of Sec. 6's ICP comparison, "High order ICP") or by Newton's method with the paper's switch
(gradient direction while E exceeds a threshold eta, Newton direction -H^-1 g below it).

Two losses: the point-to-plane reading (xslam_grad) and the paper's TSDF difference, the sum of squared
changes the query's surface update would make to the map (xslam_grad_tsdf). Every loss, gradient and
Hessian comes from those calls (orders 1 and 2, computed on the GPU); this module holds only the
host-side iteration: 6x6 solves and the step-size control; the SE(3) exponential of a step is the
library's (xslam_se3_exp_compose).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def se3_exp(xi):
    """exp of a left twist (phi then rho) as a 3x4 pose, by the library's FP64 SE(3) exponential."""
    from . import xslam
    return xslam.se3_exp_compose(xi)


def se3_step(xi, T):
    """exp(xi) T, by the library."""
    from . import xslam
    return xslam.se3_exp_compose(xi, T)


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


def _evaluator(handle, loss):
    """(depth, T, order) -> (E, g) for order 1, (E, g, H) for order 2, of the named loss."""
    if loss == "point_to_plane":
        return handle.grad
    if loss == "tsdf":
        def ev(depth, T, order=1):
            E, g, H, _ = handle.grad_tsdf(depth, T, order=order)
            return (E, g) if order == 1 else (E, g, H)
        return ev
    raise ValueError(f"unknown loss {loss!r}")


def _nlcg(ev, depth, T, iters, tol, step0, trace):
    """Polak-Ribiere+ conjugate directions (restarted when not a descent direction). The line search
    along d evaluates a trial step a, fits the parabola through E(0), E'(0) = g.d and E(a), and takes
    its minimiser if the Armijo condition E <= E(0) + 1e-4 a g.d holds there, else the trial step if it
    holds, else halves the trial step. The next trial step is twice the last accepted one."""
    E, g = ev(depth, T, order=1)
    evals = 1
    d = -g
    a = step0 / max(np.linalg.norm(g), 1e-30)
    it = 0
    for it in range(1, iters + 1):
        gd = float(g @ d)
        if gd >= 0.0:
            d, gd = -g, -float(g @ g)
        best = None
        for _ in range(16):
            Ta = se3_step(a * d, T)
            Ea, ga = ev(depth, Ta, order=1)
            evals += 1
            curv = (Ea - E - gd * a) / (a * a)
            if curv > 0.0:
                a2 = -gd / (2.0 * curv)
                T2 = se3_step(a2 * d, T)
                E2, g2 = ev(depth, T2, order=1)
                evals += 1
                if E2 <= E + 1e-4 * a2 * gd and E2 <= Ea:
                    best = (a2, T2, E2, g2)
                    break
            if Ea <= E + 1e-4 * a * gd:
                best = (a, Ta, Ea, ga)
                break
            a *= 0.5
        if best is None:
            break
        a, T1, E1, g1 = best
        step = a * d
        beta = max(0.0, float(g1 @ (g1 - g)) / max(float(g @ g), 1e-300))
        T, E, g = T1, E1, g1
        d = -g + beta * d
        a *= 2.0
        if trace is not None:
            trace.append((T, float(E)))
        if np.linalg.norm(step) < tol:
            break
    return Result(T, it, float(E), 0, evals)


def relocalise(handle, depth, T_init, method="newton", eta=1e-3, iters=30, tol=1e-6, step0=0.01, trace=None,
               loss="point_to_plane"):
    """Minimise E(T) from T_init. handle: an XSlam holding the map; depth: the query's CUDA depth.
    method "gd": steps -a g with a backtracking/expanding step size (a g at most step0 at first);
    method "nlcg": nonlinear conjugate gradients (Polak-Ribiere+, Armijo backtracking);
    method "newton": -H^-1 g when E <= eta and H is positive definite (halved until E decreases),
    otherwise the gradient step. Stops when a step's norm falls below tol. trace (a list, optional)
    receives (T, E) after every iteration. loss: "point_to_plane" (mean squared point-to-plane residual
    against the map ray cast at T) or "tsdf" (sum of squared TSDF changes of the query's surface update
    at T; eta is then on that sum)."""
    T = np.asarray(T_init, np.float64)
    ev = _evaluator(handle, loss)
    if method == "nlcg":
        return _nlcg(ev, depth, T, iters, tol, step0, trace)
    evals = 0
    if method == "newton":
        E, g, H = ev(depth, T, order=2)
    else:
        E, g = ev(depth, T, order=1)
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
                T1 = se3_step(s * direction, T)
                E1, g1, H1 = ev(depth, T1, order=2)
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
                T1 = se3_step(step, T)
                if method == "newton":
                    E1, g1, H1 = ev(depth, T1, order=2)
                else:
                    E1, g1 = ev(depth, T1, order=1)
                evals += 1
                if E1 <= E:
                    T, E, g = T1, E1, g1
                    if method == "newton":
                        H = H1
                    alpha *= 2.0
                    accepted = True
                    break
                alpha *= 0.5
        if accepted and trace is not None:
            trace.append((T, float(E)))
        if not accepted or np.linalg.norm(step) < tol:
            break
    return Result(T, it, float(E), n_newton, evals)


def main(argv=None):
    """Evaluate the TSDF-difference loss with its Hessian on a room map (the command of its profile):
    a dims^3 map from a frames-long 640x480 walk, the last frame as the query 1 cm / 0.5 degrees off."""
    import argparse
    import time

    import torch

    from . import synth, xslam

    ap = argparse.ArgumentParser(description="evaluate the TSDF-difference relocalisation loss")
    ap.add_argument("--dims", type=int, default=256)
    ap.add_argument("--voxel", type=float, default=0.01)
    ap.add_argument("--frames", type=int, default=20)
    ap.add_argument("--evals", type=int, default=5)
    ap.add_argument("--plain64", action="store_true", help="also evaluate the plain FP64 path once")
    a = ap.parse_args(argv)
    wl = synth.room_walk(seed=3, frames=a.frames, dims=a.dims, voxel=a.voxel, device="cuda", resident=True)
    cfg = xslam.default_config()
    cfg.icp_levels = len(wl.icp_iters)
    for i, it in enumerate(wl.icp_iters):
        cfg.icp_iters[i] = it
    cfg.depth_min_m, cfg.depth_max_m, cfg.bilateral = wl.depth_min, wl.depth_max, int(wl.bilateral)
    x = xslam.XSlam(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, cfg, max_lanes=0)
    x.set_pose(wl.poses[0])
    for k in range(a.frames - 1):
        x.frame(wl.depth[k], [], outputs=False)
    x.sync()
    k = a.frames - 1
    T = compose(se3_exp(np.array([0.005, -0.005, 0.0, 0.01, 0.0, 0.0])), wl.poses[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.evals):
        E, g, H, n = x.grad_tsdf(wl.depth[k], T, order=2)
    ms = (time.perf_counter() - t0) / a.evals * 1e3
    print(f"E {E:.6g} |g| {np.linalg.norm(g):.6g} voxels {n} ms/evaluation {ms:.3f} (host round trip included)")
    if a.plain64:
        E64, g64, H64, n64 = x.grad_tsdf_plain64(wl.depth[k], T)
        print(f"plain FP64: E {E64:.6g} voxels {n64} gradient rel err "
              f"{np.linalg.norm(g - g64) / np.linalg.norm(g64):.3g} Hessian rel err "
              f"{np.linalg.norm(H - H64) / np.linalg.norm(H64):.3g}")
    x.close()


if __name__ == "__main__":
    main()
