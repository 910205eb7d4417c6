"""Learned pose proposal: the small perceptron that guesses the camera motion between two depth frames
so that the coarsest ICP level of the X-KinectFusion step (Sec. 4.1) starts near the answer. The
paper has no such network; this is the oracle of the one the GPU path trains and runs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Input features. A depth map of W x H pixels (W a multiple of 80, H of 60) is cut into 80 x 60 blocks
of (W/80) x (H/60) pixels; a block's feature is the mean of its depths inside the range gate
[depth_min, depth_max] (the gate of Sec. 4.1's surface measurement), divided by DEPTH_SCALE = 4 m,
and 0 when the block has no such depth. A pair (D_i, D_j) gives x = [f(D_i), f(D_j)] (9600 values,
row-major blocks, the earlier frame first).

Network, as the GPU computes it: BF16 operands, FP32 accumulation. With q = rounding to bfloat16
(nearest, ties to even, from the FP32 value):
    a_0 = q(x);  z_l = a_{l-1} q(W_l)^T + b_l;  a_l = q(relu(z_l)) (l < L);  y = z_L.
``bf16=False`` makes q the identity (the exact FP64 network; the finite-difference pins use it).
Loss over a batch of B pairs with targets t: E = 1/(2B) sum_b |y_b - t_b|^2.

Gradient (backward pass). dz_L = (y - t) / B and, for l = L..1,
    dW_l = q(dz_l)^T a_{l-1},   db_l = sum_b dz_l,   dz_{l-1} = (q(dz_l) q(W_l)) * [a_{l-1} > 0],
i.e. the exact gradient of E with the roundings passed through as the identity (straight-through),
with the backward GEMM operands rounded where the GPU rounds them. With bf16=False it is the exact
gradient of E.

Optimiser: Adam (Kingma and Ba, 2015) with bias correction, on FP32 master weights.

Output: the network predicts the camera motion between the two frames as a twist xi = (phi, rho) in
the earlier camera's frame, T_j = T_i exp(xi), divided component-wise by a scale vector fixed from
the training targets (``se3_log`` below gives the target twist of two poses).
"""
from __future__ import annotations

import math

import numpy as np

FEAT_W, FEAT_H = 80, 60
DEPTH_SCALE = 4.0


def bf16(x):
    """Round to the nearest bfloat16 (ties to even) after rounding to float32; returns float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(D, depth_min: float, depth_max: float):
    """80 x 60 block means of the in-range depths of D, / DEPTH_SCALE (0 for an empty block); 4800
    values, row-major."""
    D = np.asarray(D, np.float64)
    H, W = D.shape
    assert W % FEAT_W == 0 and H % FEAT_H == 0, "image size must be a multiple of 80 x 60"
    by, bx = H // FEAT_H, W // FEAT_W
    out = np.zeros(FEAT_W * FEAT_H)
    for i in range(FEAT_H):
        for j in range(FEAT_W):
            s, n = 0.0, 0
            for y in range(i * by, (i + 1) * by):
                for x in range(j * bx, (j + 1) * bx):
                    d = D[y, x]
                    if depth_min <= d <= depth_max:
                        s += d
                        n += 1
            out[i * FEAT_W + j] = s / n / DEPTH_SCALE if n else 0.0
    return out


def init_params(sizes, rng):
    """He-uniform weights (bound sqrt(6 / fan_in)) and zero biases: list of (W (out, in), b (out))."""
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        bound = math.sqrt(6.0 / n_in)
        params.append((rng.uniform(-bound, bound, (n_out, n_in)), np.zeros(n_out)))
    return params


def forward(params, x, bf16_ops=True):
    """y and the per-layer inputs a_0..a_{L-1} (as the layers consume them) for a batch x (B, n_0)."""
    q = bf16 if bf16_ops else (lambda v: np.asarray(v, np.float64))
    a = q(x)
    acts = [a]
    z = None
    for l, (W, b) in enumerate(params):
        z = a @ q(W).T + b
        if l < len(params) - 1:
            a = q(np.maximum(z, 0.0))
            acts.append(a)
    return z, acts


def loss(y, t):
    return 0.5 * float(np.sum((y - t) ** 2)) / y.shape[0]


def gradient(params, x, t, bf16_ops=True):
    """(E, [(dW_l, db_l)]) for a batch x (B, n_0) with targets t (B, n_L)."""
    q = bf16 if bf16_ops else (lambda v: np.asarray(v, np.float64))
    y, acts = forward(params, x, bf16_ops)
    B = x.shape[0]
    dz = (y - t) / B
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dzq = q(dz)
        grads[l] = (dzq.T @ acts[l], dz.sum(0))
        if l > 0:
            dz = (dzq @ q(W)) * (acts[l] > 0)
    return loss(y, t), grads


def adam_step(p, g, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the arrays p (in place), with moments m, v (in place); step counts from 1."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)


def se3_log(T):
    """Twist xi = (phi, rho) with exp(xi) = T (rotation angle below pi): phi from the rotation's axis
    and angle, rho = J(phi)^-1 t with J the left Jacobian of SO(3)."""
    T = np.asarray(T, np.float64)
    R, t = T[:, :3], T[:, 3]
    c = max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))
    th = math.acos(c)
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2.0
    if th < 1e-8:
        phi = w
    else:
        phi = w * th / math.sin(th)
    P = np.array([[0.0, -phi[2], phi[1]], [phi[2], 0.0, -phi[0]], [-phi[1], phi[0], 0.0]])
    th = float(np.linalg.norm(phi))
    if th < 1e-8:
        J = np.eye(3) + 0.5 * P
    else:
        J = np.eye(3) + (1.0 - math.cos(th)) / th ** 2 * P + (th - math.sin(th)) / th ** 3 * (P @ P)
    return np.concatenate([phi, np.linalg.solve(J, t)])


def pair_target(T_i, T_j):
    """Twist of the motion from camera i to camera j in camera i's frame: log(T_i^-1 T_j)."""
    T_i = np.asarray(T_i, np.float64)
    T_j = np.asarray(T_j, np.float64)
    Ri, ti = T_i[:, :3], T_i[:, 3]
    D = np.concatenate([Ri.T @ T_j[:, :3], (Ri.T @ (T_j[:, 3] - ti))[:, None]], 1)
    return se3_log(D)
