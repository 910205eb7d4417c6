"""Seeded synthetic workloads: analytic scenes, exact depth renders and camera trajectories.

This module is the one input source shared by the CPU oracle and the CUDA path. It holds no
arithmetic of the SLAM method itself (no TSDF, no ICP, no raycast of a volume, no Lie-group
exponential): depth images are rendered by exact ray/primitive intersection of planes, spheres
and axis-aligned boxes, and camera rotations are built from unit quaternions.

The workloads stand in for the paper's Kinect-class RGB-D sequences (640x480 depth, X-SLAM
Sec. 5.1, TUM RGB-D / ICL-NUIM), which are not available here. Every draw comes from
``numpy.random.Generator(PCG64(seed))``.

Conventions shared with both implementations (they are input conventions, not method steps):
  * camera frame: x right, y down, z forward; pixel (u, v) = (column, row); the ray of pixel u
    passes through the integer pixel coordinate, direction ((u-cx)/fx, (v-cy)/fy, 1);
  * a pose is a 3x4 row-major array [R | t] mapping camera to world (X-SLAM Sec. 4.1, T_{g,k});
  * depth is float32 metres along the camera z axis, 0 marks a pixel with no return.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch


# ----------------------------------------------------------------------------------------------
# Intrinsics and workloads
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclasses.dataclass
class Workload:
    """One seeded sequence: scene, volume geometry, camera, ground-truth poses and depth frames."""

    name: str
    intr: Intrinsics
    dims: tuple  # (nx, ny, nz)
    voxel: float  # metres
    trunc: float  # truncation distance mu, metres
    origin: tuple  # world position of the volume's min corner
    poses: np.ndarray  # (F, 3, 4) float64 ground-truth camera-to-world
    depth: np.ndarray  # (F, H, W) float32 noisy depth, 0 = invalid
    scene: list  # primitives
    seed: int
    icp_iters: tuple = (10, 5, 4)  # finest level first
    depth_min: float = 0.2
    depth_max: float = 4.0
    bilateral: bool = False  # the depth noise exceeds the pixel footprint: filter the raw depth


# ----------------------------------------------------------------------------------------------
# Primitives (exact intersection along o + a*d, a = camera-z depth when d has camera z = 1)
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Plane:
    normal: tuple  # n, points x with n.x = offset
    offset: float


@dataclasses.dataclass(frozen=True)
class Sphere:
    center: tuple
    radius: float


@dataclasses.dataclass(frozen=True)
class Box:
    lo: tuple
    hi: tuple


@dataclasses.dataclass(frozen=True)
class Room:
    """Inside of an axis-aligned box: a ray from inside hits the wall where it exits."""

    lo: tuple
    hi: tuple


def _hit_plane(p: Plane, o, d):
    n = torch.tensor(p.normal, dtype=d.dtype, device=d.device)
    den = d @ n
    num = p.offset - o @ n
    ok = den.abs() > 1e-12
    a = num / torch.where(ok, den, torch.ones_like(den))
    return torch.where(ok & (a > 0), a, torch.full_like(a, math.inf))


def _hit_sphere(s: Sphere, o, d):
    c = torch.tensor(s.center, dtype=d.dtype, device=d.device)
    oc = o - c
    A = (d * d).sum(-1)
    B = 2.0 * (d @ oc)
    C = float(oc @ oc) - s.radius ** 2
    disc = B * B - 4 * A * C
    sq = disc.clamp_min(0.0).sqrt()
    a0 = (-B - sq) / (2 * A)
    a1 = (-B + sq) / (2 * A)
    inf = torch.full_like(a0, math.inf)
    a = torch.where(a0 > 0, a0, torch.where(a1 > 0, a1, inf))
    return torch.where(disc >= 0, a, inf)


def _slabs(lo, hi, o, d):
    lo = torch.tensor(lo, dtype=d.dtype, device=d.device)
    hi = torch.tensor(hi, dtype=d.dtype, device=d.device)
    zero = d == 0
    inv = 1.0 / torch.where(zero, torch.ones_like(d), d)
    t1 = (lo - o) * inv
    t2 = (hi - o) * inv
    inside = (o >= lo) & (o <= hi)
    # an axis the ray is parallel to: no constraint if the origin lies inside that slab
    tmin = torch.where(zero, torch.where(inside, -math.inf, math.inf), torch.minimum(t1, t2))
    tmax = torch.where(zero, torch.where(inside, math.inf, -math.inf), torch.maximum(t1, t2))
    return tmin.amax(-1), tmax.amin(-1)


def _hit_box(b: Box, o, d):
    tn, tf = _slabs(b.lo, b.hi, o, d)
    ok = (tn <= tf) & (tf > 0)
    a = torch.where(tn > 0, tn, tf)
    return torch.where(ok, a, torch.full_like(a, math.inf))


def _hit_room(r: Room, o, d):
    tn, tf = _slabs(r.lo, r.hi, o, d)
    ok = (tn <= tf) & (tf > 0)
    return torch.where(ok, tf, torch.full_like(tf, math.inf))


_HIT = {Plane: _hit_plane, Sphere: _hit_sphere, Box: _hit_box, Room: _hit_room}


def pixel_rays(intr: Intrinsics):
    """Camera-frame ray directions with z = 1 for every pixel, shape (H, W, 3)."""
    u = np.arange(intr.width, dtype=np.float64)
    v = np.arange(intr.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    return np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones_like(uu)], -1)


def render_depth(scene, intr: Intrinsics, pose: np.ndarray, device="cpu") -> np.ndarray:
    """Exact camera-z depth of the nearest primitive for every pixel (float64, 0 = no hit).

    Evaluated in float64 with torch on ``device``; the result is returned as a numpy array."""
    return render_depth_t(scene, intr, pose, device).cpu().numpy()


def render_depth_t(scene, intr: Intrinsics, pose: np.ndarray, device="cpu"):
    """render_depth as a float64 torch tensor on ``device`` (no copy to the host)."""
    pose = np.asarray(pose, np.float64)
    R = torch.tensor(pose[:, :3], dtype=torch.float64, device=device)
    o = torch.tensor(pose[:, 3], dtype=torch.float64, device=device)
    d = torch.tensor(pixel_rays(intr), dtype=torch.float64, device=device) @ R.T
    best = torch.full(d.shape[:2], math.inf, dtype=torch.float64, device=device)
    for prim in scene:
        best = torch.minimum(best, _HIT[type(prim)](prim, o, d))
    return torch.where(torch.isfinite(best), best, torch.zeros_like(best))


# ----------------------------------------------------------------------------------------------
# Rotations from quaternions (input synthesis only)
# ----------------------------------------------------------------------------------------------
def quat_to_matrix(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def axis_angle_quat(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera-to-world pose whose z axis points from eye to target and whose y axis points down."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.concatenate([np.stack([x, y, z], 1), eye[:, None]], 1)


def add_noise(depth: np.ndarray, rng: np.random.Generator, sigma_const=0.0, sigma_quad=0.0):
    """Gaussian depth noise with standard deviation sigma_const + sigma_quad * z^2 (metres)."""
    valid = depth > 0
    sig = sigma_const + sigma_quad * depth * depth
    noisy = depth + rng.standard_normal(depth.shape) * sig
    return np.where(valid & (noisy > 0), noisy, 0.0).astype(np.float32)


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------
def small_orbit(seed: int = 1, frames: int = 20, noise: bool = True, device="cpu") -> Workload:
    """64^3 x 2 cm volume centred at the origin, 160x120 frames (f=140), floor + 3 spheres + 1 box,
    camera on a 1 m circle around the origin, looking at it, 2 degree yaw step, sigma = 1 mm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    intr = Intrinsics(140.0, 140.0, 80.0, 60.0, 160, 120)
    floor_y = -0.5
    scene = [Plane((0.0, 1.0, 0.0), floor_y)]
    for _ in range(3):
        r = rng.uniform(0.1, 0.3)
        c = (rng.uniform(-0.35, 0.35), floor_y + r + rng.uniform(0.0, 0.15), rng.uniform(-0.35, 0.35))
        scene.append(Sphere(c, r))
    bx, bz = rng.uniform(-0.3, 0.3, 2)
    size = rng.uniform(0.12, 0.25, 3)
    scene.append(Box((bx - size[0] / 2, floor_y, bz - size[2] / 2),
                     (bx + size[0] / 2, floor_y + size[1], bz + size[2] / 2)))
    yaw0 = rng.uniform(0, 2 * math.pi)
    poses, depth = [], []
    for k in range(frames):
        yaw = yaw0 + math.radians(2.0) * k
        eye = (math.sin(yaw), 0.3, math.cos(yaw))
        T = look_at(eye, (0.0, -0.1, 0.0))
        d = render_depth(scene, intr, T, device)
        depth.append(add_noise(d, rng, sigma_const=0.001) if noise else d.astype(np.float32))
        poses.append(T)
    return Workload("orbit64_160x120", intr, (64, 64, 64), 0.02, 0.08, (-0.64, -0.64, -0.64),
                    np.array(poses), np.array(depth), scene, seed)


def _room_scene(rng, side, margin, n_prims, obj_r):
    """Walls of a side-metre room (margin inside the volume) and n_prims random spheres and boxes
    inside the central column of horizontal radius obj_r around the room's vertical axis."""
    lo, hi = np.full(3, margin), np.full(3, side - margin)
    scene = [Room(tuple(lo), tuple(hi))]
    c = side / 2.0
    while len(scene) < n_prims + 1:
        kind = rng.integers(0, 2)
        ang = rng.uniform(0, 2 * math.pi)
        rad = obj_r * math.sqrt(rng.uniform())
        if kind == 0:
            r = rng.uniform(0.08, 0.3) * side / 2.56
            cen = np.array([c + rad * math.cos(ang), rng.uniform(lo[1] + r, 0.75 * side), c + rad * math.sin(ang)])
            prim = Sphere(tuple(cen), float(r))
        else:
            size = rng.uniform(0.1, 0.5, 3) * side / 2.56
            cen = np.array([c + rad * math.cos(ang), rng.uniform(lo[1] + size[1] / 2, 0.75 * side), c + rad * math.sin(ang)])
            if rng.uniform() < 0.5:  # rest on the floor
                cen[1] = lo[1] + size[1] / 2
            prim = Box(tuple(cen - size / 2), tuple(cen + size / 2))
        scene.append(prim)
    return scene


def _inward_ok(eye, R, c, r_lo, r_hi, y_lo, y_hi):
    """The camera constraints of the room walk: on the ring around the room's vertical axis, at a
    height in range, looking inward (the horizontal view direction within 35 degrees of the axis
    direction), within 35 degrees of horizontal, upright."""
    dx, dz = c - eye[0], c - eye[2]
    rr = math.hypot(dx, dz)
    fwd = R[:, 2]
    up_cam = -R[:, 1]
    h = math.hypot(fwd[0], fwd[2])
    inward = h > 0 and (fwd[0] * dx + fwd[2] * dz) / (h * rr) > math.cos(math.radians(35))
    return (r_lo < rr < r_hi and y_lo < eye[1] < y_hi and inward and abs(fwd[1]) < math.sin(math.radians(35))
            and up_cam[1] > 0.5)


def room_walk(seed: int = 2, frames: int = 300, width: int = 640, height: int = 480, dims=256,
              voxel: float = 0.01, noise: bool = True, device="cpu", resident: bool = False,
              n_prims: int = 12, stride: int = 1) -> Workload:
    """Room of n_prims (12) random spheres/boxes in the central part of a (dims*voxel)^3 volume walled
    on all sides, seen at 640x480 (f=525, c=(319.5, 239.5)) by a camera that walks a ring around
    them facing inward (translation <= 2 cm, rotation <= 1.5 deg about a random axis per frame; the
    view within 35 degrees of the direction to the room's axis and of horizontal); depth noise
    sigma = 1.5 mm * z^2. Lengths scale with the room side (2.56 m at 256^3 x 1 cm).

    resident=True keeps the frames on ``device`` as one float32 torch tensor (frames, H, W) and draws
    the noise there from a torch generator seeded with ``seed`` (a different stream of normals than
    the numpy one, for large batched workloads). stride > 1 renders every stride-th pose of the walk
    (frames rendered frames, stride walk steps apart: a faster camera on the same kind of path)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = width / 640.0
    intr = Intrinsics(525.0 * s, 525.0 * s, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    side = dims * voxel
    k = side / 2.56
    margin = 0.06 * k
    c = side / 2.0
    r_lo, r_hi = 0.95 * k, 1.12 * k          # camera ring (walls at 1.22 k from the axis)
    y_lo, y_hi = 0.85 * k, 1.7 * k
    scene = _room_scene(rng, side, margin, n_prims, 0.5 * k)  # objects within 0.5 k + 0.3 k of the axis
    base = look_at(np.zeros(3), (0.0, 0.0, 1.0))[:, :3]  # y down, z forward along +z
    while True:  # a start pose on the ring looking at the axis, within the constraints
        ang = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(r_lo + 0.03 * k, r_hi - 0.03 * k)
        eye = np.array([c + rad * math.cos(ang), rng.uniform(y_lo + 0.05 * k, y_hi - 0.05 * k), c + rad * math.sin(ang)])
        yaw = math.atan2(c - eye[0], c - eye[2]) + rng.uniform(-0.3, 0.3)
        q = axis_angle_quat((0.0, 1.0, 0.0), yaw)
        pitch = axis_angle_quat((1.0, 0.0, 0.0), rng.uniform(-0.2, 0.2))
        q = np.array([q[0] * pitch[0] - q[1:] @ pitch[1:], *(q[0] * pitch[1:] + pitch[0] * q[1:] + np.cross(q[1:], pitch[1:]))])
        if _inward_ok(eye, quat_to_matrix(q) @ base, c, r_lo, r_hi, y_lo, y_hi):
            break
    poses, depth = [], []
    if resident:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
    for f in range((frames - 1) * stride + 1):
        if f > 0:
            for _ in range(100):
                step = rng.standard_normal(3)
                step *= rng.uniform() ** (1 / 3) * 0.02 / np.linalg.norm(step)
                ang = math.radians(1.5) * rng.uniform()
                dq = axis_angle_quat(rng.standard_normal(3), ang)
                nq = np.array([
                    dq[0] * q[0] - dq[1:] @ q[1:],
                    *(dq[0] * q[1:] + q[0] * dq[1:] + np.cross(dq[1:], q[1:]))])
                ne = eye + step
                if _inward_ok(ne, quat_to_matrix(nq) @ base, c, r_lo, r_hi, y_lo, y_hi):
                    eye, q = ne, nq
                    break
        if f % stride:
            continue
        R = quat_to_matrix(q) @ base
        T = np.concatenate([R, eye[:, None]], 1)
        if resident:
            d = render_depth_t(scene, intr, T, device)
            if noise:
                z = torch.randn(d.shape, generator=gen, dtype=torch.float64, device=d.device)
                nd = d + z * (0.0015 * d * d)
                d = torch.where((d > 0) & (nd > 0), nd, torch.zeros_like(nd))
            depth.append(d.to(torch.float32))
        else:
            d = render_depth(scene, intr, T, device)
            depth.append(add_noise(d, rng, sigma_quad=0.0015) if noise else d.astype(np.float32))
        poses.append(T)
    return Workload(f"room{dims}_{width}x{height}", intr, (dims, dims, dims), voxel, 4 * voxel,
                    (0.0, 0.0, 0.0), np.array(poses), torch.stack(depth) if resident else np.array(depth), scene,
                    seed, depth_min=0.3, depth_max=4.0, bilateral=True)


def room_smooth(seed: int = 3, frames: int = 1000, width: int = 640, height: int = 480, dims=512,
                voxel: float = 0.005, rho: float = 0.9, step_m: float = 0.02, step_deg: float = 1.5,
                jerk_every: int = 25, noise: bool = True, device="cpu", resident: bool = True,
                n_prims: int = 12) -> Workload:
    """The room of room_walk (same geometry, intrinsics, noise and ring constraints) seen by a camera
    with inertia: each frame's translation step and rotation vector are rho times the previous ones
    plus sqrt(1 - rho^2) times a fresh draw of the random walk's step (translation uniform in a ball of
    radius step_m, rotation up to step_deg about a random axis); every jerk_every frames, and whenever
    a step would leave the ring constraints, the motion is drawn afresh (an abrupt change)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = width / 640.0
    intr = Intrinsics(525.0 * s, 525.0 * s, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    side = dims * voxel
    k = side / 2.56
    margin = 0.06 * k
    c = side / 2.0
    r_lo, r_hi = 0.95 * k, 1.12 * k
    y_lo, y_hi = 0.85 * k, 1.7 * k
    scene = _room_scene(rng, side, margin, n_prims, 0.5 * k)
    base = look_at(np.zeros(3), (0.0, 0.0, 1.0))[:, :3]
    while True:
        ang = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(r_lo + 0.03 * k, r_hi - 0.03 * k)
        eye = np.array([c + rad * math.cos(ang), rng.uniform(y_lo + 0.05 * k, y_hi - 0.05 * k), c + rad * math.sin(ang)])
        yaw = math.atan2(c - eye[0], c - eye[2]) + rng.uniform(-0.3, 0.3)
        q = axis_angle_quat((0.0, 1.0, 0.0), yaw)
        if _inward_ok(eye, quat_to_matrix(q) @ base, c, r_lo, r_hi, y_lo, y_hi):
            break

    def draw():
        st = rng.standard_normal(3)
        st *= rng.uniform() ** (1 / 3) * step_m / np.linalg.norm(st)
        ax = rng.standard_normal(3)
        return st, ax / np.linalg.norm(ax) * math.radians(step_deg) * rng.uniform()

    def qmul(a, b):
        return np.array([a[0] * b[0] - a[1:] @ b[1:], *(a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:]))])

    v, w = draw()
    poses, depth = [], []
    if resident:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
    a = math.sqrt(1.0 - rho * rho)
    for f in range(frames):
        if f > 0:
            fresh = f % jerk_every == 0
            for tries in range(100):
                dv, dw = draw()
                nv, nw = (dv, dw) if fresh or tries > 0 else (rho * v + a * dv, rho * w + a * dw)
                ang = float(np.linalg.norm(nw))
                dq = axis_angle_quat(nw / ang if ang > 0 else (1.0, 0.0, 0.0), ang)
                nq = qmul(dq, q)
                ne = eye + nv
                if _inward_ok(ne, quat_to_matrix(nq) @ base, c, r_lo, r_hi, y_lo, y_hi):
                    eye, q, v, w = ne, nq, nv, nw
                    break
        R = quat_to_matrix(q) @ base
        T = np.concatenate([R, eye[:, None]], 1)
        if resident:
            d = render_depth_t(scene, intr, T, device)
            if noise:
                z = torch.randn(d.shape, generator=gen, dtype=torch.float64, device=d.device)
                nd = d + z * (0.0015 * d * d)
                d = torch.where((d > 0) & (nd > 0), nd, torch.zeros_like(nd))
            depth.append(d.to(torch.float32))
        else:
            d = render_depth(scene, intr, T, device)
            depth.append(add_noise(d, rng, sigma_quad=0.0015) if noise else d.astype(np.float32))
        poses.append(T)
    return Workload(f"roomsmooth{dims}_{width}x{height}", intr, (dims, dims, dims), voxel, 4 * voxel,
                    (0.0, 0.0, 0.0), np.array(poses), torch.stack(depth) if resident else np.array(depth), scene,
                    seed, depth_min=0.3, depth_max=4.0, bilateral=True)


def tiny(seed: int = 3, frames: int = 3, n: int = 24, width: int = 40, height: int = 30, noise=False,
         device="cpu") -> Workload:
    """A 24^3 volume of 3 cm voxels around a room corner (floor and two walls) with a sphere, seen by
    40x30 frames (f = 30) from a camera turning 1.5 degrees per frame about the vertical axis; a
    two-level pyramid. This is the size where the oracle is checked against central finite
    differences."""
    rng = np.random.Generator(np.random.PCG64(seed))
    intr = Intrinsics(30.0, 30.0, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    voxel = 0.03
    half = n * voxel / 2
    scene = [Plane((0.0, 1.0, 0.0), -0.22), Plane((0.0, 0.0, 1.0), -0.25), Plane((1.0, 0.0, 0.0), -0.25),
             Sphere((rng.uniform(-0.05, 0.0), -0.1, rng.uniform(-0.08, -0.03)), 0.1)]
    eye0 = np.array([0.3, 0.2, 0.3])
    poses, depth = [], []
    for k in range(frames):
        yaw = math.radians(1.5) * k
        c, s = math.cos(yaw), math.sin(yaw)
        eye = np.array([c * eye0[0] + s * eye0[2], eye0[1], -s * eye0[0] + c * eye0[2]])
        T = look_at(eye, (-0.15, -0.15, -0.15))
        d = render_depth(scene, intr, T, device)
        depth.append(add_noise(d, rng, sigma_const=0.0005) if noise else d.astype(np.float32))
        poses.append(T)
    return Workload("corner24_40x30", intr, (n, n, n), voxel, 4 * voxel, (-half, -half, -half),
                    np.array(poses), np.array(depth), scene, seed, icp_iters=(10, 5))


def batch_trajectories(seed: int = 7, n: int = 32, min_frames: int = 50, max_frames: int = 400,
                       grids=(128, 192, 256, 320, 384), sizes=((320, 240), (640, 480)), max_k: int = 12,
                       side: float = 2.56, noise: bool = True, device="cpu", resident: bool = False):
    """n independent room walks of uneven length for batched runs: trajectory i has a seeded length
    in [min_frames, max_frames], image size from ``sizes``, a cubic grid from ``grids`` over the same
    side-metre room (voxel = side / grid, truncation 4 voxels) and K in [1, max_k] perturbation lanes.
    Returns a list of (Workload, lanes) with lanes = [(kind, index), ...] drawn from the POSE0 twist
    components, then TRUNC, DEPTH and further POSE0 components. resident: as for room_walk."""
    rng = np.random.Generator(np.random.PCG64(seed))
    order = [(0, j) for j in range(6)] + [(2, 0), (3, -1)] + [(0, j) for j in range(6)]
    out = []
    for i in range(n):
        frames = int(rng.integers(min_frames, max_frames + 1))
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        g = int(grids[int(rng.integers(0, len(grids)))])
        k = int(rng.integers(1, max_k + 1))
        wl = room_walk(seed=int(rng.integers(0, 2 ** 31)), frames=frames, width=w, height=h, dims=g, voxel=side / g,
                       noise=noise, device=device, resident=resident)
        out.append((wl, order[:k]))
    return out
