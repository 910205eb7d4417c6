"""The per-frame X-KinectFusion step in CSFD arithmetic (X-SLAM Sec. 4.1) and whole-sequence runs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Frame k (Sec. 4.1, in the paper's order): surface measurement of D_k (range gate, optional bilateral
filter, pyramid, vertex
and normal maps), camera pose estimation by multi-level ICP against the model maps ray-cast at
T_{k-1} (frame 0 keeps its given pose), surface update of the TSDF at T_k, and ray casting at T_k
for the next frame.

Seeds (which input carries the imaginary perturbation h i; one complex run per seed):
  POSE0 (kind 0, index 0..5): T_0* = exp(h i e_index) T_0 (Eq. lie), a left twist of frame 0's pose;
  POSE (kind 1, index 0..5): frame k's own pose before ICP, T~_{k,0}* = exp(h i e_index) T~_{k,0}
    (the start of ICP; T_0 itself at frame 0);
  TRUNC (kind 2): mu* = mu + h i;
  DEPTH (kind 3, index -1 for every pixel, else one linear pixel index): D_k* = D_k + h i at every
    frame (Eq. csfd_depth);
  POSE_TRACKED (kind 4, index 0..5): frame k's tracked pose as the surface update and the ray cast use
    it, T_{g,k}* = exp(h i e_index) T_{g,k} (Eq. lie, Eq. pvnpxi and the surface update's derivative
    with respect to xi_k).
The derivative of any result X is Im(X*) / h (Eq. csfd). The two per-frame pose kinds restart at every
frame: before frame k > 0 the run drops the imaginary parts that earlier frames' perturbations left in
its pose, TSDF and model maps, so that Im(X_k*) / h is the derivative of frame k's results with respect
to frame k's pose alone (the paper's dF_k / dxi_{k,i}), not a sum over the frames.

Readings: ICP starts each frame from the previous pose T_{k-1} (Sec. 4.1, "initialized with the
previous frame pose"); on an ICP failure the frame is fused at T_{k-1} and the step reports it.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fusion, icp, measure, mlp, proposal, raycast, se3
from .csfd import H_ORACLE

POSE0, POSE, TRUNC, DEPTH, POSE_TRACKED = 0, 1, 2, 3, 4
PER_FRAME = (POSE, POSE_TRACKED)


@dataclasses.dataclass
class Config:
    icp_iters: tuple = (10, 5, 4)  # finest level first, run coarse to fine
    dist_gate: float = 0.1
    normal_gate_deg: float = 20.0
    disc_gate: float = 0.1
    min_corr_frac: float = 0.1
    ray_step_vox: float = 1.0
    depth_min: float = 0.2
    depth_max: float = 4.0
    pyr_range: float = 0.09
    w_max: float = np.inf
    bilateral: bool = False
    icp_newton: bool = False  # Newton ICP (real runs only)
    icp_newton_eta: float = 1e-4  # m^2: mean squared residual below which the Newton matrix is used
    icp_seed: str = "prev"     # ICP start: "prev" T_{k-1} (Sec. 4.1) or "cv" constant velocity
    icp_stop: float = 0.0      # > 0: a level ends after a step |x| below this (oracle/icp.py track)
    proposal: object = None    # a Proposal: learned start pose judged against the "icp_seed" start


@dataclasses.dataclass
class Proposal:
    """The learned proposal (oracle/mlp.py, oracle/proposal.py): the network seeds a second ICP run;
    both runs go from the coarsest level down to judge_level, the lower judge J wins (the network's
    run only if it did not fail and J_B <= J_A) and continues to level 0."""
    params: list
    scale: np.ndarray
    judge_level: int = 2


@dataclasses.dataclass
class Seed:
    """A perturbed input. ``imag`` True: the CSFD perturbation h i; False: a real shift by h (used
    only to evaluate central finite differences of the real pipeline)."""
    kind: int
    index: int = 0
    h: float = H_ORACLE
    imag: bool = True

    @property
    def delta(self):
        return 1j * self.h if self.imag else self.h


class XKinectFusion:
    """One run of the pipeline: real (seed None) or with one complex perturbation direction."""

    def __init__(self, dims, voxel, mu, origin, intr, T0, cfg: Config = None, seed: Seed = None):
        self.dims, self.voxel, self.origin, self.intr = tuple(dims), voxel, tuple(origin), intr
        self.cfg = cfg or Config()
        self.seed = seed
        self.cplx = seed is not None and seed.imag
        self.pert = seed is not None
        dt = np.complex128 if self.cplx else np.float64
        n = int(np.prod(dims))
        self.F = np.ones(n, dt)
        self.W = np.zeros(n)
        self.mu = mu + (seed.delta if self.pert and seed.kind == TRUNC else 0)
        T0 = np.asarray(T0, np.float64)
        if self.pert and seed.kind in (POSE0, POSE, POSE_TRACKED):  # frame 0: start = tracked = T_0
            self.T = se3.perturb_pose(T0, seed.index, seed.delta)
        else:
            self.T = T0.astype(dt)
        self.k = 0
        self.model = None
        self.decisions = []  # every discrete branch taken, for mask-identity checks
        self.T_pp = self.T   # T_{k-2} of the constant-velocity start
        self.feat_prev = None
        self.stats = dict(iterations=0, judged=0, accepted=0)

    def measure(self, depth):
        D = np.asarray(depth, np.float64)
        if self.pert and self.seed.kind == DEPTH:
            pert = np.zeros(D.shape, type(self.seed.delta))
            if self.seed.index < 0:
                pert[:] = self.seed.delta
            else:
                pert.reshape(-1)[self.seed.index] = self.seed.delta
            D = np.where(D > 0, D + pert, 0)
        D = measure.range_gate(D, self.cfg.depth_min, self.cfg.depth_max)
        if self.cfg.bilateral:
            D = measure.bilateral(D)
        return measure.pyramid(D, len(self.cfg.icp_iters), self.cfg.pyr_range)

    @property
    def per_frame(self):
        return self.pert and self.seed.kind in PER_FRAME

    def restart_lane(self):
        """A per-frame pose lane starts frame k from the real state: the imaginary parts that frame
        k-1's perturbation left in the pose, the TSDF and the model maps are dropped."""
        dt = self.T.dtype
        self.T = np.real(self.T).astype(dt)
        self.T_pp = np.real(self.T_pp).astype(dt)
        self.F = np.real(self.F).astype(self.F.dtype)
        self.model = {k: np.real(v) for k, v in self.model.items()}

    def perturb(self, T):
        """exp(h i e_index) T for the per-frame pose kinds (the identity for every other run)."""
        if not self.per_frame:
            return T
        return se3.perturb_pose(np.real(T), self.seed.index, self.seed.delta)

    def frame(self, depth):
        c = self.cfg
        pyr = self.measure(depth)
        ok = True
        if self.k > 0 and self.per_frame:
            self.restart_lane()
        if self.k > 0:
            gates = dict(dist_gate=c.dist_gate, normal_gate_deg=c.normal_gate_deg, disc_gate=c.disc_gate)
            if c.icp_newton:
                assert not self.pert, "Newton ICP runs the real pose only"
                self.T, ok = icp.track_newton(pyr, self.intr, self.T, self.T, self.model, c.icp_iters,
                                              c.min_corr_frac, eta=c.icp_newton_eta, **gates)
            else:
                self.T, ok = self.track(pyr, depth, gates)
            if self.pert and self.seed.kind == POSE_TRACKED:
                self.T = self.perturb(self.T)
        if c.proposal is not None:
            self.feat_prev = mlp.features(np.real(np.asarray(depth, np.float64)), c.depth_min, c.depth_max)
        fusion.integrate(self.F, self.W, pyr[0], self.T, self.intr, self.dims, self.origin,
                         self.voxel, self.mu, c.disc_gate, c.w_max, log=self.decisions)
        d, V, N = raycast.raycast(self.F, self.W, self.T, self.intr, self.dims, self.origin, self.voxel,
                                  c.depth_min, c.depth_max, c.ray_step_vox, log=self.decisions)
        self.model = dict(depth=d, V=V, N=N)
        self.k += 1
        return self.T, ok


    def track(self, pyr, depth, gates):
        """ICP of frame k > 0 from the configured start; returns (T_k, ok)."""
        c = self.cfg
        T1 = self.T
        seed_a = proposal.cv_seed(T1, self.T_pp) if c.icp_seed == "cv" else T1
        if self.pert and self.seed.kind == POSE:
            seed_a = self.perturb(seed_a)
        self.T_pp = T1
        kw = dict(stop_tol=c.icp_stop, stats=self.stats, **gates)
        levels = len(c.icp_iters)
        if c.proposal is None:
            T, ok = icp.track(pyr, self.intr, seed_a, T1, self.model, c.icp_iters, c.min_corr_frac,
                              log=self.decisions, **kw)
            return T, ok
        P = c.proposal
        x = np.concatenate([self.feat_prev, mlp.features(np.real(np.asarray(depth, np.float64)), c.depth_min,
                                                          c.depth_max)])[None]
        y, _ = mlp.forward(P.params, x, bf16_ops=True)
        xi = np.asarray(P.scale, np.float64) * y[0]
        seed_b = proposal.proposal_seed(T1, xi)
        if self.pert and self.seed.kind == POSE:
            seed_b = self.perturb(seed_b)
        jl = P.judge_level
        lintr = measure.level_intrinsics(self.intr, jl)
        res = []
        for seed in (seed_a, seed_b):
            T, ok = icp.track(pyr, self.intr, seed, T1, self.model, c.icp_iters, c.min_corr_frac,
                              levels=(levels - 1, jl), **kw)
            res.append((T, ok, proposal.judge(pyr[jl], lintr, jl, T, T1, self.model, c.dist_gate)))
        (Ta, oka, Ja), (Tb, okb, Jb) = res
        accept = okb and (not oka or Jb <= Ja)
        self.stats["judged"] += 1
        self.stats["accepted"] += int(accept)
        T, ok = (Tb, okb) if accept else (Ta, oka)
        if ok and jl > 0:
            T, ok = icp.track(pyr, self.intr, T, T1, self.model, c.icp_iters, c.min_corr_frac,
                              levels=(jl - 1, 0), **kw)
        return (T, True) if ok else (T1, False)


def run(wl, seeds=(), frames=None, cfg: Config = None):
    """Run the real pipeline and one complex run per seed over ``frames`` frames of workload ``wl``.

    Returns dict: pose (F, 3, 4) real trajectory; ok (F,); per seed j: dpose[j] (F, 3, 4) = Im T / h,
    dtwist[j] (F, 6) as left twists; real_match[j] = max |Re(T*) - T| over the run."""
    cfg = cfg or Config(icp_iters=tuple(wl.icp_iters), depth_min=wl.depth_min, depth_max=wl.depth_max,
                        bilateral=wl.bilateral)
    nf = wl.depth.shape[0] if frames is None else frames
    runs = [XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, None)]
    runs += [XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, s) for s in seeds]
    pose = np.zeros((nf, 3, 4))
    ok = np.zeros(nf, bool)
    dpose = np.zeros((len(seeds), nf, 3, 4))
    dtwist = np.zeros((len(seeds), nf, 6))
    real_match = np.zeros(len(seeds))
    for k in range(nf):
        T, ok[k] = runs[0].frame(wl.depth[k])
        pose[k] = T
        for j, s in enumerate(seeds):
            Tc, _ = runs[j + 1].frame(wl.depth[k])
            _, dT, tw = se3.readout(Tc, s.h) if s.h != 0 else (None, np.zeros((3, 4)), np.zeros(6))
            dpose[j, k] = dT
            dtwist[j, k] = tw
            real_match[j] = max(real_match[j], np.abs(Tc.real - T).max())
    return dict(pose=pose, ok=ok, dpose=dpose, dtwist=dtwist, real_match=real_match, runs=runs)
