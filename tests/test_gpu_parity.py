"""CUDA path vs the CPU oracle, stage by stage and end to end (X-SLAM Sec. 4.1), through the C ABI.

Tolerances (FP32 lanes against the complex128 oracle): TSDF real part 1e-4 absolute where both
sides observed the voxel with the same weight; pose 1e-5 m/rad; derivatives 1e-3 relative: a lane of
a volume or a map passes if at least 99.9% of its elements lie within 1e-3 of the lane's scale (max
|oracle|), none is further than the scale, and the Frobenius relative error is below 1e-3; the 27
normal-equation sums and the 6-component twist blocks by their Frobenius relative error. Discrete decisions taken in different precision may flip at knife edges
(a depth exactly at a gate, a TSDF sample at zero); their count is bounded and the values are
compared where both sides took the same branch."""
import numpy as np
import pytest

from gpu_helpers import (H_GPU, H_ORA, assert_lanes_close, gpu_seeds, make_handle, oracle_cfg, pose_lanes,
                         promote_seeds, rel_err, xslam_cfg)
from oracle import fusion, icp, measure, raycast, se3
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orbit():
    return synth.small_orbit(frames=20)


def _cuda(a):
    return torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _gated(wl, k):
    return measure.range_gate(wl.depth[k].astype(np.float64), wl.depth_min, wl.depth_max)


# ---------------------------------------------------------------------------------------------
def test_pyramid_parity(orbit):
    x = make_handle(orbit, max_lanes=0)
    d = _cuda(orbit.depth[3])
    ref = measure.pyramid(_gated(orbit, 3), 3, oracle_cfg(orbit).pyr_range)
    for l in range(3):
        out = torch.empty((orbit.intr.height >> l, orbit.intr.width >> l), device="cuda")
        x.measure(d, l, out)
        g = out.cpu().numpy().astype(np.float64)
        mg, mo = g > 0, ref[l] > 0
        assert (mg != mo).mean() < 1e-3
        both = mg & mo
        assert np.abs(g[both] - ref[l][both]).max() < 2e-6 * ref[l][both].max()
        if l == 0:
            assert np.array_equal(g, ref[0])


# ---------------------------------------------------------------------------------------------
SEEDS_F = [P.Seed(P.POSE0, 0), P.Seed(P.POSE0, 4), P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)]


def _oracle_fuse(wl, seeds, frames, poses):
    n = int(np.prod(wl.dims))
    F = np.ones(n)
    W = np.zeros(n)
    Fc = [np.ones(n, complex) for _ in seeds]
    Wc = [np.zeros(n) for _ in seeds]
    for k, T in zip(frames, poses):
        D = _gated(wl, k)
        fusion.integrate(F, W, D, T, wl.intr, wl.dims, wl.origin, wl.voxel, wl.trunc)
        for j, (s, Tc) in enumerate(zip(seeds, promote_seeds(T, seeds))):
            mu = wl.trunc + (1j * H_ORA if s.kind == P.TRUNC else 0)
            Dc = np.where(D > 0, D + 1j * H_ORA, 0) if s.kind == P.DEPTH else D
            fusion.integrate(Fc[j], Wc[j], Dc, Tc, wl.intr, wl.dims, wl.origin, wl.voxel, mu)
    return F, W, Fc


def test_fusion_parity(orbit):
    x = make_handle(orbit, max_lanes=6)
    x.set_lanes(gpu_seeds(SEEDS_F))
    frames = [0, 5, 10]
    poses = [orbit.poses[k] for k in frames]
    for k, T in zip(frames, poses):
        x.set_pose_lanes(pose_lanes(T, promote_seeds(T, SEEDS_F)))
        x.integrate(_cuda(orbit.depth[k]))
    F, W, Fc = _oracle_fuse(orbit, SEEDS_F, frames, poses)
    n = x.n_vox
    buf = torch.empty(n, device="cuda")
    gW = x.read_tsdf(-1, buf).cpu().numpy().astype(np.float64)
    gF = x.read_tsdf(0, buf).cpu().numpy().astype(np.float64)
    agree = gW == W
    assert (~agree).mean() < 1e-3
    obs = agree & (W > 0)
    assert obs.sum() > 10000
    assert np.abs(gF[obs] - F[obs]).max() < 1e-4
    for j in range(len(SEEDS_F)):
        gd = x.read_tsdf(j + 1, buf).cpu().numpy().astype(np.float64)
        od = Fc[j].imag / H_ORA
        assert_lanes_close(gd[obs], od[obs], what=f"TSDF lane {j}")
        assert np.all(gd[~(W > 0) & agree] == 0)


# ---------------------------------------------------------------------------------------------
SEEDS_R = [P.Seed(P.POSE0, 1), P.Seed(P.POSE0, 5), P.Seed(P.TRUNC)]


def _planes_to_maps(lanes_V):
    """[(H, W, 3) per lane] -> (L*3, H, W) float32 planes."""
    return np.concatenate([np.moveaxis(v, -1, 0) for v in lanes_V], 0).astype(np.float32)


def test_raycast_parity(orbit):
    frames = [0, 3, 6]
    poses = [orbit.poses[k] for k in frames]
    F, W, Fc = _oracle_fuse(orbit, SEEDS_R, frames, poses)
    F32 = F.astype(np.float32).astype(np.float64)
    lanes32 = [(Fc[j].imag / H_ORA * H_GPU).astype(np.float32) for j in range(len(SEEDS_R))]
    x = make_handle(orbit, max_lanes=6)
    x.set_lanes(gpu_seeds(SEEDS_R))
    x.write_tsdf(0, _cuda(F32))
    x.write_tsdf(-1, _cuda(W))
    for j, l32 in enumerate(lanes32):
        x.write_tsdf(j + 1, _cuda(l32))
    T = se3.compose(se3.se3_exp(np.array([0.01, -0.02, 0.005, 0.01, 0.0, -0.01])), orbit.poses[4])
    Tcs = promote_seeds(T, SEEDS_R)
    H, Wd = orbit.intr.height, orbit.intr.width
    L = 1 + len(SEEDS_R)
    dep = torch.empty((H, Wd), device="cuda")
    vm = torch.empty((3 * L, H, Wd), device="cuda")
    nm = torch.empty((3 * L, H, Wd), device="cuda")
    x.raycast(pose_lanes(T, Tcs), dep, vm, nm)
    gd, gv, gn = dep.cpu().numpy(), vm.cpu().numpy().astype(np.float64), nm.cpu().numpy().astype(np.float64)
    args = (orbit.intr, orbit.dims, orbit.origin, orbit.voxel, orbit.depth_min, orbit.depth_max)
    od, oV, oN = raycast.raycast(F32, W, T, *args)
    mg, mo = gd > 0, od > 0
    assert mo.mean() > 0.2
    assert (mg != mo).mean() < 5e-3
    both = mg & mo
    assert np.abs(gd[both] - od[both]).max() < 1e-4
    assert np.abs(np.moveaxis(gv[:3], 0, -1)[both] - oV[both]).max() < 1e-4
    assert np.abs(np.moveaxis(gn[:3], 0, -1)[both] - oN[both]).max() < 2e-3
    for j, s in enumerate(SEEDS_R):
        Fcj = F32 + 1j * (lanes32[j].astype(np.float64) / H_GPU * H_ORA)
        _, cV, cN = raycast.raycast(Fcj, W, Tcs[j], *args)
        gvl = np.moveaxis(gv[3 * (j + 1):3 * (j + 2)], 0, -1)[both] / H_GPU
        gnl = np.moveaxis(gn[3 * (j + 1):3 * (j + 2)], 0, -1)[both] / H_GPU
        assert_lanes_close(gvl, cV.imag[both] / H_ORA, what=f"vertex lane {j}")
        assert_lanes_close(gnl, cN.imag[both] / H_ORA, what=f"normal lane {j}")


# ---------------------------------------------------------------------------------------------
def test_icp_system_parity(orbit):
    seeds = [P.Seed(P.POSE0, 2), P.Seed(P.POSE0, 3), P.Seed(P.DEPTH, -1)]
    frames = [0, 1, 2]
    poses = [orbit.poses[k] for k in frames]
    F, W, _ = _oracle_fuse(orbit, [], frames, poses)
    Tprev = orbit.poses[2]
    Tprev_c = promote_seeds(Tprev, seeds)
    od, oV, oN = raycast.raycast(F, W, Tprev, orbit.intr, orbit.dims, orbit.origin, orbit.voxel,
                                 orbit.depth_min, orbit.depth_max)
    models = []
    for Tc in Tprev_c:
        _, cV, cN = raycast.raycast(F.astype(complex), W, Tc, orbit.intr, orbit.dims, orbit.origin, orbit.voxel,
                                    orbit.depth_min, orbit.depth_max)
        models.append((cV, cN))
    # the GPU gets the float32-rounded model
    vm = _planes_to_maps([oV] + [m[0].imag / H_ORA * H_GPU for m in models])
    nm = _planes_to_maps([oN] + [m[1].imag / H_ORA * H_GPU for m in models])
    od32 = od.astype(np.float32).astype(np.float64)
    oV32 = vm[:3].astype(np.float64)
    oN32 = nm[:3].astype(np.float64)
    x = make_handle(orbit, max_lanes=6)
    x.set_lanes(gpu_seeds(seeds))
    x.set_model(_cuda(od32), _cuda(vm), _cuda(nm), pose_lanes(Tprev, Tprev_c))
    x.measure(_cuda(orbit.depth[3]), 0, None)
    Tj = se3.compose(se3.se3_exp(np.array([0.004, -0.003, 0.002, 0.006, -0.004, 0.003])), orbit.poses[3])
    Tj_c = promote_seeds(Tj, seeds)
    pyr = measure.pyramid(_gated(orbit, 3), 3, oracle_cfg(orbit).pyr_range)
    iu = np.triu_indices(6)
    for level in (2, 1, 0):
        g, nv = x.icp_system(level, pose_lanes(Tj, Tj_c))
        li = measure.level_intrinsics(orbit.intr, level)
        model = dict(depth=od32, V=np.moveaxis(oV32, 0, -1), N=np.moveaxis(oN32, 0, -1))
        r, J, valid = icp.correspondences(pyr[level], li, level, Tj, Tprev, model)
        A, b, n = icp.normal_equations(r, J, valid)
        assert abs(nv - n) <= max(2, 2e-3 * n), (level, nv, n)
        ref = np.concatenate([A[iu], -b])
        assert rel_err(g[0], ref) < 2e-4, level
        for j, s in enumerate(seeds):
            mV = np.moveaxis(oV32, 0, -1) + 1j * np.moveaxis(vm[3 * (j + 1):3 * (j + 2)].astype(np.float64), 0, -1) / H_GPU * H_ORA
            mN = np.moveaxis(oN32, 0, -1) + 1j * np.moveaxis(nm[3 * (j + 1):3 * (j + 2)].astype(np.float64), 0, -1) / H_GPU * H_ORA
            Dl = pyr[level] if s.kind != P.DEPTH else np.where(pyr[level] > 0, pyr[level] + 1j * H_ORA, 0)
            rc, Jc, vc = icp.correspondences(Dl, li, level, Tj_c[j], Tprev_c[j], dict(depth=od32, V=mV, N=mN))
            Ac, bc, _ = icp.normal_equations(rc, Jc, vc)
            refj = np.concatenate([Ac[iu], -bc]).imag / H_ORA
            assert rel_err(g[j + 1] / H_GPU, refj) < 1e-3, (level, j)


# ---------------------------------------------------------------------------------------------
def _gpu_sequence(wl, seeds, frames, **kw):
    x = make_handle(wl, max_lanes=max(1, len(seeds)))
    x.set_pose(wl.poses[0])
    out = []
    for k in range(frames):
        pose, dpose, dtw, st = x.frame(_cuda(wl.depth[k]), gpu_seeds(seeds))
        out.append((pose, dpose, dtw, st))
    return x, out


def test_sequence_parity_small(orbit):
    """64^3, 160x120, 20 frames: tracked poses and their derivatives against the oracle."""
    seeds = [P.Seed(P.POSE0, 0), P.Seed(P.POSE0, 4), P.Seed(P.TRUNC)]
    nf = 20
    _, g = _gpu_sequence(orbit, seeds, nf)
    ref = P.run(orbit, seeds, frames=nf)
    assert ref["ok"].all()
    for k in range(nf):
        pose, dpose, dtw, st = g[k]
        assert st == xslam.OK
        assert np.abs(pose - ref["pose"][k]).max() < 1e-5, k
        for j in (0, 1):
            assert rel_err(dtw[j], ref["dtwist"][j, k]) < 1e-3, (k, j)
        assert np.abs(dtw[2] - ref["dtwist"][2, k]).max() < 1e-3, k


def test_empty_frame_does_not_track(orbit):
    x = make_handle(orbit, max_lanes=1)
    x.set_pose(orbit.poses[0])
    p0, _, _, st = x.frame(_cuda(orbit.depth[0]), [(P.POSE0, 0, H_GPU)])
    assert st == xslam.OK
    p1, _, _, st = x.frame(_cuda(np.zeros_like(orbit.depth[1])), [(P.POSE0, 0, H_GPU)])
    assert st == xslam.ENOTRACK
    assert np.array_equal(p1, p0)
    with pytest.raises(xslam.XSlamError):
        x.frame(_cuda(orbit.depth[2]), [(P.POSE0, 1, H_GPU)])  # seeds cannot change mid-sequence


def test_deterministic_and_graph_equals_direct(orbit, monkeypatch):
    seeds = [P.Seed(P.POSE0, 0), P.Seed(P.TRUNC)]
    _, a = _gpu_sequence(orbit, seeds, 6)
    _, b = _gpu_sequence(orbit, seeds, 6)
    monkeypatch.setenv("XSLAM_GRAPHS", "0")
    _, c = _gpu_sequence(orbit, seeds, 6)
    for ra, rb, rc in zip(a, b, c):
        for u, v, w in zip(ra[:3], rb[:3], rc[:3]):
            assert np.array_equal(u, v) and np.array_equal(u, w)
