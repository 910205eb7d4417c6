"""End-to-end pins of the oracle's complex-step pipeline (X-SLAM Sec. 3 and 4.1).

On the 24^3 / 40x30 corner workload: the real part of every complex run equals the uncomplexified
run; h = 0 gives identically zero imaginary parts; Im/h does not depend on h; CSFD derivatives agree
with central finite differences of the real pipeline (with every discrete decision identical at
+-h_fd); a left twist of the first pose moves the final pose rigidly (gauge invariance)."""
import numpy as np
import pytest

from oracle import pipeline as P
from paper_2405_02187_gb300 import synth

FRAMES = 3


@pytest.fixture(scope="module")
def wl():
    return synth.tiny(frames=FRAMES)


def _cfg(w, iters=None):
    return P.Config(icp_iters=tuple(iters or w.icp_iters), depth_min=w.depth_min, depth_max=w.depth_max)


# ICP converges fully on these noise-free frames with its 10/5 iterations, so the derivative with
# respect to ICP's start is zero up to rounding; with one iteration per level it is not
SHORT_ICP = (1, 1)


def _run_one(w, seed, iters=None):
    r = P.XKinectFusion(w.dims, w.voxel, w.trunc, w.origin, w.intr, w.poses[0], _cfg(w, iters), seed)
    oks = [r.frame(w.depth[k])[1] for k in range(FRAMES)]
    return r, oks


PIX = 15 * 40 + 20  # an interior pixel of the 40x30 frames, valid in every frame


def test_real_part_equals_uncomplexified(wl):
    out = P.run(wl, [P.Seed(P.POSE0, j) for j in (0, 4)] + [P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)] +
                [P.Seed(P.POSE, 2), P.Seed(P.POSE_TRACKED, 5), P.Seed(P.DEPTH, PIX)])
    assert out["ok"].all()
    assert out["real_match"].max() < 1e-12
    # the ground-truth trajectory is followed to within the voxel discretisation
    assert np.abs(out["pose"][:, :, 3] - wl.poses[:, :, 3]).max() < 0.01


def test_zero_step_gives_zero_imaginary(wl):
    for s in (P.Seed(P.POSE0, 1, h=0.0), P.Seed(P.TRUNC, h=0.0), P.Seed(P.DEPTH, -1, h=0.0),
              P.Seed(P.POSE, 1, h=0.0), P.Seed(P.POSE_TRACKED, 4, h=0.0), P.Seed(P.DEPTH, PIX, h=0.0)):
        r, _ = _run_one(wl, s)
        assert np.all(r.T.imag == 0) and np.all(r.F.imag == 0)
        assert np.all(r.model["V"].imag == 0) and np.all(r.model["N"].imag == 0)


@pytest.mark.parametrize("kind,index", [(P.POSE0, 3), (P.POSE, 3), (P.POSE_TRACKED, 3), (P.DEPTH, PIX)])
def test_derivative_independent_of_h(wl, kind, index):
    ref = None
    for h in (1e-20, 1e-30, 1e-100):
        r, _ = _run_one(wl, P.Seed(kind, index, h=h), SHORT_ICP if kind == P.POSE else None)
        d = np.concatenate([r.T.imag.ravel(), r.F.imag]) / h
        if ref is None:
            ref = d
        else:
            assert np.abs(d - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [P.Seed(P.POSE0, j) for j in range(6)] + [P.Seed(P.DEPTH, -1),
                                  P.Seed(P.DEPTH, PIX), P.Seed(P.DEPTH, PIX + 41)],
                         ids=[f"pose0_{j}" for j in range(6)] + ["depth_all", "depth_pixel", "depth_pixel2"])
def test_csfd_matches_central_fd(wl, seed):
    """Eq. csfd vs (f(x+h) - f(x-h)) / 2h with h = 1e-8 on the final pose, the TSDF and the model
    vertex map, after asserting that every branch taken (masks, pixel and voxel cells) is identical in
    the three runs, so that no kink of the piecewise-smooth pipeline lies between -h and +h."""
    # a single pixel moves the pose by ~1e-3 per metre, near the rounding floor of a 1e-8 difference
    # taken through 15 ICP solves; a 1e-6 step keeps the O(h^2) term far below the tolerance
    hfd = 1e-6 if seed.kind == P.DEPTH and seed.index >= 0 else 1e-8
    rc, okc = _run_one(wl, seed)
    rp, okp = _run_one(wl, P.Seed(seed.kind, seed.index, hfd, imag=False))
    rm, okm = _run_one(wl, P.Seed(seed.kind, seed.index, -hfd, imag=False))
    assert all(okc) and all(okp) and all(okm)
    assert len(rc.decisions) == len(rp.decisions) == len(rm.decisions)
    for a, b, c in zip(rc.decisions, rp.decisions, rm.decisions):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    for get in (lambda r: r.T, lambda r: r.F, lambda r: r.model["V"]):
        cs = np.imag(get(rc)) / seed.h
        fd = (get(rp) - get(rm)) / (2 * hfd)
        scale = max(np.abs(cs).max(), 1e-3)
        assert np.abs(cs - fd).max() <= 1e-6 * scale


def test_trunc_derivative_fd(wl):
    """d/dmu: the structurally small pose derivative is compared with an absolute tolerance."""
    hfd = 1e-8
    rc, _ = _run_one(wl, P.Seed(P.TRUNC))
    rp, _ = _run_one(wl, P.Seed(P.TRUNC, 0, hfd, imag=False))
    rm, _ = _run_one(wl, P.Seed(P.TRUNC, 0, -hfd, imag=False))
    for a, b, c in zip(rc.decisions, rp.decisions, rm.decisions):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    cs = rc.T.imag / 1e-20
    fd = (rp.T - rm.T) / (2 * hfd)
    assert np.abs(cs - fd).max() < 1e-6
    csF = rc.F.imag / 1e-20
    fdF = (rp.F - rm.F) / (2 * hfd)
    assert np.abs(csF - fdF).max() <= 1e-6 * np.abs(csF).max()


def test_gauge_invariance(wl):
    """A left twist of the first pose moves the whole trajectory rigidly: d xi_final / d xi_0 ~ I6
    (up to the volume's discretisation, which is fixed in the world)."""
    out = P.run(wl, [P.Seed(P.POSE0, j) for j in range(6)])
    M = out["dtwist"][:, -1, :]  # rows: seed direction j; columns: twist components
    assert np.abs(M - np.eye(6)).max() < 0.1


def test_relocalisation_gradient_matches_fd(wl):
    """The relocalisation loss gradient (Sec. 5.2 point-to-plane reading): CSFD vs central finite
    differences of the real loss, and a smaller loss at the true pose than at a displaced one."""
    from oracle import reloc, se3
    r, _ = _run_one(wl, None)
    D = r.measure(wl.depth[2])[0]
    args = (wl.intr, wl.dims, wl.origin, wl.voxel)
    T = se3.compose(se3.se3_exp(np.array([0.004, -0.003, 0.002, 0.003, 0.002, -0.002])), wl.poses[2])
    E, g, n = reloc.gradient(r.F, r.W, T, D, *args)
    assert n > 200
    hfd = 1e-7
    for j in range(6):
        e = np.zeros(6)
        e[j] = hfd
        Ep, _ = reloc.loss(r.F, r.W, se3.compose(se3.se3_exp(e), T), D, *args)
        Em, _ = reloc.loss(r.F, r.W, se3.compose(se3.se3_exp(-e), T), D, *args)
        assert abs((Ep - Em) / (2 * hfd) - g[j]) <= 1e-4 * np.abs(g).max() + 1e-12
    E_true, _ = reloc.loss(r.F, r.W, wl.poses[2], D, *args)
    assert E_true < E


# ---------------------------------------------------------------------------------------------
# per-frame pose seeds: frame k's own pose, restarted at every frame
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,j", [(P.POSE, 0), (P.POSE, 4), (P.POSE_TRACKED, 1), (P.POSE_TRACKED, 3),
                                    (P.POSE_TRACKED, 5)])
def test_per_frame_pose_matches_central_fd(wl, kind, j):
    """At every frame k >= 1 the lane's Im / h equals central differences of frame k alone: the real
    pipeline is run to frame k - 1, copied, and frame k is run twice with the pose in question
    (ICP's start for POSE, the tracked pose for POSE_TRACKED) moved by exp(+-delta e_j); every
    decision of the three runs is asserted identical. This pins that earlier frames' perturbations do
    not leak into frame k, and where the perturbation enters."""
    import copy
    # ICP shrinks a start perturbation to ~1e-3 after one iteration per level: a 1e-6 step keeps the
    # difference above its rounding floor
    hfd = 1e-6 if kind == P.POSE else 1e-8
    cfg = _cfg(wl, SHORT_ICP if kind == P.POSE else None)
    rc = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, P.Seed(kind, j))
    rr = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0], cfg, None)
    for k in range(FRAMES):
        side = []
        for sgn in (1, -1):
            r = copy.deepcopy(rr)
            r.seed, r.pert, r.cplx = P.Seed(kind, j, sgn * hfd, imag=False), True, False
            if k == 0:
                r.T = P.se3.perturb_pose(wl.poses[0], j, sgn * hfd)
            assert r.frame(wl.depth[k])[1]
            side.append(r)
        assert rc.frame(wl.depth[k])[1] and rr.frame(wl.depth[k])[1]
        rp, rm = side
        for a, b, c in zip(rc.decisions, rp.decisions, rm.decisions):
            assert np.array_equal(a, b) and np.array_equal(a, c)
        assert len(rc.decisions) == len(rp.decisions) == len(rm.decisions)
        for get in (lambda r: r.T, lambda r: r.F, lambda r: r.model["V"], lambda r: r.model["N"]):
            cs = np.imag(get(rc)) / 1e-20
            fd = (get(rp) - get(rm)) / (2 * hfd)
            scale = max(np.abs(cs).max(), 1e-3)
            assert np.abs(cs - fd).max() <= 1e-6 * scale, k
        assert np.abs(rc.T.real - rr.T).max() < 1e-12


def test_tracked_pose_lane_closed_form(wl):
    """POSE_TRACKED: Im T_k* / h = G_j T_k exactly at every frame (the read-out's left twist is e_j),
    and the derivative of the fused TSDF is nonzero. POSE (ICP's start): Gauss-Newton contracts the
    start's error at every iteration, so d T_k / d xi_start shrinks with the iteration count: below
    the unit response after one iteration per level, and at rounding level after 10 and 5."""
    out = P.run(wl, [P.Seed(P.POSE_TRACKED, j) for j in range(6)])
    assert out["ok"].all()
    for j in range(6):
        assert np.abs(out["dtwist"][j] - np.eye(6)[j]).max() < 1e-12
        assert np.abs(out["runs"][1 + j].F.imag).max() > 0
    seeds = [P.Seed(P.POSE, j) for j in range(6)]
    short = P.run(wl, seeds, cfg=_cfg(wl, SHORT_ICP))
    full = P.run(wl, seeds, cfg=_cfg(wl))
    assert short["ok"].all() and full["ok"].all()
    # frame 0 has no ICP: its start is its tracked pose
    assert np.abs(short["dtwist"][:, 0] - np.eye(6)).max() < 1e-12
    s1 = np.abs(short["dtwist"][:, 1:]).max()
    assert 1e-4 < s1 < 0.9
    assert np.abs(full["dtwist"][:, 1:]).max() < 1e-6
