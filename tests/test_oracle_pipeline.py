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


def _cfg(w):
    return P.Config(icp_iters=tuple(w.icp_iters), depth_min=w.depth_min, depth_max=w.depth_max)


def _run_one(w, seed):
    r = P.XKinectFusion(w.dims, w.voxel, w.trunc, w.origin, w.intr, w.poses[0], _cfg(w), seed)
    oks = [r.frame(w.depth[k])[1] for k in range(FRAMES)]
    return r, oks


def test_real_part_equals_uncomplexified(wl):
    out = P.run(wl, [P.Seed(P.POSE0, j) for j in (0, 4)] + [P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)])
    assert out["ok"].all()
    assert out["real_match"].max() < 1e-12
    # the ground-truth trajectory is followed to within the voxel discretisation
    assert np.abs(out["pose"][:, :, 3] - wl.poses[:, :, 3]).max() < 0.01


def test_zero_step_gives_zero_imaginary(wl):
    for s in (P.Seed(P.POSE0, 1, h=0.0), P.Seed(P.TRUNC, h=0.0), P.Seed(P.DEPTH, -1, h=0.0)):
        r, _ = _run_one(wl, s)
        assert np.all(r.T.imag == 0) and np.all(r.F.imag == 0)
        assert np.all(r.model["V"].imag == 0) and np.all(r.model["N"].imag == 0)


def test_derivative_independent_of_h(wl):
    ref = None
    for h in (1e-20, 1e-30, 1e-100):
        r, _ = _run_one(wl, P.Seed(P.POSE0, 3, h=h))
        d = np.concatenate([r.T.imag.ravel(), r.F.imag]) / h
        if ref is None:
            ref = d
        else:
            assert np.abs(d - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [P.Seed(P.POSE0, j) for j in range(6)] + [P.Seed(P.DEPTH, -1)],
                         ids=[f"pose0_{j}" for j in range(6)] + ["depth_all"])
def test_csfd_matches_central_fd(wl, seed):
    """Eq. csfd vs (f(x+h) - f(x-h)) / 2h with h = 1e-8 on the final pose, the TSDF and the model
    vertex map, after asserting that every branch taken (masks, pixel and voxel cells) is identical in
    the three runs, so that no kink of the piecewise-smooth pipeline lies between -h and +h."""
    hfd = 1e-8
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
