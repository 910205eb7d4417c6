"""Pins of the ICP start poses and of the learned proposal's judge and selection in the oracle
(oracle/proposal.py, oracle/pipeline.py): a closed-form judge value on a plane, constant velocity
reproducing a constant-velocity path, the stop tolerance's iteration counts, and the selection
reducing to the method without a proposal (a network that proposes no motion is accepted and changes
nothing; one that proposes a 15 cm jump is rejected and changes nothing)."""
import numpy as np
import pytest

from oracle import icp, measure, mlp, proposal, se3
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth


def _plane_model(intr, z):
    """Model maps of the plane z = const seen from the identity pose: depth z, V = z K^-1 u, N = -e_z."""
    lin = measure.level_intrinsics(intr, 0)
    H, W = intr.height, intr.width
    D = np.full((H, W), z)
    V = measure.vertex_map(D, lin)
    N = np.zeros((H, W, 3))
    N[..., 2] = -1.0
    return dict(depth=D, V=V, N=N)


def test_judge_plane_closed_form():
    intr = synth.Intrinsics(60.0, 60.0, 39.5, 29.5, 80, 60)
    model = _plane_model(intr, 1.0)
    lin = measure.level_intrinsics(intr, 0)
    I = np.eye(4)[:3]
    g = 0.1
    for delta in (0.0, 0.01, 0.03):
        D = np.full((60, 80), 1.0 + delta)
        assert proposal.judge(D, lin, 0, I, I, model, g) == pytest.approx(delta * delta, rel=1e-9, abs=1e-18)
    # half the model missing: those pixels are charged g^2
    model["depth"][:, 40:] = 0.0
    D = np.full((60, 80), 1.02)
    assert proposal.judge(D, lin, 0, I, I, model, g) == pytest.approx((0.02 ** 2 + g * g) / 2, rel=1e-9)
    # farther than the gate: g^2
    assert proposal.judge(np.full((60, 80), 1.5), lin, 0, I, I, model, g) == pytest.approx(g * g)
    # no depth at all: g^2
    assert proposal.judge(np.zeros((60, 80)), lin, 0, I, I, model, g) == g * g


def test_judge_level_reads_level0_model_at_stride():
    intr = synth.Intrinsics(60.0, 60.0, 39.5, 29.5, 80, 60)
    model = _plane_model(intr, 1.0)
    lin1 = measure.level_intrinsics(intr, 1)
    D1 = np.full((30, 40), 1.01)
    I = np.eye(4)[:3]
    assert proposal.judge(D1, lin1, 1, I, I, model, 0.1) == pytest.approx(1e-4, rel=1e-9)


def test_polar_step_takes_a_pose_to_so3_to_second_order():
    import scipy.linalg
    rng = np.random.default_rng(4)
    T = se3.se3_exp(rng.normal(0, 0.7, 6))
    E = rng.normal(0, 1e-6, (3, 3))
    E = 0.5 * (E + E.T)  # a symmetric deviation from SO(3)
    Tb = T.copy()
    Tb[:, :3] = T[:, :3] @ (np.eye(3) + E)
    P = proposal.polar_step(Tb)
    dev = lambda R: np.abs(R.T @ R - np.eye(3)).max()  # noqa: E731
    d0 = dev(Tb[:, :3])
    assert d0 > 1e-7 and dev(P[:, :3]) < 2 * d0 ** 2 + 1e-15  # quadratic
    U, _ = scipy.linalg.polar(Tb[:, :3])  # the nearest rotation
    assert np.abs(P[:, :3] - U).max() < 2 * d0 ** 2 + 1e-15
    np.testing.assert_array_equal(P[:, 3], Tb[:, 3])
    # a tangent of SO(3) at R (R S, S skew) on a complex lane passes unchanged
    S = se3.hat(rng.normal(0, 1, 3))
    Tc = T.astype(np.complex128)
    Tc[:, :3] += 1j * 1e-20 * (T[:, :3] @ S)
    Pc = proposal.polar_step(Tc)
    np.testing.assert_allclose(Pc.imag[:, :3], 1e-20 * (T[:, :3] @ S), rtol=0, atol=1e-33)


def test_cv_seed_keeps_the_deviation_from_so3_bounded():
    """Without the polar step, T_1 T_2^-1 T_1 multiplies a deviation from SO(3) by about 1 + sqrt(2)
    per frame (e_k = 2 e_{k-1} + e_{k-2}); with it the deviation stays at rounding level."""
    rng = np.random.default_rng(5)
    xi = np.array([0.01, -0.02, 0.015, 0.02, 0.01, -0.01])
    dev = lambda T: np.abs(T[:, :3].T @ T[:, :3] - np.eye(3)).max()  # noqa: E731

    def drift(T):  # what FP32 increments leave: a deviation of 1e-9
        E = rng.normal(0, 1e-9, (3, 3))
        T = T.copy()
        T[:, :3] = T[:, :3] @ (np.eye(3) + 0.5 * (E + E.T))
        return T

    for seed_fn in (proposal.cv_seed, lambda T1, T2: se3.compose(T1, se3.compose(se3.inverse(T2), T1))):
        T2 = se3.se3_exp(rng.normal(0, 0.5, 6))
        T1 = drift(se3.compose(T2, se3.se3_exp(xi)))
        worst = 0.0
        for _ in range(30):
            T1, T2 = drift(seed_fn(T1, T2)), T1
            worst = max(worst, dev(T1))
        if seed_fn is proposal.cv_seed:
            assert worst < 1e-8
        else:
            assert worst > 1e-3  # the plain extrapolation: 2.4^30 * 1e-9


def test_cv_seed_repeats_camera_frame_motion():
    rng = np.random.default_rng(1)
    T0 = se3.se3_exp(rng.normal(0, 0.7, 6))
    xi = np.array([0.02, -0.01, 0.015, 0.03, -0.02, 0.01])
    T1 = se3.compose(T0, se3.se3_exp(xi))
    np.testing.assert_allclose(proposal.cv_seed(T1, T0), se3.compose(T0, se3.se3_exp(2 * xi)), atol=1e-14)
    np.testing.assert_allclose(proposal.cv_seed(T0, T0), T0, atol=1e-15)
    np.testing.assert_allclose(proposal.proposal_seed(T0, xi), T1, atol=1e-15)


@pytest.fixture(scope="module")
def wl():
    return synth.tiny(frames=3, width=80, height=60)


def test_stop_tolerance_iteration_counts(wl):
    r = P.XKinectFusion(wl.dims, wl.voxel, wl.trunc, wl.origin, wl.intr, wl.poses[0],
                        P.Config(icp_iters=tuple(wl.icp_iters), depth_min=wl.depth_min, depth_max=wl.depth_max))
    r.frame(wl.depth[0])
    pyr = r.measure(wl.depth[1])
    for tol, expect in ((0.0, sum(wl.icp_iters)), (1e9, len(wl.icp_iters))):
        stats = {}
        T, ok = icp.track(pyr, wl.intr, r.T, r.T, r.model, wl.icp_iters, stop_tol=tol, stats=stats)
        assert ok and stats["iterations"] == expect
    # a realistic tolerance stops early, at a pose within the tolerance's reach of the full run
    stats = {}
    Tf, _ = icp.track(pyr, wl.intr, r.T, r.T, r.model, wl.icp_iters)
    Ts, _ = icp.track(pyr, wl.intr, r.T, r.T, r.model, wl.icp_iters, stop_tol=1e-6, stats=stats)
    assert stats["iterations"] < sum(wl.icp_iters)
    assert np.abs(Ts - Tf).max() < 1e-5


def _cfg(w, **kw):
    return P.Config(icp_iters=tuple(w.icp_iters), depth_min=w.depth_min, depth_max=w.depth_max, **kw)


def _run(w, cfg, frames=3):
    r = P.XKinectFusion(w.dims, w.voxel, w.trunc, w.origin, w.intr, w.poses[0], cfg, None)
    out = [r.frame(w.depth[k]) for k in range(frames)]
    return r, np.array([T for T, _ in out]), [ok for _, ok in out]


def _const_net(y, sizes=(9600, 16, 16, 16, 6)):
    params = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(sizes[:-1], sizes[1:])]
    params[-1][1][:] = y
    return params


def test_zero_motion_proposal_changes_nothing(wl):
    _, ref, ok_ref = _run(wl, _cfg(wl))
    prop = P.Proposal(_const_net(np.zeros(6)), np.ones(6), judge_level=1)
    r, got, ok = _run(wl, _cfg(wl, proposal=prop))
    # both runs start at T_{k-1}: equal judges, the proposal is accepted, nothing changes
    assert r.stats["judged"] == 2 and r.stats["accepted"] == 2
    np.testing.assert_array_equal(got, ref)
    assert all(ok) and all(ok_ref)


def test_far_proposal_is_rejected(wl):
    for seed in ("prev", "cv"):
        _, ref, _ = _run(wl, _cfg(wl, icp_seed=seed))
        prop = P.Proposal(_const_net(np.array([0.0, 0.0, 0.0, 0.15, 0.0, 0.0])), np.ones(6), judge_level=1)
        r, got, ok = _run(wl, _cfg(wl, icp_seed=seed, proposal=prop))
        assert r.stats["judged"] == 2 and r.stats["accepted"] == 0
        assert all(ok)
        np.testing.assert_array_equal(got, ref)


def test_features_of_tiny_frames_follow_range_gate(wl):
    f = mlp.features(wl.depth[0], wl.depth_min, wl.depth_max)
    assert f.shape == (4800,) and (f >= 0).all() and f.max() <= wl.depth_max / mlp.DEPTH_SCALE
    assert (f > 0).mean() > 0.9
