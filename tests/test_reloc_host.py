"""Host side of relocalisation (paper_2405_02187_gb300/reloc.py) without a GPU: the library's SE(3)
exponential (xslam_se3_exp_compose, host code) against the matrix exponential, and the optimiser's control
flow on a fake handle whose loss is a known quadratic in the left twist."""
import numpy as np
import pytest
import scipy.linalg

from paper_2405_02187_gb300 import reloc, xslam


def _twist_matrix(xi):
    M = np.zeros((4, 4))
    w = xi[:3]
    M[:3, :3] = [[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]]
    M[:3, 3] = xi[3:]
    return M


def test_se3_exp_is_the_matrix_exponential():
    rng = np.random.default_rng(0)
    # both branches of the coefficient series (theta^2 < 1e-2, < 1/4) and the closed form
    for scale in (1e-9, 1e-3, 0.04, 0.2, 0.3, 2.0):
        xi = rng.standard_normal(6) * scale
        assert np.allclose(reloc.se3_exp(xi), scipy.linalg.expm(_twist_matrix(xi))[:3], atol=1e-12, rtol=1e-10)


def test_se3_exp_compose_composes_and_checks_arguments():
    rng = np.random.default_rng(1)
    xi, T = rng.standard_normal(6) * 0.5, reloc.se3_exp(rng.standard_normal(6))
    want = scipy.linalg.expm(_twist_matrix(xi)) @ np.vstack([T, [0, 0, 0, 1]])
    assert np.allclose(xslam.se3_exp_compose(xi, T), want[:3], atol=1e-12)
    with pytest.raises(xslam.XSlamError):
        xslam.se3_exp_compose(np.array([np.nan, 0, 0, 0, 0, 0]), T)


class _Quadratic:
    """E(T) = 1/2 d^T A d with d the left twist taking T* to T (a log of T T*^-1, to first order)."""

    def __init__(self, A, T_star):
        self.A, self.T_star, self.calls = A, T_star, 0

    def _d(self, T):
        dR = T[:, :3] @ self.T_star[:, :3].T
        w = 0.5 * np.array([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]])
        t = T[:, 3] - dR @ self.T_star[:, 3]
        return np.concatenate([w, t])

    def grad(self, depth, T, order=1):
        self.calls += 1
        d = self._d(np.asarray(T))
        E = 0.5 * d @ self.A @ d
        g = self.A @ d
        return (E, g, self.A.copy()) if order == 2 else (E, g)


def test_newton_converges_faster_than_gradient_descent():
    rng = np.random.default_rng(1)
    Q = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    A = Q @ np.diag([1e-2, 3e-2, 0.1, 0.5, 1.0, 2.0]) @ Q.T  # condition number 200
    T_star = reloc.se3_exp(rng.standard_normal(6) * 0.3)
    T0 = reloc.compose(reloc.se3_exp(np.array([0.03, -0.02, 0.01, 0.05, -0.04, 0.02])), T_star)
    f = _Quadratic(A, T_star)
    rn = reloc.relocalise(f, None, T0, method="newton", eta=1.0, iters=30)
    rg = reloc.relocalise(_Quadratic(A, T_star), None, T0, method="gd", iters=30)
    en = reloc.pose_error(rn.T, T_star)
    eg = reloc.pose_error(rg.T, T_star)
    assert rn.newton_steps >= 1 and en[0] < 1e-6 and en[1] < 1e-4
    assert eg[0] > 10 * en[0] and rg.loss > rn.loss
    # above eta the Newton method takes gradient steps only
    r = reloc.relocalise(_Quadratic(A, T_star), None, T0, method="newton", eta=0.0, iters=5)
    assert r.newton_steps == 0


def test_conjugate_gradients_beat_gradient_descent_and_newton_beats_both():
    """The ordering of Sec. 6's ICP optimiser comparison on an ill-conditioned quadratic: after the same
    number of iterations Newton is exact, nonlinear CG is far closer than gradient descent."""
    rng = np.random.default_rng(2)
    Q = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    A = Q @ np.diag([1e-2, 3e-2, 0.1, 0.5, 1.0, 2.0]) @ Q.T
    T_star = reloc.se3_exp(rng.standard_normal(6) * 0.3)
    T0 = reloc.compose(reloc.se3_exp(np.array([0.03, -0.02, 0.01, 0.05, -0.04, 0.02])), T_star)
    err = {}
    traces = {}
    for m in ("gd", "nlcg", "newton"):
        tr = []
        r = reloc.relocalise(_Quadratic(A, T_star), None, T0, method=m, eta=np.inf, iters=30, trace=tr)
        err[m] = np.linalg.norm(_Quadratic(A, T_star)._d(r.T))
        traces[m] = tr
        assert len(tr) == r.iterations or len(tr) == r.iterations - 1
        # every accepted iteration lowers the loss
        losses = [e for _, e in tr]
        assert all(b <= a + 1e-15 for a, b in zip(losses, losses[1:]))
    assert err["newton"] < 1e-6
    assert err["nlcg"] < 0.1 * err["gd"]


class _TsdfOnly(_Quadratic):
    """The same quadratic served only through the TSDF-loss call (E, g, H or None, voxel count)."""

    def grad(self, depth, T, order=1):
        raise AssertionError("the point-to-plane loss was called")

    def grad_tsdf(self, depth, T, order=2):
        E, g, H = _Quadratic.grad(self, depth, T, order=2)
        return E, g, (H if order == 2 else None), 1000


def test_the_tsdf_loss_routes_through_grad_tsdf():
    rng = np.random.default_rng(3)
    A = np.diag([0.5, 1.0, 2.0, 1.0, 0.7, 1.5])
    T_star = reloc.se3_exp(rng.standard_normal(6) * 0.3)
    T0 = reloc.compose(reloc.se3_exp(np.array([0.02, -0.01, 0.01, 0.03, -0.02, 0.01])), T_star)
    for m in ("gd", "nlcg", "newton"):
        r = reloc.relocalise(_TsdfOnly(A, T_star), None, T0, method=m, eta=np.inf, iters=30, loss="tsdf")
        assert reloc.pose_error(r.T, T_star)[0] < 1e-3
    try:
        reloc.relocalise(_TsdfOnly(A, T_star), None, T0, loss="sdf")
    except ValueError:
        pass
    else:
        raise AssertionError("an unknown loss name was accepted")
