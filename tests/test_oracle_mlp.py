"""Pins of the learned-proposal oracle (oracle/mlp.py) against things other than itself: a library's
bfloat16 conversion, a vectorised block mean, central finite differences, a least-squares minimiser,
the closed form of Adam under a constant gradient, and scipy's matrix logarithm."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import mlp, se3


def test_bf16_known_values():
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie, even neighbour below
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie, even neighbour above
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-3.0) == -3.0
    assert mlp.bf16(0.0) == 0.0


def test_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-30, 500), rng.uniform(-1e4, 1e4, 500)])
    x32 = x.astype(np.float32)
    lib = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32), lib)


def _block_mean_vectorised(D, dmin, dmax):
    H, W = D.shape
    by, bx = H // 60, W // 80
    ok = (D >= dmin) & (D <= dmax)
    s = np.where(ok, D, 0.0).reshape(60, by, 80, bx).sum((1, 3))
    n = ok.reshape(60, by, 80, bx).sum((1, 3))
    return np.where(n > 0, s / np.maximum(n, 1), 0.0).reshape(-1) / mlp.DEPTH_SCALE


@pytest.mark.parametrize("shape", [(120, 160), (240, 320)])
def test_features_block_mean(shape):
    rng = np.random.default_rng(2)
    D = rng.uniform(0.0, 5.0, shape)
    D[rng.random(shape) < 0.3] = 0.0
    D[:shape[0] // 60, : shape[1] // 80] = 0.0          # an empty block
    f = mlp.features(D, 0.2, 4.0)
    assert f.shape == (4800,)
    assert f[0] == 0.0
    np.testing.assert_allclose(f, _block_mean_vectorised(D, 0.2, 4.0), rtol=1e-14, atol=0)


def test_features_constant_and_gate():
    D = np.full((120, 160), 2.0)
    np.testing.assert_allclose(mlp.features(D, 0.2, 4.0), 0.5)
    D[0, 0] = 5.0                                          # out of range: excluded, not averaged
    assert mlp.features(D, 0.2, 4.0)[0] == 0.5


def _tiny(rng, sizes=(7, 5, 4, 3, 2)):
    params = mlp.init_params(sizes, rng)
    params = [(W, rng.normal(0, 0.1, b.shape)) for W, b in params]
    x = rng.uniform(0, 1, (3, sizes[0]))
    t = rng.normal(0, 1, (3, sizes[-1]))
    return params, x, t


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    params, x, t = _tiny(rng)
    E, grads = mlp.gradient(params, x, t, bf16_ops=False)
    y, _ = mlp.forward(params, x, bf16_ops=False)
    assert E == pytest.approx(mlp.loss(y, t))
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + eps
                Ep = mlp.loss(mlp.forward(params, x, False)[0], t)
                arr[idx] = old - eps
                Em = mlp.loss(mlp.forward(params, x, False)[0], t)
                arr[idx] = old
                fd[idx] = (Ep - Em) / (2 * eps)
            np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_bf16_ops_reduce_to_exact_on_representable_values():
    # every value of the forward and backward pass is a small multiple of 1/4: exact in bfloat16
    rng = np.random.default_rng(4)
    sizes = (6, 5, 4, 3)
    params = [(rng.integers(-2, 3, (o, i)).astype(float), rng.integers(-2, 3, o).astype(float))
              for i, o in zip(sizes[:-1], sizes[1:])]
    x = rng.integers(0, 4, (4, sizes[0])).astype(float)
    t = rng.integers(-5, 6, (4, sizes[-1])).astype(float)
    E1, g1 = mlp.gradient(params, x, t, bf16_ops=True)
    E0, g0 = mlp.gradient(params, x, t, bf16_ops=False)
    assert E1 == E0
    for (a, b), (c, d) in zip(g1, g0):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)


def test_bf16_forward_close_to_exact():
    rng = np.random.default_rng(5)
    params = mlp.init_params((64, 32, 32, 4), rng)
    x = rng.uniform(0, 1, (8, 64))
    y1, _ = mlp.forward(params, x, True)
    y0, _ = mlp.forward(params, x, False)
    # three roundings of relative size 2^-9 per layer: a few percent of the output scale at most
    assert np.abs(y1 - y0).max() < 0.05 * np.abs(y0).max()
    assert np.abs(y1 - y0).max() > 0.0


def test_gradient_vanishes_at_least_squares_minimiser():
    rng = np.random.default_rng(6)
    B, n, m = 20, 5, 3
    x = rng.normal(0, 1, (B, n))
    t = rng.normal(0, 1, (B, m))
    X1 = np.concatenate([x, np.ones((B, 1))], 1)
    sol = np.linalg.lstsq(X1, t, rcond=None)[0]          # (n + 1, m)
    params = [(sol[:n].T.copy(), sol[n].copy())]
    E, grads = mlp.gradient(params, x, t, bf16_ops=False)
    assert np.abs(grads[0][0]).max() < 1e-12 and np.abs(grads[0][1]).max() < 1e-12
    assert E == pytest.approx(0.5 * np.sum((X1 @ sol - t) ** 2) / B, rel=1e-12)
    # and a step away from the minimiser gives the closed-form gradient direction back
    params[0][1][0] += 0.5
    _, grads = mlp.gradient(params, x, t, bf16_ops=False)
    assert grads[0][1][0] == pytest.approx(0.5, rel=1e-12)


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(7)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    m = np.zeros(50)
    v = np.zeros(50)
    p0 = p.copy()
    for step in range(1, 6):
        mlp.adam_step(p, g, m, v, step, lr=0.01)
        # with a constant gradient the bias-corrected moments are g and g^2 at every step
        np.testing.assert_allclose(p, p0 - step * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-14)


def test_se3_log_inverts_exp_and_matches_logm():
    rng = np.random.default_rng(8)
    for scale in (1e-9, 1e-3, 0.3, 2.5):
        xi = rng.normal(0, 1, 6)
        xi[:3] *= scale / np.linalg.norm(xi[:3])
        T = se3.se3_exp(xi)
        np.testing.assert_allclose(mlp.se3_log(T), xi, rtol=1e-9, atol=1e-12)
        M = np.eye(4)
        M[:3] = T
        L = scipy.linalg.logm(M).real
        ref = np.array([L[2, 1], L[0, 2], L[1, 0], L[0, 3], L[1, 3], L[2, 3]])
        np.testing.assert_allclose(mlp.se3_log(T), ref, rtol=1e-7, atol=1e-12)


def test_pair_target_is_motion_in_first_camera():
    rng = np.random.default_rng(9)
    Ti = se3.se3_exp(rng.normal(0, 0.5, 6))
    xi = np.array([0.01, -0.02, 0.005, 0.03, 0.01, -0.02])
    Tj = se3.compose(Ti, se3.se3_exp(xi))
    np.testing.assert_allclose(mlp.pair_target(Ti, Tj), xi, rtol=1e-9, atol=1e-13)
    assert math.isclose(np.abs(mlp.pair_target(Ti, Ti)).max(), 0.0, abs_tol=1e-14)


def test_reflected_motion_twist():
    """The twist of a motion seen in a mirror: T -> M T M with M = diag(-1, 1, 1) or diag(1, -1, 1)
    maps (phi, rho) to (-M phi, M rho)."""
    rng = np.random.default_rng(10)
    for M, sign in ((np.diag([-1.0, 1, 1]), [1, -1, -1, -1, 1, 1]), (np.diag([1.0, -1, 1]), [-1, 1, -1, 1, -1, 1])):
        Ti = se3.se3_exp(rng.normal(0, 0.5, 6))
        Tj = se3.compose(Ti, se3.se3_exp(rng.normal(0, 0.05, 6)))
        refl = lambda T: np.concatenate([M @ T[:, :3] @ M, (M @ T[:, 3])[:, None]], 1)  # noqa: E731
        np.testing.assert_allclose(mlp.pair_target(refl(Ti), refl(Tj)), np.array(sign) * mlp.pair_target(Ti, Tj),
                                   atol=1e-12)
