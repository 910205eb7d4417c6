"""The learned proposal's network on the GPU (include/xslam_mlp.h) against the CPU oracle
(oracle/mlp.py), through the C ABI: the tcgen05 GEMM, the forward pass, the gradient, Adam, training,
the input features and the training targets.

Tolerances, from the arithmetic. A GEMM of BF16 operands accumulates K products in FP32: its error
is at most K 2^-23 sum_k |a_k b_k| (FP32 rounding of each partial sum, allowing a truncating
accumulator). The network oracle rounds to BF16 at the points the GPU does, so the two differ by
those accumulation errors plus the rare rounding to the neighbouring BF16 value (2^-8 relative) of
an activation or gradient near a rounding midpoint; the forward output and the gradients are held
to 2^-6 relative (Frobenius norm per tensor), the features to one BF16 ulp, Adam's update to 1e-5 of
the step on the same gradient."""
import numpy as np
import pytest

from oracle import mlp as OM
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (9600, 512, 512, 512, 6)


def _bf16_dev(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda").to(torch.bfloat16)


def _host(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K,splits", [(1, 6, 64, 1), (200, 300, 192, 1), (200, 300, 192, 3), (128, 128, 64, 1),
                                          (256, 512, 9600, 16), (512, 640, 256, 1), (64, 9600, 256, 2)])
def test_gemm_matches_exact_product(M, N, K, splits):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    ws = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
    xslam.gemm_bf16(A, B, C, splits=splits, workspace=ws)
    a, b = _host(A), _host(B)
    ref = a @ b.T
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T)
    err = np.abs(_host(C) - ref)
    assert np.isfinite(err).all()
    assert (err <= bound + 1e-30).all(), err.max()
    # typical errors are far below the bound
    assert np.median(err / np.maximum(bound, 1e-30)) < 0.05


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(4, 96, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(4, 4, device="cuda")
    with pytest.raises(xslam.XSlamError):
        xslam.gemm_bf16(A, A, C)                      # K = 96 is not a multiple of 64
    A = torch.zeros(4, 128, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(xslam.XSlamError):
        xslam.gemm_bf16(A, A, C, splits=3)            # more splits than 64-wide slices


@pytest.fixture(scope="module")
def net():
    rng = np.random.default_rng(11)
    params = OM.init_params(SIZES, rng)
    params = [(W, rng.normal(0, 0.05, b.shape)) for W, b in params]
    m = xslam.Mlp(SIZES, max_batch=256)
    m.set_params(params)
    # the oracle sees the FP32 masters the GPU holds
    return m, [(np.float32(W).astype(np.float64), np.float32(b).astype(np.float64)) for W, b in params]


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("B", [1, 64, 100])
def test_forward_parity(net, B):
    m, params = net
    rng = np.random.default_rng(B)
    x = OM.bf16(rng.uniform(0, 1, (B, SIZES[0])))
    y = _host(m.forward(_bf16_dev(x)))
    ref, _ = OM.forward(params, x, bf16_ops=True)
    assert _rel(y, ref) < 2.0 ** -6
    # and against the exact network: the BF16 network is close to it, not equal
    ex, _ = OM.forward(params, x, bf16_ops=False)
    assert 0 < _rel(y, ex) < 0.05


def test_params_round_trip(net):
    m, params = net
    got = m.get_params()
    for (W, b), (Wg, bg) in zip(params, got):
        np.testing.assert_array_equal(Wg, W.astype(np.float32))
        np.testing.assert_array_equal(bg, b.astype(np.float32))


@pytest.mark.parametrize("B", [64, 192])
def test_gradient_parity(net, B):
    m, params = net
    rng = np.random.default_rng(100 + B)
    x = OM.bf16(rng.uniform(0, 1, (B, SIZES[0])))
    t = rng.normal(0, 1, (B, 6))
    loss, grads = m.gradient(_bf16_dev(x), torch.tensor(t, dtype=torch.float32, device="cuda"))
    E, ref = OM.gradient(params, x, np.float32(t).astype(np.float64), bf16_ops=True)
    assert loss == pytest.approx(E, rel=1e-4)
    for (gW, gb), (rW, rb) in zip(grads, ref):
        assert _rel(gW, rW) < 2.0 ** -6
        assert _rel(gb, rb) < 2.0 ** -6


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(21)
    sizes = (9600, 64, 6)
    params = OM.init_params(sizes, rng)
    m = xslam.Mlp(sizes, max_batch=64)
    m.set_params(params)
    p0 = [(np.float32(W).astype(np.float64), np.float32(b).astype(np.float64)) for W, b in params]
    feat = _bf16_dev(OM.bf16(rng.uniform(0, 1, (10, 4800))))
    pairs = rng.integers(0, 10, (64, 2)).astype(np.int32)
    t = rng.normal(0, 1, (64, 6)).astype(np.float32)
    # the gradient of the same batch (the training step visits its rows in another order)
    x = torch.cat([feat[torch.tensor(pairs[:, 0], device="cuda").long()],
                   feat[torch.tensor(pairs[:, 1], device="cuda").long()]], 1).contiguous()
    _, g = m.gradient(x, torch.tensor(t, device="cuda"))
    lr = 1e-3
    m.train(feat, torch.tensor(pairs, device="cuda"), torch.tensor(t, device="cuda"), epochs=1, batch=64, lr=lr)
    got = m.get_params()
    for (W0, b0), (gW, gb), (W1, b1) in zip(p0, g, got):
        for p, gr, p1 in ((W0, gW, W1), (b0, gb, b1)):
            q = p.copy()
            OM.adam_step(q, gr.astype(np.float64), np.zeros_like(q), np.zeros_like(q), 1, lr)
            # first step: -lr g / (|g| + eps); elements whose gradient is at the noise level may differ
            big = np.abs(gr) > 1e-5
            np.testing.assert_allclose(p1[big], q[big], rtol=0, atol=1e-5 * lr + 1e-7)
            assert np.abs(p1 - p).max() <= lr * 1.001


def test_training_reduces_loss_on_a_learnable_map():
    rng = np.random.default_rng(31)
    n_feat, P = 200, 2048
    feat_h = rng.uniform(0, 1, (n_feat, 4800))
    pairs = rng.integers(0, n_feat, (P, 2)).astype(np.int32)
    proj = rng.normal(0, 1, (9600, 6)) / np.sqrt(9600)
    x = np.concatenate([feat_h[pairs[:, 0]], feat_h[pairs[:, 1]]], 1)
    t = ((x - 0.5) @ proj).astype(np.float32)
    t /= t.std(0)
    m = xslam.Mlp(SIZES, max_batch=256)
    m.set_params(OM.init_params(SIZES, rng))
    losses = m.train(_bf16_dev(OM.bf16(feat_h)), torch.tensor(pairs, device="cuda"), torch.tensor(t, device="cuda"),
                     epochs=30, batch=256, lr=1e-3, seed=5)
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.2 * losses[0], losses


def test_features_parity():
    wl = synth.room_walk(frames=2, width=640, height=480, dims=64)
    d = torch.tensor(wl.depth, device="cuda")
    f = _host(xslam.features(d, wl.depth_min, wl.depth_max))
    for k in range(2):
        ref = OM.bf16(OM.features(wl.depth[k], wl.depth_min, wl.depth_max))
        ulp = np.maximum(np.abs(ref), 1e-30) * 2.0 ** -7
        assert (np.abs(f[k] - ref) <= ulp).all()
        assert (f[k] == ref).mean() > 0.99


def test_pair_targets_match_oracle():
    rng = np.random.default_rng(41)
    from oracle import se3
    poses = np.stack([se3.se3_exp(rng.normal(0, 0.6, 6)) for _ in range(8)])
    pairs = np.array([[0, 1], [2, 5], [7, 3], [4, 4]], np.int32)
    scale = np.array([0.02, 0.02, 0.02, 0.05, 0.05, 0.05], np.float32)
    got = xslam.pair_targets(poses, pairs, scale)
    for (i, j), g in zip(pairs, got):
        ref = OM.pair_target(poses[i], poses[j]) / scale.astype(np.float64)
        np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-6)
    with pytest.raises(xslam.XSlamError):
        xslam.pair_targets(poses, np.array([[0, 8]], np.int32), scale)


def _mirror_rows(x, g):
    """Both 80 x 60 halves of the rows x (n, 9600) reflected left-right (g & 1) and/or top-bottom (g & 2)."""
    v = x.reshape(-1, 2, 60, 80)
    if g & 1:
        v = v[..., ::-1]
    if g & 2:
        v = v[..., ::-1, :]
    return np.ascontiguousarray(v).reshape(x.shape)


# a reflection maps the motion twist (phi, rho) to (-M phi, M rho)
_SIGN = {0: np.ones(6), 1: np.array([1, -1, -1, -1, 1, 1.0]), 2: np.array([-1, 1, -1, 1, -1, 1.0])}
_SIGN[3] = _SIGN[1] * _SIGN[2]


def test_mirror_augmentation_is_consistent():
    """With more distinct inputs than a linear map can absorb (4800 feature rows: each half of the
    input spans its whole 4800-dimensional space), a map that commutes with the reflections
    (A P_g = S_g A) stays learnable under mirroring and a generic one does not; without mirroring
    both are. A wrong reflection of the features or of the target signs breaks the first."""
    rng = np.random.default_rng(51)
    n_feat, P = 4800, 16384
    feat = OM.bf16(rng.uniform(-1, 1, (n_feat, 4800)))  # zero mean: a well-conditioned least-squares fit
    pairs = rng.integers(0, n_feat, (P, 2)).astype(np.int32)
    A0 = rng.normal(0, 1, (6, 9600)) / np.sqrt(9600)
    # A = 1/4 sum_g S_g A0 P_g, with (A0 P_g) x = A0 (P_g x)
    A = sum(_SIGN[g][:, None] * _mirror_rows(A0, g) for g in range(4)) / 4
    x4 = np.concatenate([feat[pairs[:4, 0]], feat[pairs[:4, 1]]], 1)
    for g in range(4):
        np.testing.assert_allclose(_mirror_rows(x4, g) @ A.T, (x4 @ A.T) * _SIGN[g], atol=1e-12)
    dev_feat = _bf16_dev(feat)
    dev_pairs = torch.tensor(pairs, device="cuda")
    final = {}
    for name, M, mirror in (("equivariant", A, True), ("generic", A0, True), ("generic_plain", A0, False)):
        t = np.concatenate([feat[pairs[:, 0]], feat[pairs[:, 1]]], 1) @ M.T
        m = xslam.Mlp((9600, 6), max_batch=256)
        m.set_params([(np.zeros((6, 9600)), np.zeros(6))])
        # Adam moves every weight by about lr per step, the output by about lr sum_i |x_i| = 4800 lr:
        # lr = 1e-5 keeps that jitter near a tenth of the targets' spread (0.58)
        losses = m.train(dev_feat, dev_pairs, torch.tensor(t.astype(np.float32), device="cuda"), epochs=60,
                         batch=256, lr=1e-5, seed=3, mirror=mirror)
        final[name] = (float(losses[0]), float(losses[-1]))
        m.close()
    print(final)
    assert final["equivariant"][1] < 0.15 * final["equivariant"][0], final
    assert final["generic_plain"][1] < 0.2 * final["generic_plain"][0], final
    assert final["generic"][1] > 0.5 * final["generic"][0], final
