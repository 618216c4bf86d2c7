"""Pins for the oracle's residual CNN denoiser (the learned D of Step 4)."""
import numpy as np
import pytest

from oracle import cnn


def _tiny(seed=0, layers=3, ch=4):
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for l in range(layers):
        cin = 1 if l == 0 else ch
        cout = 1 if l == layers - 1 else ch
        ws.append(rng.standard_normal((3, 3, cin, cout)) * 0.5)
        bs.append(rng.standard_normal(cout) * 0.1)
    return ws, bs


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    ref = np.zeros((2, 5, 6, 4))
    for n in range(2):
        for y in range(5):
            for x in range(6):
                acc = b.copy()
                for ky in range(3):
                    for kx in range(3):
                        yy, xx = y + ky - 1, x + kx - 1
                        if 0 <= yy < 5 and 0 <= xx < 6:
                            acc += a[n, yy, xx] @ w[ky, kx]
                ref[n, y, x] = acc
    assert np.allclose(cnn.conv3x3(a, w, b), ref, atol=1e-12)


def test_input_gradient_is_adjoint():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((2, 7, 5, 3))
    w = rng.standard_normal((3, 3, 3, 4))
    g = rng.standard_normal((2, 7, 5, 4))
    lhs = np.sum(cnn.conv3x3(a, w, np.zeros(4)) * g)
    rhs = np.sum(a * cnn.conv3x3_input_grad(g, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_backward_matches_finite_differences():
    ws, bs = _tiny()
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 7))
    gout = rng.standard_normal((2, 6, 7))
    f, acts = cnn.net_forward(x, ws, bs)
    gws, gbs = cnn.net_backward(gout, ws, acts)
    h = 1e-6
    for l in range(len(ws)):
        for idx in [(0, 0, 0, 0), (1, 1, 0, -1), (2, 1, -1, 0)]:
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[l][idx] += h
            wm[l][idx] -= h
            num = (np.sum(cnn.net_forward(x, wp, bs)[0] * gout)
                   - np.sum(cnn.net_forward(x, wm, bs)[0] * gout)) / (2 * h)
            assert gws[l][idx] == pytest.approx(num, rel=1e-5, abs=1e-8)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        num = (np.sum(cnn.net_forward(x, ws, bp)[0] * gout) - np.sum(cnn.net_forward(x, ws, bm)[0] * gout)) / (2 * h)
        assert gbs[l][0] == pytest.approx(num, rel=1e-5, abs=1e-8)


def test_identity_network_and_residual_form():
    # centre-tap identities, zero biases: every ReLU sees a non-negative input,
    # so f(x) = x for x >= 0 and the residual denoiser returns 0
    L, C = 5, 4
    ws = []
    for l in range(L):
        cin = 1 if l == 0 else C
        cout = 1 if l == L - 1 else C
        w = np.zeros((3, 3, cin, cout))
        if l == 0:
            w[1, 1, 0, :] = 1.0
        elif l == L - 1:
            w[1, 1, :, 0] = 1.0 / C
        else:
            w[1, 1] = np.eye(C)
        ws.append(w)
    bs = [np.zeros(w.shape[3]) for w in ws]
    x = np.random.default_rng(4).uniform(0, 2, (1, 9, 8))
    f, _ = cnn.net_forward(x, ws, bs)
    assert np.allclose(f, x, atol=1e-14)
    assert np.allclose(cnn.denoise(x[0] * 3.0, 3.0, ws, bs), 0.0, atol=1e-13)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-6, 6, 10000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(v), ref)
    assert cnn.bf16_round(np.array([1 + 2 ** -8]))[0] == 1.0          # tie to even
    assert cnn.bf16_round(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6


def test_loss_of_identity_network_is_normalised_error():
    """With every weight and bias zero, f = 0 and D(r) = r: the loss is the
    noise-normalised input error, each image weighted by 1 / sigma^2."""
    ws, bs = _tiny(seed=3)
    ws = [np.zeros_like(w) for w in ws]
    bs = [np.zeros_like(b) for b in bs]
    rng = np.random.default_rng(8)
    xt = rng.standard_normal((2, 6, 6))
    sig = np.array([0.25, 4.0])
    noise = rng.choice([-1.0, 1.0], size=(2, 6, 6))
    r = xt + sig[:, None, None] * noise          # error / sigma is exactly +-1
    loss, _, _ = cnn.loss_and_grads(r, xt, sig, ws, bs)
    assert loss == pytest.approx(1.0, rel=1e-14)


def test_loss_gradient_matches_finite_differences():
    ws, bs = _tiny(seed=6)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((2, 5, 5))
    xt = rng.standard_normal((2, 5, 5))
    sig = np.array([0.5, 2.0])
    loss, gws, gbs = cnn.loss_and_grads(r, xt, sig, ws, bs)
    h = 1e-6
    wp = [w.copy() for w in ws]
    wm = [w.copy() for w in ws]
    wp[1][0, 2, 1, 3] += h
    wm[1][0, 2, 1, 3] -= h
    num = (cnn.loss_and_grads(r, xt, sig, wp, bs)[0] - cnn.loss_and_grads(r, xt, sig, wm, bs)[0]) / (2 * h)
    assert gws[1][0, 2, 1, 3] == pytest.approx(num, rel=1e-5)


def test_jvp_matches_central_differences_of_the_fp64_network():
    """J_f t from the forward-mode pass equals the central difference of the
    FP64 network: f is piecewise linear, so for a step too small to cross a
    ReLU boundary the difference quotient is exact up to rounding."""
    ws, bs = _tiny(seed=9, layers=4, ch=5)
    rng = np.random.default_rng(10)
    x = rng.standard_normal((2, 7, 6))
    t = rng.standard_normal((2, 7, 6))
    f, tf = cnn.net_jvp(x, t, ws, bs)
    f0, _ = cnn.net_forward(x, ws, bs)
    assert np.array_equal(f, f0)
    h = 1e-7
    fp, _ = cnn.net_forward(x + h * t, ws, bs)
    fm, _ = cnn.net_forward(x - h * t, ws, bs)
    assert np.allclose(tf, (fp - fm) / (2 * h), rtol=1e-6, atol=1e-8)


def test_jvp_is_linear_in_the_direction_and_denoiser_tangent_is_identity_minus_jf():
    ws, bs = _tiny(seed=12, layers=3, ch=4)
    rng = np.random.default_rng(13)
    r = rng.standard_normal((6, 6))
    b1, b2 = rng.standard_normal((2, 6, 6))
    sigma = 0.7
    _, j1 = cnn.denoise_jvp(r, b1, sigma, ws, bs)
    _, j2 = cnn.denoise_jvp(r, b2, sigma, ws, bs)
    _, j12 = cnn.denoise_jvp(r, 2.0 * b1 - 3.0 * b2, sigma, ws, bs)
    assert np.allclose(j12, 2.0 * j1 - 3.0 * j2, rtol=1e-12, atol=1e-12)
    # D = r - sigma f(r / sigma): J_D b = b - J_f(r / sigma) b
    _, tf = cnn.net_jvp((r / sigma)[None], b1[None], ws, bs)
    assert np.allclose(j1, b1 - tf[0], rtol=1e-12, atol=1e-12)
    # zero network: D(r) = r, so the tangent is b itself and D' = |b|^2 / N
    z_ws = [np.zeros_like(w) for w in ws]
    z_bs = [np.zeros_like(v) for v in bs]
    d, jb = cnn.denoise_jvp(r, b1, sigma, z_ws, z_bs)
    assert np.array_equal(d, r) and np.array_equal(jb, b1)
