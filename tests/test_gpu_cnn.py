"""GPU parity of the learned denoiser (forward, gradients, training) against the
FP64 reference in oracle/cnn.py.

The GPU stores hidden activations in BF16 and accumulates in FP32; the
reference emulates the BF16 rounding at the same points (bf16=True), so the
remaining differences come from accumulation order, which can flip a BF16
rounding now and then.  Bounds: 1e-2 relative L2 on f and on every layer's
gradient (the BF16 tolerance for this network), 1e-3 on the loss.
"""
import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04661_gb300 import build
    build.build()
    import paper_1609_04661_gb300 as dg
    dg.load()
    return dg


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _params(seed):
    ws, bs = cnn.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    bs = [np.asarray(rng.standard_normal(b.shape) * 0.05, dtype=np.float32).astype(np.float64) for b in bs]
    return ws, bs


def _images(seed, B=2, H=40, W=36):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    base = np.sin(xx / 5.0) + np.cos(yy / 7.0)
    r = np.stack([base * (1 + 0.3 * b) + rng.standard_normal((H, W)) * 0.4 for b in range(B)])
    x = np.stack([base * (1 + 0.3 * b) for b in range(B)])
    return r.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W", [(40, 36), (37, 45)])        # ragged tiles of the end layers
def test_forward_matches_reference(dg, H, W):
    from paper_1609_04661_gb300.binding import flatten_params
    ws, bs = _params(3)
    r, _ = _images(4, H=H, W=W)
    sig = np.array([0.5, 2.0])
    with dg.CNN(17, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        d = net.denoise(torch.as_tensor(r, dtype=torch.float32).cuda(), sig.astype(np.float32))
        torch.cuda.synchronize()
        d = d.cpu().numpy().astype(np.float64)
    f_ref, _ = cnn.net_forward(r / sig[:, None, None], ws, bs, bf16=True)
    f_gpu = (r - d) / sig[:, None, None]
    assert rel(f_gpu, f_ref) < 1e-2
    # against the un-rounded FP64 network too (BF16 activations cost more)
    f64, _ = cnn.net_forward(r / sig[:, None, None], ws, bs, bf16=False)
    assert rel(f_gpu, f64) < 5e-2


def test_gradients_match_reference(dg):
    from paper_1609_04661_gb300.binding import flatten_params, unflatten_params
    ws, bs = _params(5)
    r, x = _images(6)
    sig = np.array([0.7, 1.3])
    with dg.CNN(17, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        loss, g = net.gradients(torch.as_tensor(r, dtype=torch.float32).cuda(),
                                torch.as_tensor(x, dtype=torch.float32).cuda(), sig.astype(np.float32))
    loss_ref, gws_ref, gbs_ref = cnn.loss_and_grads(r, x, sig, ws, bs, bf16=True)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    gws, gbs = unflatten_params(g)
    for l in range(17):
        assert rel(gws[l], gws_ref[l]) < 1e-2, l
        assert rel(gbs[l], gbs_ref[l]) < 1e-2, l


def test_training_reduces_loss(dg):
    r, x = _images(7, B=4, H=32, W=32)
    sig = np.full(4, 0.4, dtype=np.float32)
    rt = torch.as_tensor(r, dtype=torch.float32).cuda()
    xt = torch.as_tensor(x, dtype=torch.float32).cuda()
    with dg.CNN(17, seed=1) as net:
        losses = [net.train_step(rt, xt, sig, 1e-3) for _ in range(100)]
    assert all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.7 * np.mean(losses[:5])


@pytest.mark.parametrize("sigma", [0.7, 1.0])
def test_forward_mode_derivative_matches_reference(dg, sigma):
    """J_D(r) b through the C ABI against the oracle's forward-mode pass with the
    same BF16 rounding of the primal and tangent activations.  The tangent
    passes 16 BF16 roundings and, besides the flips the forward pass sees, a
    ReLU mask flips wherever a primal activation straddles zero between the
    FP32 and FP64 sums, so its bound is 3e-2 rather than the forward's 1e-2."""
    from paper_1609_04661_gb300.binding import flatten_params
    ws, bs = _params(5)
    r, _ = _images(8, B=1, H=40, W=36)
    b = np.random.default_rng(9).standard_normal((40, 36)).astype(np.float32).astype(np.float64)
    with dg.CNN(17, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        d, jb = net.denoise_jvp(torch.as_tensor(r[0], dtype=torch.float32).cuda(),
                                torch.as_tensor(b, dtype=torch.float32).cuda(), sigma)
        d, jb = d.cpu().numpy(), jb.cpu().numpy()
    d_ref, jb_ref = cnn.denoise_jvp(r[0], b, sigma, ws, bs, bf16=True)
    assert rel(d, d_ref) < 1e-2
    assert rel(jb, jb_ref) < 3e-2
    # the divergence b^T J_D b / N the solve uses
    assert float(b.ravel() @ jb.ravel()) / b.size == pytest.approx(float(b.ravel() @ jb_ref.ravel()) / b.size,
                                                                  rel=2e-2, abs=2e-2)
