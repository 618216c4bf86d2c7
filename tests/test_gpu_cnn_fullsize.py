"""GPU parity of the tensor-core convolution at the sizes and launch shapes
the solve runs it, against the FP64 reference in oracle/cnn.py (BF16
activation rounding emulated at the same points), and the reporting of a
timed-out wait.

The hidden layers' kernel gives each CTA a contiguous range of 128-pixel
strips (rows of one 128-column band), up to one CTA per SM.  Small images
give every CTA one or two strips; these cases give them many:
  * B = 2, H = 96, W = 300: three bands per row (edges at 128 and 256, the
    third ragged, 44 live columns), 576 strips, so each CTA runs about four
    strips, with runs that cross from one band (or image) into the next;
  * B = 1, H = W = 512: the 512 x 512 solve's own shape, 2048 strips, about
    14 per CTA: the six-slot row ring wraps many times, both MMA warps
    alternate over all four accumulators, and the mbarrier phases wrap.

Two kinds of bound.
  * The kernel itself: a 3-layer network has exactly one tensor-core layer
    (1 -> 64, 64 -> 64 on tcgen05, 64 -> 1), so the GPU and the oracle
    differ only by FP32 summation order and the BF16 roundings that order
    flips (one BF16 step, 2^-8, on the few activations that sit at a tie).
    Held to 1e-3 relative L2 (measured: 3e-5 to 1e-4), forward and every
    gradient, at both shapes; the forward-mode derivative to 5e-3 (its ReLU
    masks are the primal's: where a primal activation sits at zero, FP32 and
    FP64 sums can give different masks, and the masked tangent element then
    differs outright; measured 1.2e-3).  A wrong tap, halo, band edge, ring
    slot or accumulator anywhere would show far above that.
  * The 17-layer network: each flipped rounding perturbs its activation by
    one BF16 step, and 15 layers amplify that, by a factor that depends on
    the weights and the input.  The same mechanism, applied to every
    rounding, is the distance between the oracle's BF16-rounded and
    unrounded FP64 evaluations of the network on the same input, so the GPU
    must lie within 1.5 times that distance of the BF16 oracle (and within
    5e-2 in any case).  Measured: the GPU is at 0.9 times it.  The tangent
    pass adds mask flips to the same mechanism (the oracle's own BF16 and
    FP64 tangents differ by 0.21 on the 512 x 512 case); it is held to 1.5
    times that distance, with no cap, and the divergence the solve uses,
    b^T J_D b / N, to 2e-2 (the two oracle forms agree to 2e-5 on it).
The learned solve keeps the 2e-2 bound of the small learned-solve test.
"""
import numpy as np
import pytest

import synth
from oracle import cnn, gamp
from oracle.geometry import Geometry

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


def _images(seed, B, H, W):
    """Smooth structure plus noise, different per image (float32-exact)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    r, x = [], []
    for b in range(B):
        base = np.sin(xx / (5.0 + 2 * b)) + np.cos(yy / (7.0 + b)) + 0.5 * ((xx - W / 2) ** 2 + (yy - H / 2) ** 2
                                                                            < (0.3 * min(H, W)) ** 2)
        x.append(base)
        r.append(base + rng.standard_normal((H, W)) * 0.4)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return f32(np.stack(r)), f32(np.stack(x))


def _strips_per_cta(B, H, W):
    nx = (W + 127) // 128
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    return -(-B * H * nx // sm)


SHAPES = [(2, 96, 300), (1, 512, 512)]


def _net(layers, seed):
    ws, bs = cnn.init_params(seed, layers=layers)
    rng = np.random.default_rng(seed + 1)
    bs = [np.asarray(rng.standard_normal(b.shape) * 0.05, dtype=np.float32).astype(np.float64) for b in bs]
    return ws, bs


def _bound(layers, gpu, ref_bf16, ref_fp64, cap=5e-2):
    """The 1e-3 kernel bound for one tensor-core layer; for deeper networks
    1.5 times the oracle's own BF16-vs-FP64 distance (at most `cap`)."""
    if layers == 3:
        return 1e-3
    return min(1.5 * rel(ref_bf16, ref_fp64), cap)


@pytest.mark.parametrize("B,H,W", SHAPES)
@pytest.mark.parametrize("layers", [3, 17])
def test_forward_at_full_size(dg, layers, B, H, W):
    from paper_1609_04661_gb300.binding import flatten_params
    assert _strips_per_cta(B, H, W) >= 3
    ws, bs = _net(layers, 31)
    r, _ = _images(32, B, H, W)
    sig = np.array([0.6, 1.5])[:B]
    with dg.CNN(layers, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        d = net.denoise(torch.as_tensor(r, dtype=torch.float32).cuda(), sig.astype(np.float32))
        d = d.cpu().numpy().astype(np.float64)
    f_gpu = (r - d) / sig[:, None, None]
    f_ref, _ = cnn.net_forward(r / sig[:, None, None], ws, bs, bf16=True)
    bound = 1e-3 if layers == 3 else _bound(layers, f_gpu, f_ref, cnn.net_forward(r / sig[:, None, None], ws, bs)[0])
    assert rel(f_gpu, f_ref) < bound
    for b in range(B):                    # each image, and each 128-column band on its own
        for x0 in range(0, W, 128):
            blk = (b, slice(None), slice(x0, x0 + 128))
            assert rel(f_gpu[blk], f_ref[blk]) < 1.5 * bound, (b, x0)


@pytest.mark.parametrize("B,H,W", SHAPES[:1])
@pytest.mark.parametrize("layers", [3, 17])
def test_gradients_at_full_size(dg, layers, B, H, W):
    """Training's backward pass runs the same kernel (masked, transposed
    weights) over every hidden layer at this shape."""
    from paper_1609_04661_gb300.binding import flatten_params, unflatten_params
    ws, bs = _net(layers, 33)
    r, x = _images(34, B, H, W)
    sig = np.array([0.8, 1.2])[:B]
    with dg.CNN(layers, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        loss, g = net.gradients(torch.as_tensor(r, dtype=torch.float32).cuda(),
                                torch.as_tensor(x, dtype=torch.float32).cuda(), sig.astype(np.float32))
    loss_ref, gws_ref, gbs_ref = cnn.loss_and_grads(r, x, sig, ws, bs, bf16=True)
    if layers != 3:
        _, gws64, gbs64 = cnn.loss_and_grads(r, x, sig, ws, bs, bf16=False)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    gws, gbs = unflatten_params(g, layers=layers)
    for l in range(layers):
        bw = 1e-3 if layers == 3 else _bound(layers, gws[l], gws_ref[l], gws64[l])
        bb = 1e-3 if layers == 3 else _bound(layers, gbs[l], gbs_ref[l], gbs64[l])
        assert rel(gws[l], gws_ref[l]) < bw, l
        assert rel(gbs[l], gbs_ref[l]) < bb, l


@pytest.mark.parametrize("layers", [3, 17])
def test_forward_mode_derivative_at_the_solve_shape(dg, layers):
    """512 x 512, one image: the launch shape of the learned 512 x 512 solve
    (primal and tangent passes, about 14 strips per CTA)."""
    from paper_1609_04661_gb300.binding import flatten_params
    n = 512
    assert _strips_per_cta(1, n, n) >= 12
    ws, bs = _net(layers, 35)
    r, _ = _images(36, 1, n, n)
    b = np.random.default_rng(37).standard_normal((n, n)).astype(np.float32).astype(np.float64)
    sigma = 0.8
    with dg.CNN(layers, seed=0) as net:
        net.set_params(flatten_params(ws, bs))
        d, jb = net.denoise_jvp(torch.as_tensor(r[0], dtype=torch.float32).cuda(),
                                torch.as_tensor(b, dtype=torch.float32).cuda(), sigma)
        d, jb = d.cpu().numpy(), jb.cpu().numpy()
    d_ref, jb_ref = cnn.denoise_jvp(r[0], b, sigma, ws, bs, bf16=True)
    sf, sf_ref = r[0] - d, r[0] - d_ref              # sigma f, the part the network computes
    tf, tf_ref = b - jb, b - jb_ref                  # sigma J_f b / sigma, likewise
    if layers == 3:
        bd, bt = 1e-3, 5e-3
    else:
        d64, jb64 = cnn.denoise_jvp(r[0], b, sigma, ws, bs, bf16=False)
        bd = _bound(layers, sf, sf_ref, r[0] - d64)
        bt = _bound(layers, tf, tf_ref, b - jb64, cap=np.inf)
    assert rel(sf, sf_ref) < bd
    assert rel(tf, tf_ref) < bt
    div, div_ref = float(b.ravel() @ jb.ravel()) / b.size, float(b.ravel() @ jb_ref.ravel()) / b.size
    assert div == pytest.approx(div_ref, rel=2e-2, abs=2e-2)
    for y0 in range(0, n, 128):          # every 128 x 128 block (bands and row ranges of different CTAs)
        for x0 in range(0, n, 128):
            blk = (slice(y0, y0 + 128), slice(x0, x0 + 128))
            assert rel(sf[blk], sf_ref[blk]) < 1.5 * bd, (y0, x0)


def _case300(seed=1500):
    n, nv = 300, 40
    nd = int(np.ceil(1.42 * n))
    ph = synth.random_phantom(n, 8, seed, rho_max=0.02, with_rect=True)
    z = synth.analytic_sinogram(ph, synth.view_angles(nv), nd)
    return dict(n=n, n_views=nv, n_det=nd, I0=1e5, y=synth.poisson_counts(z, 1e5, seed + 7),
                mu=synth.rasterise(ph, n))


def test_learned_solve_300_wide_matches_oracle(dg):
    """Two damped iterations of the learned solve on a 300 x 300 geometry
    (three bands per row, 900 strips per pass) against the oracle."""
    from paper_1609_04661_gb300.binding import flatten_params
    c = _case300()
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 2
    ws, bs = cnn.init_params(41)
    rng = np.random.default_rng(42)
    bs = [np.asarray(rng.standard_normal(b.shape) * 0.02, dtype=np.float32).astype(np.float64) for b in bs]
    log = []
    mu_ref, x_ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(damp_x=0.5, damp_s=0.5), return_x=True,
                                  log=log, cnn=(ws, bs, True))
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(g.n, g.n_views, g.n_det, denoiser=1, cnn_scale=1,
                                            damp_x=0.5, damp_s=0.5) as pl:
        net.set_params(flatten_params(ws, bs))
        pl.set_cnn(net)
        xo = torch.empty((g.n, g.n), device="cuda")
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True, x_out=xo)
        mu, xo = mu.cpu().numpy(), xo.cpu().numpy()
    assert st["iters_done"] == T
    assert np.allclose(st["tau_r"], [lg.tau_r for lg in log], rtol=2e-2)
    assert np.allclose(st["div"], [lg.div for lg in log], rtol=2e-2, atol=2e-2)
    assert rel(xo, x_ref) < 2e-2
    assert rel(mu, mu_ref) < 2e-2


def test_timed_out_wait_is_reported_and_the_context_stays_usable(dg):
    """With the network's timeout test on, every tensor-core convolution
    waits 1 ms on a barrier that nothing arrives at and computes nothing;
    each synchronous entry point must return DGAMP_CT_ERR_TIMEOUT (-5).
    Switched off, the same calls give the results they gave before."""
    from paper_1609_04661_gb300.binding import flatten_params
    c = synth.make_case("ellipse64_v30")
    ws, bs = _net(17, 43)
    r, x = _images(44, 2, 40, 36)
    rt = torch.as_tensor(r, dtype=torch.float32).cuda()
    xt = torch.as_tensor(x, dtype=torch.float32).cuda()
    sig = np.array([0.5, 1.0], dtype=np.float32)
    y = torch.as_tensor(c["y"]).cuda()
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(c["n"], c["n_views"], c["n_det"], denoiser=1, cnn_scale=1,
                                            damp_x=0.5, damp_s=0.5) as pl:
        net.set_params(flatten_params(ws, bs))
        pl.set_cnn(net)
        d0 = net.denoise(rt, sig).cpu().numpy()
        mu0 = pl.solve(y, c["I0"], 2).cpu().numpy()

        net.test_timeout(True)
        calls = [lambda: net.denoise(rt, sig),
                 lambda: net.denoise_jvp(rt[0].contiguous(), xt[0].contiguous(), 0.7),
                 lambda: net.gradients(rt, xt, sig),
                 lambda: pl.solve(y, c["I0"], 2, with_stats=True),
                 lambda: pl.solve_host(c["y"], c["I0"], 2)]
        for k, call in enumerate(calls):
            with pytest.raises(dg.DgampError) as e:
                call()
            assert e.value.code == -5, k
        pl.solve(y, c["I0"], 2)                            # no stats: enqueued only; the flag stays set
        torch.cuda.synchronize()

        net.test_timeout(False)
        with pytest.raises(dg.DgampError) as e:            # the next synchronous call reports it
            net.denoise(rt, sig)
        assert e.value.code == -5
        assert np.array_equal(net.denoise(rt, sig).cpu().numpy(), d0)
        mu1, st = pl.solve(y, c["I0"], 2, with_stats=True)
        assert st["iters_done"] == 2
        assert np.array_equal(mu1.cpu().numpy(), mu0)
