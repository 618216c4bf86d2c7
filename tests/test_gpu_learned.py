"""GPU parity of the learned D-GAMP-CT solve: Algorithm 1 with the residual
CNN as the Step 4 denoiser, through the C ABI, against the FP64 oracle with
the same BF16-rounded weights and BF16 activation rounding.

The parity network is a seeded He-initialised one: its BF16 evaluation
stays within 2e-3 of its own FP64 evaluation on these inputs, so the test
measures the solve, not the network's sensitivity.  (The shipped trained
weights, fed inputs far outside their training range -- sigma = sqrt(tau_r)
near 1 while the actual error of r is near 0.003 -- differ from their own
FP64 evaluation by about 27% in BF16; no two BF16 implementations can agree
more closely than that there.)

Tolerance: the GPU and the oracle round the same activations to BF16
(relative step 2^-8) from FP32 and FP64 sums; a rounding decision flips when
the two sums straddle a BF16 tie, which perturbs that activation by one BF16
step.  One network evaluation then agrees to a few 1e-3 (the forward parity
test bounds it at 1e-2); three iterations of the loop feed that through
tau_x, tau_r and r, so the reconstruction and the variances are held to
2e-2 relative.
"""
import numpy as np
import pytest

import synth
from oracle import cnn, gamp
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04661_gb300 import build
    build.build()
    import paper_1609_04661_gb300 as dg
    dg.load()
    return dg


@pytest.fixture(scope="module")
def weights():
    from paper_1609_04661_gb300.train_denoiser import load_weights
    layers, params, scaled = load_weights()
    assert layers == cnn.LAYERS
    return params, scaled


@pytest.mark.parametrize("scaled", [1, 0])
def test_learned_solve_matches_oracle(dg, scaled):
    from paper_1609_04661_gb300.binding import flatten_params
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 3
    ws, bs = cnn.init_params(21)                  # BF16-valued weights, zero biases
    rng = np.random.default_rng(22)
    bs = [np.asarray(rng.standard_normal(b.shape) * 0.02, dtype=np.float32).astype(np.float64) for b in bs]
    params = flatten_params(ws, bs)
    log = []
    opts = gamp.Options(damp_x=0.5, damp_s=0.5)
    mu_ref, x_ref = gamp.ct_solve(c["y"], c["I0"], g, T, opts, return_x=True, log=log,
                                  cnn=(ws, bs, bool(scaled)))
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(g.n, g.n_views, g.n_det, denoiser=1, cnn_scale=scaled,
                                            damp_x=0.5, damp_s=0.5) as pl:
        net.set_params(params)
        pl.set_cnn(net)
        xo = torch.empty((g.n, g.n), device="cuda")
        y = torch.as_tensor(c["y"]).cuda()
        mu, st = pl.solve(y, c["I0"], T, with_stats=True, x_out=xo)
        mu, xo = mu.cpu().numpy(), xo.cpu().numpy()
    assert st["iters_done"] == T
    assert np.allclose(st["tau_r"], [lg.tau_r for lg in log], rtol=2e-2)
    assert np.allclose(st["div"], [lg.div for lg in log], rtol=2e-2, atol=2e-2)
    assert rel(xo, x_ref) < 2e-2
    assert rel(mu, mu_ref) < 2e-2


@pytest.mark.parametrize("c_tv", [3.0, 0.3])
def test_judged_learned_solve_matches_oracle(dg, c_tv):
    """Denoiser 2: the seeded network and prox-TV both run every iteration
    and the lower SURE risk estimate keeps one, the network only while its
    divergence is below M/N (oracle.gamp.Selected).  The
    GPU must keep the same denoiser as the oracle in every iteration, with
    the same risk estimates and reconstruction to the learned solve's 2e-2.
    c_tv = 0.3 makes prox-TV a weak smoother, so the network is kept in some
    iterations; with c_tv = 3 prox-TV is kept throughout."""
    from paper_1609_04661_gb300.binding import flatten_params
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 5
    ws, bs = cnn.init_params(21)
    rng = np.random.default_rng(22)
    bs = [np.asarray(rng.standard_normal(b.shape) * 0.02, dtype=np.float32).astype(np.float64) for b in bs]
    kw = dict(c_tv=c_tv, k_tv=20, damp_x=0.5, damp_s=0.5)
    log = []
    mu_ref, x_ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(**kw), return_x=True, log=log,
                                  cnn=(ws, bs, True), select=True)
    keep_ref = [lg.kept == 1 for lg in log]
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(g.n, g.n_views, g.n_det, denoiser=2, cnn_scale=1, **kw) as pl:
        net.set_params(flatten_params(ws, bs))
        pl.set_cnn(net)
        xo = torch.empty((g.n, g.n), device="cuda")
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True, x_out=xo)
        mu, xo = mu.cpu().numpy(), xo.cpu().numpy()
    keep = [bool(k) for k in st["kept_learned"]]
    print(f"c_tv {c_tv}: kept the network in iterations {[t + 1 for t, k in enumerate(keep_ref) if k]}")
    assert st["iters_done"] == T
    assert keep == keep_ref
    assert st["learned_kept"] == sum(keep_ref)
    assert np.allclose(st["risk_plain"], [lg.risks[0] for lg in log], rtol=2e-2, atol=1e-4)
    assert np.allclose(st["risk_learned"], [lg.risks[1] for lg in log], rtol=2e-2, atol=1e-4)
    assert np.allclose(st["tau_r"], [lg.tau_r for lg in log], rtol=2e-2)
    assert rel(xo, x_ref) < 2e-2
    assert rel(mu, mu_ref) < 2e-2


def _linear_network(beta, layers):
    """17-layer weights computing f(u) = beta u exactly in the network's own
    form: layer 1 passes u and -u to channels 0 and 1, the hidden layers keep
    both (ReLU leaves them as they are), the last one takes beta (relu(u) -
    relu(-u)).  So D(r) = r - sigma f(r / sigma) = (1 - beta) r, with
    divergence 1 - beta, whatever sigma is."""
    ws, bs = [], []
    w = np.zeros((3, 3, 1, 64))
    w[1, 1, 0, 0], w[1, 1, 0, 1] = 1.0, -1.0
    ws.append(w)
    bs.append(np.zeros(64))
    for _ in range(layers - 2):
        w = np.zeros((3, 3, 64, 64))
        w[1, 1, 0, 0] = w[1, 1, 1, 1] = 1.0
        ws.append(w)
        bs.append(np.zeros(64))
    w = np.zeros((3, 3, 64, 1))
    w[1, 1, 0, 0], w[1, 1, 1, 0] = beta, -beta
    ws.append(w)
    bs.append(np.zeros(1))
    return ws, bs


def test_judged_solve_keeps_the_network_where_it_wins(dg):
    """Denoiser 2 with a network that is the linear shrink D(r) = (1 - beta) r,
    beta = 1 - 2^-7 (exact in BF16), and a weak prox-TV (c_tv = 0.3) on the
    64 x 64 case: the oracle keeps the network in iterations 1 and 2 (its
    divergence 2^-7 lies in (0, M/N) and its SURE estimate is lower) and
    prox-TV afterwards, by margins of 3% and more.  The GPU must make the
    same choices, with the same risk estimates, and reach the same x."""
    from paper_1609_04661_gb300.binding import flatten_params
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 6
    ws, bs = _linear_network(1.0 - 2.0 ** -7, cnn.LAYERS)
    kw = dict(c_tv=0.3, k_tv=20, damp_x=0.5, damp_s=0.5)
    log = []
    mu_ref, x_ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(**kw), return_x=True, log=log,
                                  cnn=(ws, bs, True), select=True)
    keep_ref = [lg.kept == 1 for lg in log]
    assert keep_ref == [True, True, False, False, False, False]
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(g.n, g.n_views, g.n_det, denoiser=2, cnn_scale=1, **kw) as pl:
        net.set_params(flatten_params(ws, bs))
        pl.set_cnn(net)
        xo = torch.empty((g.n, g.n), device="cuda")
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True, x_out=xo)
        mu, xo = mu.cpu().numpy(), xo.cpu().numpy()
    assert [bool(k) for k in st["kept_learned"]] == keep_ref
    assert st["learned_kept"] == 2
    assert np.allclose(st["risk_plain"], [lg.risks[0] for lg in log], rtol=1e-3, atol=1e-6)
    assert np.allclose(st["risk_learned"], [lg.risks[1] for lg in log], rtol=1e-3, atol=1e-6)
    assert np.allclose(st["div"], [lg.div for lg in log], rtol=1e-3, atol=1e-6)
    assert rel(xo, x_ref) < 2e-3
    assert rel(mu, mu_ref) < 2e-3


def test_shipped_network_in_a_solve_matches_oracle(dg, weights):
    """The shipped weights inside two damped iterations of the 64 x 64 solve,
    against the oracle with the same BF16-rounded weights and activation
    rounding.  These weights amplify BF16 rounding flips far more than a
    random network on this input (their inputs lie outside their training
    range), so the bound is 1.5 times the oracle's own distance between its
    BF16 and FP64 evaluations of the same solve, as for deep networks in
    test_gpu_cnn_fullsize.py."""
    from paper_1609_04661_gb300.binding import unflatten_params
    params, scaled = weights
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 2
    ws, bs = unflatten_params(params)
    ws = [cnn.bf16_round(w) for w in ws]
    opts = gamp.Options(damp_x=0.5, damp_s=0.5)
    mu16 = gamp.ct_solve(c["y"], c["I0"], g, T, opts, cnn=(ws, bs, bool(scaled)))
    mu64 = gamp.ct_solve(c["y"], c["I0"], g, T, opts, cnn=(ws, bs, bool(scaled)), cnn_bf16=False)
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(g.n, g.n_views, g.n_det, denoiser=1, cnn_scale=int(scaled),
                                            damp_x=0.5, damp_s=0.5) as pl:
        net.set_params(params)
        pl.set_cnn(net)
        mu = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T).cpu().numpy()
    bound = max(1.5 * rel(mu16, mu64), 2e-2)
    print(f"shipped network, {T} iterations: GPU vs BF16 oracle {rel(mu, mu16):.2e}, "
          f"oracle BF16 vs FP64 {rel(mu16, mu64):.2e}")
    assert rel(mu, mu16) < bound


def test_learned_solve_needs_a_network(dg):
    c = synth.make_case("ellipse64_v30")
    with dg.Plan(c["n"], c["n_views"], c["n_det"], denoiser=1) as pl:
        with pytest.raises(dg.DgampError):
            pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], 2)


def test_shipped_network_denoises_gaussian_noise(dg, weights):
    """The shipped weights are a noise-level-scaled Gaussian denoiser: on a
    held-out phantom in the preconditioned space it must remove most of the
    noise at every level it was trained for."""
    params, scaled = weights
    assert scaled
    c = synth.make_case("ellipse512_v64", seed=1000)
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(c["n"], c["n_views"], c["n_det"]) as pl:
        net.set_params(params)
        xt = pl.precond_image(torch.as_tensor(c["mu"], dtype=torch.float32).cuda(), inverse=False)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        for sigma in (0.01, 0.1, 1.0):
            r = (xt + sigma * torch.randn(xt.shape, generator=gen, device="cuda")).contiguous()
            d = net.denoise(r[None].contiguous(), np.array([sigma], dtype=np.float32))[0]
            mse_in = float(((r - xt) ** 2).mean())
            mse_out = float(((d - xt) ** 2).mean())
            assert mse_out < 0.1 * mse_in, (sigma, mse_in, mse_out)


def test_shipped_network_beats_prox_tv_as_a_denoiser(dg, weights):
    """What the trained network gains over the method's plain denoiser, as a
    denoiser: on a held-out phantom in the preconditioned space with Gaussian
    noise of level sigma, its output error against that of the prox-TV the
    solve uses at the same level (lambda = 3 sigma, 20 Chambolle steps)."""
    params, scaled = weights
    c = synth.make_case("ellipse512_v64", seed=1000)
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(c["n"], c["n_views"], c["n_det"], c_tv=3.0, k_tv=20) as pl:
        net.set_params(params)
        xt = pl.precond_image(torch.as_tensor(c["mu"], dtype=torch.float32).cuda(), inverse=False)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        for sigma in (0.01, 0.1, 1.0):
            r = (xt + sigma * torch.randn(xt.shape, generator=gen, device="cuda")).contiguous()
            d_net = net.denoise(r[None].contiguous(), np.array([sigma], dtype=np.float32))[0]
            d_tv = pl.denoise_tv(r, 3.0 * sigma)
            mse_net = float(((d_net - xt) ** 2).mean())
            mse_tv = float(((d_tv - xt) ** 2).mean())
            print(f"sigma {sigma}: network MSE {mse_net:.3e}, prox-TV MSE {mse_tv:.3e}")
            assert mse_net < mse_tv, (sigma, mse_net, mse_tv)


def test_graph_recaptured_after_network_workspace_grows(dg, weights):
    """Using the attached network elsewhere (here: a gradient pass that keeps
    all 17 activations) regrows its workspace; the next solve must re-capture
    the iteration graph and give the same result as before."""
    params, scaled = weights
    c = synth.make_case("ellipse64_v30")
    y = torch.as_tensor(c["y"]).cuda()
    with dg.CNN(cnn.LAYERS) as net, dg.Plan(c["n"], c["n_views"], c["n_det"], denoiser=1,
                                            cnn_scale=int(scaled), damp_x=0.5, damp_s=0.5) as pl:
        net.set_params(params)
        pl.set_cnn(net)
        mu1 = pl.solve(y, c["I0"], 3).cpu().numpy()
        r = torch.rand((4, 96, 96), device="cuda")
        net.gradients(r, r, np.ones(4, dtype=np.float32))
        mu2 = pl.solve(y, c["I0"], 3).cpu().numpy()
    assert np.array_equal(mu1, mu2)
