"""GPU parity of the prox-TV in the (V^T V)^{-1} norm (Section 6.3, option
tv_metric) against the FP64 oracle.

Tolerances: 1e-4 relative L2 on the denoised image (20 dual steps, each with
an FP32 2-D FFT filter on the m x m padded grid, against FP64), 5e-3 on the
MC divergence (a difference of two FP32 denoisings at eps = 1e-3 max|r|),
1e-3 on a 5-iteration solve.
"""
import numpy as np
import pytest

import synth
from oracle import gamp, philox, precond, tv
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


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.float64)


def metric_prox(r, lam, k, g):
    return tv.tv_prox_metric(r, lam, k, lambda u: precond.vtv_inverse(u, g),
                             precond.vtv_inverse_norm_bound(g))


@pytest.mark.parametrize("n,lam,k", [(37, 0.3, 20), (64, 0.05, 20), (100, 1.0, 7), (16, 0.2, 1)])
def test_metric_tv_matches_oracle(dg, n, lam, k):
    r = np.cumsum(np.random.default_rng(n).standard_normal((n, n)), axis=1) * 0.1
    g = Geometry(n, 10, 2 * n)
    with dg.Plan(n, 10, 2 * n, k_tv=k, tv_metric=1) as pl:
        x = host(pl.denoise_tv(cu(r), lam))
    ref = metric_prox(r, lam, k, g)
    assert rel(x, ref) < 1e-4
    assert rel(x, tv.tv_prox(r, lam, k)) > 1e-3        # not the l2 prox


def test_metric_tv_identity_cases(dg):
    n = 24
    r = np.random.default_rng(1).standard_normal((n, n))
    with dg.Plan(n, 6, 40, k_tv=0, tv_metric=1) as pl:
        assert np.array_equal(host(pl.denoise_tv(cu(r), 0.5)), r.astype(np.float32))
    with dg.Plan(n, 6, 40, k_tv=10, tv_metric=1) as pl:
        assert np.array_equal(host(pl.denoise_tv(cu(r), 0.0)), r.astype(np.float32))


def test_metric_divergence_matches_oracle(dg):
    n = 64
    r = np.cumsum(np.random.default_rng(9).standard_normal((n, n)), axis=0) * 0.2
    tau_r, t = 0.01, 4
    g = Geometry(n, 10, 2 * n)
    with dg.Plan(n, 10, 2 * n, k_tv=20, c_tv=3.0, seed=77, tv_metric=1) as pl:
        x, dv = pl.denoise_div(cu(r), tau_r, t)
        x, dv = host(x), float(host(dv)[0])
    lam = 3.0 * np.sqrt(tau_r)
    D = lambda v: metric_prox(v, lam, 20, g)
    x_ref = D(r)
    b = philox.probe_normals(n * n, 77, t, 0).reshape(n, n)
    eps = 1e-3 * max(np.max(np.abs(r)), 1e-6)
    assert rel(x, x_ref) < 1e-4
    assert dv == pytest.approx(gamp.mc_divergence(D, r, x_ref, b, eps), rel=5e-3)


def test_metric_solve_matches_oracle(dg):
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    T = 5
    ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(c_tv=3.0, k_tv=20, tv_metric=True))
    with dg.Plan(g.n, g.n_views, g.n_det, c_tv=3.0, k_tv=20, tv_metric=1) as pl:
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True)
        prof = pl.profile_iteration(reps=1)
        launches = pl.solve_launches(T)
        pl.set_options(tv_metric=0)
        assert pl.solve_launches(T) < launches
    assert st["iters_done"] == T
    assert rel(host(mu), ref) < 1e-3
    assert "tvm_rows_inv20" in prof and "tv_final" in prof and "tvm_dual0" in prof
    assert sum(k.startswith("tvm_") for k in prof) == 4 * 20


def test_metric_option_is_validated(dg):
    with dg.Plan(16, 3, 24) as pl:
        with pytest.raises(dg.DgampError):
            pl.set_options(tv_metric=2)
        pl.set_options(tv_metric=1)


def test_metric_full_size_psnr_follows_oracle(dg):
    """The 512 x 512 / 64-view headline slice, damped, with the metric prox:
    the GPU solve's PSNR after 3 and 6 iterations (6 is the curve's peak)
    against the oracle's stored curve (tests/golden/metric_psnr.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "metric_psnr.txt")
    curve = [float(v) for v in [ln for ln in open(path) if not ln.startswith("#")][0].split()]
    c = synth.make_case("ellipse512_v64")
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5, tv_metric=1)
    with dg.Plan(c["n"], c["n_views"], c["n_det"], **kw) as pl:
        y = torch.as_tensor(c["y"]).cuda()
        for T in (3, 6):
            mu = host(pl.solve(y, c["I0"], T))
            psnr = 10 * np.log10(c["mu"].max() ** 2 / np.mean((mu - c["mu"]) ** 2))
            assert abs(psnr - curve[T - 1]) < 0.05
