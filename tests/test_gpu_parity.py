"""GPU parity: every step of the D-GAMP-CT iteration through the C ABI against
the FP64 oracle on the same seeded inputs.

Tolerances: 1e-5 relative L2 for each linear operator (A, A^T, H, V^-1) and
for the elementwise/denoiser steps, computed in FP32 against FP64; 1e-3
relative L2 on the reconstruction after a fixed number of iterations; integer
probe words bit-exact.
"""
import numpy as np
import pytest

import synth
from oracle import gamp, joseph, output_step, philox, precond, tv
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
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


# geometries: several tiles and a ragged tail in both the ray and the pixel
# direction, odd and even sizes, the 45-degree tie, explicit angles.
GEOMS = [
    (64, 30, 95, None),
    (37, 13, 55, None),
    (50, 8, 73, (0.0, 0.3, np.pi / 4, 1.2, np.pi / 2, 2.0, 3 * np.pi / 4, 3.0)),
    (129, 7, 190, None),
]


def _img(n, seed, kind="random"):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.uniform(0.0, 1.0, (n, n))
    ph = synth.random_phantom(n, 5, seed)
    return synth.rasterise(ph, n)


@pytest.mark.parametrize("n,nv,nd,ang", GEOMS + [(512, 4, 729, None), (300, 5, 1100, None)])
@pytest.mark.parametrize("kind", ["random", "phantom"])
@pytest.mark.parametrize("pj_seg", [8, 16, 32])            # warps splitting the steps of 32 rays
def test_project_matches_oracle(dg, n, nv, nd, ang, kind, pj_seg):
    g = Geometry(n, nv, nd, ang)
    x = _img(n, 3, kind)
    with dg.Plan(n, nv, nd, angles=ang) as pl:
        pl.set_tuning(pj_seg=pj_seg)
        assert pl.tuning()["pj_seg"] == pj_seg
        z = host(pl.project(cu(x)))
        zp = host(pl.project(cu(x), precond=True))
        again = host(pl.project(cu(x)))
    assert rel(z, joseph.forward_project(x, g)) < 1e-5
    assert rel(zp, precond.project(x, g)) < 1e-5
    assert np.array_equal(z, again)                          # deterministic


# the banded A: bands of 16 or 32 staged lines in shared memory, the rays cut
# into chunks that fill one or two waves (chunks that start and end inside a
# view); 37 views leave an odd number of each orientation, 4096 views make a
# chunk span many views' worth of the limit, n = 37, 50, 129, 300 a short last band
@pytest.mark.parametrize("n,nv,nd,ang", GEOMS + [(512, 4, 729, None), (300, 5, 1100, None), (96, 37, 140, None),
                                                 (16, 4096, 24, None)])
@pytest.mark.parametrize("band,waves", [(16, 1), (16, 2), (32, 1), (32, 2)])
def test_banded_project_matches_oracle(dg, n, nv, nd, ang, band, waves):
    g = Geometry(n, nv, nd, ang)
    x = _img(n, 3, "phantom")
    with dg.Plan(n, nv, nd, angles=ang) as pl:
        pl.set_tuning(pj_band=band, pj_waves=waves)
        t = pl.tuning()
        assert (t["pj_band"], t["pj_waves"]) == (band, waves)
        z = host(pl.project(cu(x)))
        zp = host(pl.project(cu(x), precond=True))
        again = host(pl.project(cu(x)))
        pl.set_tuning(pj_seg=8)                               # a segment count picks the ray-group form
        assert pl.tuning()["pj_band"] == 0
    assert rel(z, joseph.forward_project(x, g)) < 1e-5
    assert rel(zp, precond.project(x, g)) < 1e-5
    assert np.array_equal(z, again)


@pytest.mark.parametrize("storage", [0, 1])
def test_banded_project_equals_sixteen_segments_at_512(dg, storage):
    """At n = 512 a 32-line band is one of 16 segments of the ray-group form:
    both forms add the same steps in the same order, so A x and a solve that
    stores its sinograms in FP32 or BF16 agree bit for bit."""
    n, nv, nd = 512, 16, 729
    x = _img(n, 4, "phantom")
    g = Geometry(n, nv, nd)
    y = np.random.default_rng(5).poisson(1e4 * np.exp(-joseph.forward_project(0.02 * x, g))).astype(np.float32)
    out = {}
    rest = dict(filter_mode=1, sino_fused=2, bp_mode=1, tv_kb=10, tv_rows=64, tv_vrows=4)   # the same elsewhere
    for form in ({"pj_seg": 16}, {"pj_band": 32, "pj_waves": 1}):
        with dg.Plan(n, nv, nd, storage=storage, damp_x=0.5, damp_s=0.5) as pl:
            pl.set_tuning(**rest, **form)
            out[len(form)] = (host(pl.project(cu(x))), host(pl.solve(cu(y), 1e4, 3)))
    assert np.array_equal(out[1][0], out[2][0])
    assert np.array_equal(out[1][1], out[2][1])


def test_banded_project_tuning_checks(dg):
    with dg.Plan(64, 10, 95) as pl:
        for bad in ({"pj_band": 8}, {"pj_band": 64}, {"pj_waves": 3}):
            with pytest.raises(Exception):
                pl.set_tuning(**bad)


@pytest.mark.parametrize("n,nv,nd,ang", GEOMS + [(512, 4, 729, None)])
@pytest.mark.parametrize("bp_mode", [0, 1])                # pixel-driven gather, ray-driven tiles
def test_backproject_matches_oracle(dg, n, nv, nd, ang, bp_mode):
    g = Geometry(n, nv, nd, ang)
    s = np.random.default_rng(4).standard_normal((nv, nd))
    with dg.Plan(n, nv, nd, angles=ang) as pl:
        pl.set_tuning(bp_mode=bp_mode)
        assert pl.tuning()["bp_mode"] == bp_mode
        b = host(pl.backproject(cu(s)))
        bp = host(pl.backproject(cu(s), precond=True))
        again = host(pl.backproject(cu(s)))
    assert rel(b, joseph.back_project(s, g)) < 1e-5
    assert rel(bp, precond.backproject(s, g)) < 1e-5
    assert np.array_equal(b, again)                         # deterministic


@pytest.mark.parametrize("bp_mode", [0, 1])
def test_gpu_pair_is_adjoint(dg, bp_mode):
    n, nv, nd = 96, 17, 139
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, n))
    s = rng.standard_normal((nv, nd))
    with dg.Plan(n, nv, nd) as pl:
        pl.set_tuning(bp_mode=bp_mode)
        for pc in (False, True):
            ax = host(pl.project(cu(x), precond=pc))
            ats = host(pl.backproject(cu(s), precond=pc))
            lhs, rhs = np.sum(ax * s), np.sum(x * ats)
            assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(ax * ax) * np.sum(s * s))


@pytest.mark.parametrize("mode", [0, 1])                  # FFT, Toeplitz
@pytest.mark.parametrize("n,nv,nd", [(64, 30, 95), (40, 9, 300), (16, 3, 24), (512, 5, 729)])
def test_filter_matches_oracle(dg, n, nv, nd, mode):
    g = Geometry(n, nv, nd)
    s = np.random.default_rng(6).standard_normal((nv, nd))
    with dg.Plan(n, nv, nd) as pl:
        pl.set_tuning(filter_mode=mode)
        assert pl.tuning()["filter_mode"] == mode
        h = host(pl.filter(cu(s)))
        # in place as well
        t = cu(s)
        pl.filter(t, out=t)
        h2 = host(t)
    ref = precond.filter_views(s, g)
    assert rel(h, ref) < 1e-5 and rel(h2, ref) < 1e-5


def test_frobenius_matches_oracle(dg):
    for n, nv, nd in [(64, 30, 95), (37, 13, 55)]:
        with dg.Plan(n, nv, nd) as pl:
            assert pl.frob_sq == pytest.approx(precond.frobenius_sq(Geometry(n, nv, nd)), rel=1e-11)


@pytest.mark.parametrize("tau_p", [1e-4, 0.05, 3.0])
def test_output_step_matches_oracle(dg, tau_p):
    n, nv, nd = 32, 21, 401          # M = 8421: several blocks and a ragged tail
    rng = np.random.default_rng(7)
    I0 = 1e5
    z_true = rng.uniform(0.0, 14.0, (nv, nd))
    y = rng.poisson(I0 * np.exp(-z_true)).astype(np.float64)
    z = z_true + rng.normal(0, 0.5, (nv, nd))
    s_prev = rng.normal(0, 1.0, (nv, nd))
    with dg.Plan(n, nv, nd) as pl:
        s, ts = pl.output_step(cu(z), cu(y), cu(s_prev), I0, tau_p)
        s, ts = host(s), float(host(ts)[0])
    # the kernel forms p = fma(-tau_p, s_prev, z) in FP32; give the oracle that same p
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    p = f32(f32(z).reshape(-1) - f32(tau_p) * f32(s_prev).reshape(-1))
    s_ref, tsi_ref, _, _ = output_step.output_step(p, y.reshape(-1), float(f32(tau_p)), I0)
    assert rel(s.reshape(-1), s_ref) < 1e-5
    assert ts == pytest.approx(np.mean(tsi_ref), rel=1e-5)
    assert (y == 0).any()


def test_truncated_output_step_matches_oracle(dg):
    """truncate_z = 1: rays through (almost) nothing, where counts can exceed
    I0 and the unconstrained mode falls below 0, mixed with ordinary rays."""
    n, nv, nd = 32, 9, 301
    rng = np.random.default_rng(11)
    I0, tau_p = 1e4, 0.4
    z_true = np.where(rng.random((nv, nd)) < 0.4, rng.uniform(-0.03, 0.01, (nv, nd)), rng.uniform(0.5, 8, (nv, nd)))
    y = rng.poisson(I0 * np.exp(-z_true)).astype(np.float64)
    z = z_true + rng.normal(0, 0.3, (nv, nd))
    with dg.Plan(n, nv, nd, truncate_z=1) as pl:
        s, ts = pl.output_step(cu(z), cu(y), None, I0, tau_p)
        s, ts = host(s), float(host(ts)[0])
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    s_ref, tsi_ref, z0, _ = output_step.output_step(f32(z).reshape(-1), y.reshape(-1), float(f32(tau_p)), I0,
                                                    truncate=True)
    assert (z0 == 0).sum() > 100
    assert rel(s.reshape(-1), s_ref) < 1e-5
    assert ts == pytest.approx(np.mean(tsi_ref), rel=1e-5)


@pytest.mark.parametrize("rows,vrows", [(32, 4), (64, 4), (128, 4), (64, 8), (64, 2)])   # region height, rows per thread
@pytest.mark.parametrize("kb", [1, 3, 7, 10])           # steps per blocked launch (remainders too)
@pytest.mark.parametrize("n,lam", [(64, 0.3), (77, 0.05), (33, 0.0), (130, 0.2), (300, 0.1)])
def test_tv_matches_oracle(dg, n, lam, kb, rows, vrows):
    r = np.cumsum(np.random.default_rng(8).standard_normal((n, n)), axis=1) * 0.1
    with dg.Plan(n, 10, 2 * n, k_tv=20) as pl:
        pl.set_tuning(tv_kb=kb, tv_rows=rows, tv_vrows=vrows)
        x = host(pl.denoise_tv(cu(r), lam))
    assert rel(x, tv.tv_prox(r, lam, 20)) < 1e-5


@pytest.mark.parametrize("kb", [3, 10])
@pytest.mark.parametrize("n", [64, 77, 300])
def test_tv_pair_forms_agree(dg, n, kb):
    """The MC pair (r and r + eps b) with both images in one thread (packed
    FP32 pairs: 32- and 64-row regions of 4-row threads, 64-row regions of
    2-row threads) or in separate blocks (128-row regions, 8-row threads):
    the same x bit for bit, the same divergence up to the order of its FP64
    sum, and the oracle's to its tolerance."""
    r = np.cumsum(np.random.default_rng(10).standard_normal((n, n)), axis=0) * 0.2
    tau_r, t = 0.01, 5
    shapes = [(32, 4), (64, 4), (64, 2), (128, 4), (64, 8)]
    out = []
    with dg.Plan(n, 10, 2 * n, k_tv=20, c_tv=3.0, seed=77) as pl:
        for rows, vrows in shapes:
            pl.set_tuning(tv_kb=kb, tv_rows=rows, tv_vrows=vrows)
            x, dv = pl.denoise_div(cu(r), tau_r, t)
            out.append((host(x), float(host(dv)[0])))
    for (x, dv), shape in zip(out[1:], shapes[1:]):
        assert np.array_equal(x, out[0][0]), shape
        assert dv == pytest.approx(out[0][1], rel=1e-9), shape
    lam = 3.0 * np.sqrt(tau_r)
    D = lambda v: tv.tv_prox(v, lam, 20)
    x_ref = D(r)
    b = philox.probe_normals(n * n, 77, t, 0).reshape(n, n)
    eps = 1e-3 * max(np.max(np.abs(r)), 1e-6)
    assert rel(out[0][0], x_ref) < 1e-5
    assert out[0][1] == pytest.approx(gamp.mc_divergence(D, r, x_ref, b, eps), rel=2e-3)


def test_probe_words_bitexact_and_normals_close(dg):
    n = 10_003
    with dg.Plan(16, 4, 24, seed=0x1234_5678_9ABC, slice_id=3) as pl:
        b, w = pl.probe(7, n, words=True)
        b, w = host(b), w.cpu().numpy().view(np.uint32)
    ref_w = philox.probe_words(n, 0x1234_5678_9ABC, 7, 3)
    assert np.array_equal(w, ref_w)
    ref_b = philox.probe_normals(n, 0x1234_5678_9ABC, 7, 3)
    assert np.max(np.abs(b - ref_b)) < 1e-5


def test_denoise_divergence_matches_oracle(dg):
    n = 64
    r = np.cumsum(np.random.default_rng(9).standard_normal((n, n)), axis=0) * 0.2
    tau_r, t = 0.01, 4
    opts = gamp.Options(c_tv=3.0, k_tv=20, seed=77, slice_id=0)
    with dg.Plan(n, 10, 2 * n, k_tv=20, c_tv=3.0, seed=77) as pl:
        x, dv = pl.denoise_div(cu(r), tau_r, t)
        x, dv = host(x), float(host(dv)[0])
    lam = opts.c_tv * np.sqrt(tau_r)
    D = lambda v: tv.tv_prox(v, lam, 20)
    x_ref = D(r)
    b = philox.probe_normals(n * n, 77, t, 0).reshape(n, n)
    eps = 1e-3 * max(np.max(np.abs(r)), 1e-6)
    div_ref = gamp.mc_divergence(D, r, x_ref, b, eps)
    assert rel(x, x_ref) < 1e-5
    assert dv == pytest.approx(div_ref, rel=2e-3)


@pytest.mark.parametrize("n", [64, 48])
def test_precond_image_matches_oracle(dg, n):
    g = Geometry(n, 10, 2 * n)
    x = np.random.default_rng(10).standard_normal((n, n))
    with dg.Plan(n, 10, 2 * n) as pl:
        vi = host(pl.precond_image(cu(x), inverse=True))
        vf = host(pl.precond_image(cu(x), inverse=False))
    assert rel(vi, precond.v_inverse(x, g)) < 1e-5
    assert rel(vf, precond.v_forward(x, g)) < 1e-5


# ---------------------------------------------------------------- solve ----
@pytest.fixture(scope="module")
def case64():
    c = synth.make_case("ellipse64_v30")
    return c, Geometry(c["n"], c["n_views"], c["n_det"])


@pytest.mark.parametrize("use_graph,damp,trunc,onsager", [(1, 1.0, 0, 1), (0, 1.0, 0, 1), (1, 0.5, 0, 1),
                                                            (1, 1.0, 1, 1), (1, 1.0, 0, 0), (1, 0.5, 0, 0)])
def test_solve_matches_oracle_after_20_iterations(dg, case64, use_graph, damp, trunc, onsager):
    """onsager = 0 is Section 7.1's form without the Onsager term (p = z)."""
    c, g = case64
    T = c["iters"]
    log = []
    opts = gamp.Options(c_tv=3.0, k_tv=20, damp_x=damp, damp_s=damp, truncate_z=bool(trunc),
                        onsager=bool(onsager))
    mu_ref, x_ref = gamp.ct_solve(c["y"], c["I0"], g, T, opts, return_x=True, log=log)
    with dg.Plan(g.n, g.n_views, g.n_det, c_tv=3.0, k_tv=20, use_graph=use_graph, damp_x=damp, damp_s=damp,
                 truncate_z=trunc, onsager=onsager) as pl:
        xo = torch.empty((g.n, g.n), device="cuda")
        mu, st = pl.solve(cu(c["y"]), c["I0"], T, with_stats=True, x_out=xo)
        mu, xo = host(mu), host(xo)
    assert st["iters_done"] == T
    assert rel(xo, x_ref) < 1e-3
    assert rel(mu, mu_ref) < 1e-3
    ref_tx = np.array([lg.tau_x for lg in log])
    ref_tr = np.array([lg.tau_r for lg in log])
    assert np.allclose(st["tau_r"], ref_tr, rtol=1e-3)
    assert np.allclose(st["tau_x"], ref_tx, rtol=2e-2)


@pytest.mark.parametrize("storage", [0, 1])
def test_solve_same_with_either_backprojection(dg, case64, storage):
    """The two forms of A^T sum the same products in different orders: the
    solves agree to FP32 rounding amplified over the iterations (BF16
    storage: to its own rounding, as both read the same BF16 values)."""
    c, g = case64
    out = {}
    for mode in (0, 1):
        with dg.Plan(g.n, g.n_views, g.n_det, c_tv=3.0, k_tv=20, damp_x=0.7, damp_s=0.7, storage=storage) as pl:
            pl.set_tuning(bp_mode=mode, pj_seg=8)
            out[mode] = host(pl.solve(cu(c["y"]), c["I0"], 5))
    # BF16: each form rounds the same stored values, but the sinogram step's
    # summation order (the plan's fused form) decides which BF16 roundings
    # flip; measured up to 3.5e-3 after 5 iterations
    assert rel(out[1], out[0]) < (1e-4 if storage == 0 else 6e-3)


def test_solve_host_buffers_match_device_path(dg, case64):
    c, g = case64
    with dg.Plan(g.n, g.n_views, g.n_det) as pl:
        mu_d = host(pl.solve(cu(c["y"]), c["I0"], 5))
        mu_h = pl.solve_host(c["y"], c["I0"], 5)
    assert np.array_equal(mu_h.astype(np.float64), mu_d)


def test_solve_rejects_bad_arguments(dg, case64):
    c, g = case64
    with dg.Plan(g.n, g.n_views, g.n_det) as pl:
        for bad in [dict(I0=0.0, iters=3), dict(I0=float("nan"), iters=3), dict(I0=1e4, iters=0)]:
            with pytest.raises(dg.DgampError):
                pl.solve(cu(c["y"]), bad["I0"], bad["iters"])


def test_solve_after_profiling_equals_a_fresh_solve(dg, case64):
    """profile_iteration runs iterations on the plan's state and may leave the
    denoiser's divergence partials pending; the next solve starts clean."""
    c, g = case64
    with dg.Plan(g.n, g.n_views, g.n_det) as pl:
        fresh = host(pl.solve(cu(c["y"]), c["I0"], 4))
        pl.profile_iteration(reps=2)
        mu, st = pl.solve(cu(c["y"]), c["I0"], 4, with_stats=True)
        again = host(mu)
    assert np.array_equal(fresh, again)
    assert st["iters_done"] == 4 and np.all(np.isfinite(st["tau_x"]))
