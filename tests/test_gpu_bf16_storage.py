"""Solves with BF16 storage (option storage = 1) against the FP64 oracle, and
the FP32 path at the large 1024 x 1024 / 90-view / 1449-bin geometry.

Tolerances.  With storage = 1 the sinograms A x, H A x, s, H s and the image
copies the projector reads are rounded to BF16 (relative step 2^-8, at most
2^-9 relative error per stored value); every sum stays FP32 and the GAMP
scalars FP64.  The output step forms p = z - tau_p s_prev from the rounded z,
so on a long ray (z near 10) the rounding is about 0.02 absolute in z, that
is 2% in the expected counts I0 e^-z -- of the order of the Poisson noise of a
low-count ray.  Measured on the GPU: 5e-3 relative in mu after 5 iterations
and 1.5e-2 after 20 at 64 x 64, 2.8e-2 after 2 iterations at 1024 x 1024 (the
first iterations run at the largest tau_p, where the output step is most
sensitive).  The bounds are twice those.  The FP32 path keeps the 1e-3
relative bound of the other solve tests at every size.
"""
import numpy as np
import pytest

import synth
from oracle import gamp
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


@pytest.mark.parametrize("T,bound", [(5, 1e-2), (20, 3e-2)])
def test_bf16_storage_solve_against_oracle_small(dg, T, bound):
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(c_tv=3.0, k_tv=20))
    with dg.Plan(g.n, g.n_views, g.n_det, c_tv=3.0, k_tv=20, storage=1) as pl:
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True)
        mu = mu.cpu().numpy()
    assert st["iters_done"] == T and np.all(np.isfinite(mu))
    assert rel(mu, ref) < bound


def test_large_geometry_fp32_and_bf16_against_oracle(dg):
    """1024 x 1024, 90 views, 1449 bins, I0 = 1e5, damped, two iterations: the
    FP32 path within 1e-3 of the oracle, BF16 storage within 6e-2."""
    n, nv, nd, I0, T = 1024, 90, 1449, 1e5, 2
    ph = synth.random_phantom(n, 10, 4000)
    y = synth.poisson_counts(synth.analytic_sinogram(ph, synth.view_angles(nv), nd), I0, 4007)
    g = Geometry(n, nv, nd)
    opts = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    ref = gamp.ct_solve(y, I0, g, T, gamp.Options(**opts))
    out = {}
    for storage in (0, 1):
        with dg.Plan(n, nv, nd, storage=storage, **opts) as pl:
            out[storage] = pl.solve(torch.as_tensor(y).cuda(), I0, T).cpu().numpy()
    assert rel(out[0], ref) < 1e-3
    assert rel(out[1], ref) < 6e-2


@pytest.mark.parametrize("k", [0, 97])
def test_large128_sampled_slices_against_oracle(dg, k, record_property):
    """Slices of the 128-slice 1024 x 1024 / 90-view / 1449-bin workload
    itself (large128, slice k), two damped prox-TV iterations: the per-slice
    relative error of the BF16-storage solve (and of the FP32 one) against
    the FP64 oracle, recorded as a test property and bounded as above.  (The
    learned form at this size is not compared here: one FP64 evaluation of
    the network on a 1024 x 1024 image takes minutes on the host.)"""
    c = synth.make_batch("large128", count=k + 1)[k]
    n, nv, nd, I0, T = c["n"], c["n_views"], c["n_det"], c["I0"], 2
    g = Geometry(n, nv, nd)
    opts = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    ref = gamp.ct_solve(c["y"], I0, g, T, gamp.Options(**opts))
    err = {}
    for storage in (0, 1):
        with dg.Plan(n, nv, nd, storage=storage, **opts) as pl:
            err[storage] = rel(pl.solve(torch.as_tensor(c["y"]).cuda(), I0, T).cpu().numpy(), ref)
    record_property("rel_error_vs_fp64_oracle", {"slice": k, "fp32": err[0], "bf16": err[1]})
    print(f"large128[{k}]: rel error vs FP64 oracle after {T} iterations: FP32 {err[0]:.2e}, BF16 storage {err[1]:.2e}")
    assert err[0] < 1e-3
    assert err[1] < 6e-2


def test_storage_option_is_validated_and_single_steps_stay_fp32(dg):
    """storage accepts 0 and 1 only.  FP32 and BF16 stagings share the
    projector's image buffers: a BF16 solve leaves the single-step projection
    (FP32 buffers) unchanged, and a BF16 solve after an FP32 projection equals
    one on a fresh plan (the guard cells are rewritten at each staging)."""
    c = synth.make_case("ellipse64_v30")
    y = torch.as_tensor(c["y"]).cuda()
    pin = dict(pj_seg=8, bp_mode=1)      # the two plans sum in the same order
    with dg.Plan(c["n"], c["n_views"], c["n_det"], storage=1) as fresh:
        fresh.set_tuning(**pin)
        mu_fresh = fresh.solve(y, c["I0"], 3).cpu().numpy()
    with dg.Plan(c["n"], c["n_views"], c["n_det"]) as pl:
        pl.set_tuning(**pin)
        with pytest.raises(dg.DgampError):
            pl.set_options(storage=2)
        pl.set_options(storage=0)
        img = torch.rand((c["n"], c["n"]), device="cuda") + 0.5
        before = pl.project(img).cpu().numpy()
        pl.set_options(storage=1)
        mu_after_fp32 = pl.solve(y, c["I0"], 3).cpu().numpy()
        after = pl.project(img).cpu().numpy()
    assert np.array_equal(before, after)
    assert np.array_equal(mu_fresh, mu_after_fp32)
