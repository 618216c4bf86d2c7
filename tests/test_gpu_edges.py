"""GPU parity at the edges of the accepted inputs: the smallest image, the
most views and the most detector bins the library takes, the denoiser with
no Chambolle steps or zero weight (the identity), and a dose so low that
most counts are zero.  Each against the FP64 oracle on the same seeded
inputs, to the bounds of the main parity tests (1e-5 per operator, 1e-3 on
a reconstruction)."""
import numpy as np
import pytest

from oracle import gamp, joseph, precond
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


def _counts(g, I0, seed, peak=0.05):
    """Poisson counts of a smooth seeded object through the oracle's A."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:g.n, 0:g.n]
    c = 0.5 * (g.n - 1)
    mu = peak * np.clip(1.0 - ((xx - c) ** 2 + (yy - c) ** 2) / (0.45 * g.n) ** 2, 0.0, None)
    z = joseph.forward_project(mu, g)
    return rng.poisson(I0 * np.exp(-z)).astype(np.float32)


# (n, views, bins): the smallest image; the most views (DGAMP_CT_MAX_VIEWS);
# the most bins (DGAMP_CT_MAX_P = 8192 = 2 x 4096)
EDGE_GEOMS = [(2, 3, 3), (16, 4096, 24), (16, 2, 4096)]


@pytest.mark.parametrize("n,nv,nd", EDGE_GEOMS)
def test_operators_at_the_edges(dg, n, nv, nd):
    g = Geometry(n, nv, nd)
    rng = np.random.default_rng(n + nv)
    x = rng.uniform(0.0, 1.0, (n, n))
    s = rng.standard_normal((nv, nd))
    with dg.Plan(n, nv, nd) as pl:
        z = host(pl.project(cu(x)))
        zp = host(pl.project(cu(x), precond=True))
        b = host(pl.backproject(cu(s)))
        bp = host(pl.backproject(cu(s), precond=True))
    assert rel(z, joseph.forward_project(x, g)) < 1e-5
    assert rel(zp, precond.project(x, g)) < 1e-5
    assert rel(b, joseph.back_project(s, g)) < 1e-5
    assert rel(bp, precond.backproject(s, g)) < 1e-5


@pytest.mark.parametrize("n,nv,nd", EDGE_GEOMS)
def test_solve_at_the_edges(dg, n, nv, nd):
    g = Geometry(n, nv, nd)
    I0, T = 1e4, 5
    y = _counts(g, I0, 7)
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    mu_ref = gamp.ct_solve(y, I0, g, T, gamp.Options(**kw))
    with dg.Plan(n, nv, nd, **kw) as pl:
        mu, st = pl.solve(cu(y), I0, T, with_stats=True)
        mu = host(mu)
    assert st["iters_done"] == T
    assert np.all(np.isfinite(mu))
    assert rel(mu, mu_ref) < 1e-3


@pytest.mark.parametrize("k_tv,c_tv", [(0, 3.0), (20, 0.0)])
def test_identity_denoiser_solve(dg, k_tv, c_tv):
    """No Chambolle steps, or zero TV weight: D(r) = r, whose MC divergence
    is ||b||^2 / N; the iteration then carries no prior at all."""
    n, nv, nd = 32, 20, 47
    g = Geometry(n, nv, nd)
    I0, T = 1e4, 4
    y = _counts(g, I0, 8)
    kw = dict(c_tv=c_tv, k_tv=k_tv, damp_x=0.5, damp_s=0.5)
    log = []
    mu_ref = gamp.ct_solve(y, I0, g, T, gamp.Options(**kw), log=log)
    with dg.Plan(n, nv, nd, **kw) as pl:
        mu, st = pl.solve(cu(y), I0, T, with_stats=True)
        mu = host(mu)
    assert rel(mu, mu_ref) < 1e-3
    assert np.allclose(st["div"], [lg.div for lg in log], rtol=1e-4)


def test_mostly_zero_counts_solve(dg):
    """I0 = 2 through a dense object: most counts are 0, where the output
    step's Poisson posterior is at its most skewed."""
    n, nv, nd = 32, 20, 47
    g = Geometry(n, nv, nd)
    I0, T = 2.0, 5
    y = _counts(g, I0, 9, peak=0.4)
    assert np.mean(y == 0) > 0.5
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    mu_ref = gamp.ct_solve(y, I0, g, T, gamp.Options(**kw))
    with dg.Plan(n, nv, nd, **kw) as pl:
        mu = host(pl.solve(cu(y), I0, T))
    assert np.all(np.isfinite(mu))
    assert rel(mu, mu_ref) < 1e-3
