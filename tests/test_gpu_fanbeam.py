"""GPU parity of the flat-detector fan-beam operator (dgamp_ct_plan_fan)
against the FP64 oracle.

Tolerances: 1e-5 relative L2 for A, A^T, Phi~ and Phi~^T (FP32 against FP64;
32.32 positions, fraction truncated to 23 bits); the adjoint identity to
FP32 rounding; ||Phi~||_F^2 to 1e-5 (FP32 filter per ray, FP64 sums).
"""
import math

import numpy as np
import pytest

import synth
from oracle import fanbeam

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


GEOMS = [
    (37, 11, 53, 60.0, 45.0, 1.3, None),
    (64, 30, 96, 112.0, 92.0, 1.95, None),
    (48, 8, 70, 1e7, 1e7, 2.0, tuple(np.linspace(0, math.pi, 8, endpoint=False))),   # 45 degrees, far source
    (40, 6, 61, 40 / math.sqrt(2) + 2.5, 40 / math.sqrt(2) + 2.5, 0.8, None),          # closest source allowed
]


def plan(dg, n, nv, nd, sd, dd, du, ang, **kw):
    return dg.Plan(n, nv, nd, angles=ang, fan=dict(src_dist=sd, det_dist=dd, det_spacing=du), **kw)


# A^T in both forms: ray-driven tiles (bp_mode 1; the first three geometries
# admit a lane stride, the closest-source one does not) and the pixel gather
TILE_OK = [True, True, True, False]


@pytest.mark.parametrize("bp_mode", [0, 1])
@pytest.mark.parametrize("n,nv,nd,sd,dd,du,ang,tile_ok", [g + (t,) for g, t in zip(GEOMS, TILE_OK)])
def test_fan_operators_match_oracle(dg, n, nv, nd, sd, dd, du, ang, tile_ok, bp_mode):
    g = fanbeam.FanGeometry(n, nv, nd, sd, dd, du, angles=ang)
    rng = np.random.default_rng(n)
    x = np.cumsum(rng.standard_normal((n, n)), axis=0) * 0.1
    s = rng.standard_normal((nv, nd))
    with plan(dg, n, nv, nd, sd, dd, du, ang) as pl:
        assert pl.tuning()["bp_mode"] == (1 if tile_ok else 0)      # the plan's default form
        if bp_mode == 1 and not tile_ok:
            with pytest.raises(dg.binding.DgampError):
                pl.set_tuning(bp_mode=1)
            return
        pl.set_tuning(bp_mode=bp_mode)
        z = host(pl.project(cu(x), precond=False))
        bt = host(pl.backproject(cu(s), precond=False))
        zp = host(pl.project(cu(x), precond=True))
        bp = host(pl.backproject(cu(s), precond=True))
    assert rel(z, fanbeam.forward_project(x, g)) < 1e-5
    assert rel(bt, fanbeam.back_project(s, g)) < 1e-5
    assert rel(zp, fanbeam.project(x, g)) < 1e-5
    assert rel(bp, fanbeam.backproject(s, g)) < 1e-5
    # A^T is the transpose of A
    lhs, rhs = float(np.sum(z * s)), float(np.sum(x * bt))
    assert lhs == pytest.approx(rhs, rel=1e-5)


def test_fan_frobenius_matches_oracle(dg):
    c = synth.make_case("fan64_v30")
    f = c["fan"]
    g = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"])
    with plan(dg, c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"], None) as pl:
        fr = pl.frob_sq
    assert fr == pytest.approx(fanbeam.frobenius_sq(g), rel=1e-5)


def test_fan_solve_matches_oracle(dg):
    from oracle import gamp
    c = synth.make_case("fan64_v30")
    f = c["fan"]
    g = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"])
    T = 5
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(**kw), frob2=fanbeam.frobenius_sq(g))
    with plan(dg, c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"], None,
              **kw) as pl:
        mu, st = pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T, with_stats=True)
        prof = pl.profile_iteration(reps=1)
        with pytest.raises(dg.DgampError):
            pl.filter(torch.zeros((c["n_views"], c["n_det"]), device="cuda"))
    assert st["iters_done"] == T
    assert rel(host(mu), ref) < 1e-3
    assert list(prof)[:5] == ["vinv_stage_project", "output_step", "backproject", "vinv_update", "probe_input"]


def _golden_frobenius(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "fan_frobenius.txt")
    for line in open(path):
        if line.startswith(name + " "):
            return float(line.split()[1])
    raise KeyError(name)


def test_fan_full_size_matches_oracle(dg):
    """fan512_v102 at its own size: ||Phi~||_F^2 against the stored oracle
    value, and two damped iterations against the oracle (which uses that
    stored value)."""
    from oracle import gamp
    c = synth.make_case("fan512_v102")
    f = c["fan"]
    g = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"])
    frob2 = _golden_frobenius("fan512_v102")
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    T = 2
    ref = gamp.ct_solve(c["y"], c["I0"], g, T, gamp.Options(**kw), frob2=frob2)
    with plan(dg, c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"], None,
              **kw) as pl:
        assert pl.frob_sq == pytest.approx(frob2, rel=1e-5)
        mu = host(pl.solve(torch.as_tensor(c["y"]).cuda(), c["I0"], T))
    assert rel(mu, ref) < 1e-3


def test_fan_full_size_psnr_follows_oracle(dg):
    """fan512_v102, 10 and 30 damped iterations: the GPU solve's PSNR against
    the oracle's stored curve (tests/golden/fan_psnr.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fan_psnr.txt")
    curve = [float(v) for v in [ln for ln in open(path) if not ln.startswith("#")][0].split()]
    c = synth.make_case("fan512_v102")
    f = c["fan"]
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
    with plan(dg, c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"], None,
              **kw) as pl:
        y = torch.as_tensor(c["y"]).cuda()
        for T in (10, 30):
            mu = host(pl.solve(y, c["I0"], T))
            psnr = 10 * np.log10(c["mu"].max() ** 2 / np.mean((mu - c["mu"]) ** 2))
            assert abs(psnr - curve[T - 1]) < 0.05
