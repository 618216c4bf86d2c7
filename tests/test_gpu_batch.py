"""Batched solves through the C ABI (dgamp_ct_solve_batched): a mix of
geometries solved concurrently must give, slice by slice, exactly the result
of the plan's own dgamp_ct_solve, and match the FP64 oracle to the same
1e-3 as a single solve."""
import numpy as np
import pytest

import synth
from oracle import gamp
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SLICES = [  # (n, views, bins, seed, I0)
    (64, 30, 95, 1000, 1e4),
    (48, 13, 73, 1001, 3e4),
    (37, 8, 55, 1002, 1e5),
    (80, 21, 116, 1003, 2e4),
]


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


def _slices():
    out = []
    for n, nv, nd, seed, I0 in SLICES:
        ph = synth.random_phantom(n, 5, seed)
        y = synth.poisson_counts(synth.analytic_sinogram(ph, synth.view_angles(nv), nd), I0, seed + 7)
        out.append(dict(n=n, nv=nv, nd=nd, y=y, I0=I0))
    return out


def test_batched_equals_single_solves_and_oracle(dg):
    sl = _slices()
    T = 5
    plans = [dg.Plan(s["n"], s["nv"], s["nd"], c_tv=3.0, k_tv=20) for s in sl]
    try:
        counts = [torch.as_tensor(s["y"]).cuda() for s in sl]
        mus, stats = dg.solve_batched(plans, counts, [s["I0"] for s in sl], T, with_stats=True)
        single = [p.solve(c, s["I0"], T) for p, c, s in zip(plans, counts, sl)]
        torch.cuda.synchronize()
        for k, s in enumerate(sl):
            assert torch.equal(mus[k], single[k]), k
            assert stats[k]["iters_done"] == T
            g = Geometry(s["n"], s["nv"], s["nd"])
            ref = gamp.ct_solve(s["y"], s["I0"], g, T, gamp.Options(c_tv=3.0, k_tv=20))
            assert rel(mus[k].cpu().numpy(), ref) < 1e-3, k
    finally:
        for p in plans:
            p.close()


def test_batched_rejects_a_repeated_plan(dg):
    s = _slices()[0]
    with dg.Plan(s["n"], s["nv"], s["nd"]) as p:
        c = torch.as_tensor(s["y"]).cuda()
        with pytest.raises(dg.DgampError):
            dg.solve_batched([p, p], [c, c], [s["I0"], s["I0"]], 2)
        with pytest.raises(dg.DgampError):
            dg.solve_batched([p], [c], [0.0], 2)


def test_learned_batch_equals_single_solves_and_rejects_a_shared_network(dg):
    """A batch of learned slices, one network per slice (same weights): every
    slice equals its own solve bit for bit; two plans sharing a network are
    rejected (a network's workspace serves one solve at a time)."""
    from oracle import cnn as ocnn
    from paper_1609_04661_gb300.binding import flatten_params
    ws, bs = ocnn.init_params(31)
    params = flatten_params(ws, bs)
    sl = _slices()[:3]
    T = 3
    nets = [dg.CNN(17) for _ in sl]
    plans = [dg.Plan(s["n"], s["nv"], s["nd"], denoiser=1, damp_x=0.5, damp_s=0.5) for s in sl]
    try:
        for net, pl in zip(nets, plans):
            net.set_params(params)
            pl.set_cnn(net)
        counts = [torch.as_tensor(s["y"]).cuda() for s in sl]
        I0 = [s["I0"] for s in sl]
        mus = dg.solve_batched(plans, counts, I0, T)
        single = [p.solve(c, i0, T) for p, c, i0 in zip(plans, counts, I0)]
        torch.cuda.synchronize()
        for k in range(len(sl)):
            assert torch.equal(mus[k], single[k]), k
        plans[1].set_cnn(nets[0])
        with pytest.raises(dg.DgampError):
            dg.solve_batched(plans, counts, I0, T)
    finally:
        for p in plans:
            p.close()
        for n in nets:
            n.close()
