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
            assert bool(torch.isfinite(single[k]).all()), k
            assert torch.equal(mus[k], single[k]), k
        plans[1].set_cnn(nets[0])
        with pytest.raises(dg.DgampError):
            dg.solve_batched(plans, counts, I0, T)
    finally:
        for p in plans:
            p.close()
        for n in nets:
            n.close()


# ------------------------------------------- one launch per phase (Batch) --
BATCH_TUNING = dict(pj_seg=16, bp_mode=1, sino_fused=2, tv_kb=10, tv_rows=64, tv_vrows=4)
MIXED = [  # (n, views, bins, seed, I0): sizes that leave ragged tiles, regions and clusters
    (64, 30, 95, 1000, 1e4),
    (48, 13, 73, 1001, 3e4),
    (37, 8, 55, 1002, 1e5),
    (96, 17, 137, 1004, 1e5),
    (128, 40, 182, 1005, 2e4),
    (72, 11, 103, 1006, 1e4),
]


def _mixed():
    out = []
    for n, nv, nd, seed, I0 in MIXED:
        ph = synth.random_phantom(n, 5, seed)
        y = synth.poisson_counts(synth.analytic_sinogram(ph, synth.view_angles(nv), nd), I0, seed + 7)
        out.append(dict(n=n, nv=nv, nd=nd, y=y, I0=I0))
    return out


@pytest.mark.parametrize("storage,groups", [(0, 1), (1, 1), (0, 3)])
def test_batch_one_launch_per_phase_is_bit_identical_to_single_solves(dg, storage, groups):
    """dgamp_ct_batch_solve runs each phase of an iteration as one launch over
    all slices; every block runs the single-slice kernel's block body, so
    each slice must equal its own solve with the batch's implementation
    choices bit for bit (mu and the log of scalars), whether the slices run
    as one group or as three groups on parallel branches of the graph."""
    sl = _mixed()
    T = 6
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.2, damp_s=0.15, storage=storage)
    plans = [dg.Plan(s["n"], s["nv"], s["nd"], **kw) for s in sl]
    try:
        counts = [torch.as_tensor(s["y"]).cuda() for s in sl]
        I0 = [s["I0"] for s in sl]
        with dg.Batch(plans, groups=groups) as b:
            assert b.launches(T) == 1 + 6 * groups * T + 4
            mus, stats = b.solve(counts, I0, T, with_stats=True)
            mus2 = b.solve(counts, I0, T)                     # the captured graph replays the same
            torch.cuda.synchronize()
            mus = [m.clone() for m in mus]
        single, sst = [], []
        for p, c, s in zip(plans, counts, sl):
            p.set_tuning(**BATCH_TUNING)
            mu, st = p.solve(c, s["I0"], T, with_stats=True)
            single.append(mu)
            sst.append(st)
        torch.cuda.synchronize()
        for k in range(len(sl)):
            assert bool(torch.isfinite(single[k]).all()), k
            assert torch.equal(mus[k], single[k]), k
            assert torch.equal(mus2[k], single[k]), k
            assert stats[k]["iters_done"] == T
            for key in ("tau_x", "tau_p", "tau_s", "tau_r", "div"):
                assert np.array_equal(stats[k][key], sst[k][key]), (k, key)
        if storage == 0:
            s = sl[0]
            ref = gamp.ct_solve(s["y"], s["I0"], Geometry(s["n"], s["nv"], s["nd"]), T,
                                gamp.Options(c_tv=3.0, k_tv=20, damp_x=0.2, damp_s=0.15))
            assert rel(mus[0].cpu().numpy(), ref) < 1e-3
    finally:
        for p in plans:
            p.close()


def test_batch_mixed64_subset_matches_stream_pool(dg):
    """Twelve slices of the mixed 64-slice workload (256-512 pixels, 32-128
    views), 30 iterations: the batch object against the stream-pool path,
    whose plans use their own tuned implementation choices (other summation
    orders), to the 1e-3 of the solve tests."""
    batch = synth.make_batch("mixed64", count=12)
    kw = dict(c_tv=3.0, k_tv=20, damp_x=0.2, damp_s=0.15)
    plans = [dg.Plan(c["n"], c["n_views"], c["n_det"], **kw) for c in batch]
    try:
        counts = [torch.as_tensor(c["y"]).cuda() for c in batch]
        I0 = [c["I0"] for c in batch]
        T = batch[0]["iters"]
        with dg.Batch(plans) as b:
            mb = [m.cpu().numpy() for m in b.solve(counts, I0, T)]
        mp = [m.cpu().numpy() for m in dg.solve_batched(plans, counts, I0, T)]
        for k in range(len(batch)):
            assert rel(mb[k], mp[k]) < 1e-3, k
    finally:
        for p in plans:
            p.close()


def test_batch_rejects_what_it_cannot_run(dg):
    with dg.Plan(32, 5, 48, c_tv=3.0, k_tv=20) as a, dg.Plan(32, 5, 48, c_tv=3.0, k_tv=15) as b15, \
            dg.Plan(32, 5, 48, denoiser=1) as learned, dg.Plan(32, 5, 48, tv_metric=1) as metric, \
            dg.Plan(32, 5, 48, storage=1) as bf:
        for bad in ([a, a], [a, b15], [a, learned], [a, metric], [a, bf], []):
            with pytest.raises((dg.DgampError, ValueError)):
                dg.Batch(bad)
