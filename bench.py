#!/usr/bin/env python
"""Benchmark of the D-GAMP-CT hot path on one GB300 (or N independent replicas).

One step = one full D-GAMP-CT solve (Algorithm 1: 30 iterations of Steps 1-4
and the final mu = V^-1 x) of the 512 x 512 / 64-view / 729-bin ellipse
workload with I0 = 1e5 and the prox-TV denoiser, counts resident in HBM.
The metric is D-GAMP-CT iterations per second (whole job: all ranks).

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; L2 is flushed (a 256 MiB write) between steps,
outside the events; barrier + synchronize around the timed region; the time
is the max over ranks.  ``e2e`` repeats the measurement through the host-
buffer entry point (dgamp_ct_solve_host): counts copied in and mu copied out
inside the timed region.

Under torchrun (N > 1) every rank solves its own slice (seed 1000 + rank):
replicas only, no data-path collective.

Extra objects on the line: ``learned_vs_plain`` (the learned denoiser in the
same solve: iterations/s and PSNR per iteration of both forms),
``batched`` (the 64-slice mixed batch through dgamp_ct_solve_batched,
split largest-first across ranks) and ``ablation`` (Onsager term and
damping on and off).

``--impl reference`` times the FP64 CPU oracle instead, one iteration of the
same workload per step, on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D-GAMP-CT iters/s at 512²/64 views; A+Aᵀ GB/s; learned vs plain at equal PSNR"
UNIT = "iters/s"
WORKLOAD = "ellipse512_v64"
# the headline solve: prox-TV (c = 3, 20 Chambolle steps) with the damping
# that maximises the PSNR after the workload's 30 iterations on the training
# seeds (eta_x = 0.2, eta_s = 0.15; Section 7.2)
TV = dict(c_tv=3.0, k_tv=20, damp_x=0.2, damp_s=0.15)
# the fan-beam and the 1024 x 1024 workloads keep the damping their own
# sweeps found (0.5: the iteration converges there; with the weaker damping
# above the fan-beam solve diverges)
TV_HALF = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch, from
# ncu captures of this workload's headline plan (cold cache), valid only for
# the configuration captured and the kernels as they were then: the blocked-TV
# launches of one iteration (both images per thread, 10 steps per launch,
# 64-row regions of 2-row threads), the banded projector (32-line bands, one
# wave) and the tile back-projection.
TV_TRAFFIC = {"tv_kb": 10, "tv_rows": 64, "tv_vrows": 2, "bytes_per_iteration": 2112512 + 8421888 + 256}
A_TRAFFIC = {"form": (32, 1), "bytes_per_launch": 2145280}      # (pj_band, pj_waves), or (0, pj_seg)
AT_TRAFFIC = {"bp_mode": 1, "bytes_per_launch": 1263872}


# ----------------------------------------------------------------- helpers --
def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# FLOP of one 17-layer 64-channel 3x3 network evaluation per pixel:
# 15 hidden layers x 64 x 64 x 9 x 2 plus the 1->64 and 64->1 layers (64 x 9 x 2 each)
CNN_FLOP_PER_PIXEL = 15 * (64 * 64 * 9 * 2) + 2 * (64 * 9 * 2)


def _learned_vs_plain(dg, plan, case, counts, T, plain_iters_per_s):
    """The learned denoiser (shipped weights) in the same solve: iterations per
    second, the PSNR after t = 1..T iterations of each form, and how many
    learned iterations reach the plain form's final PSNR (None if none does)."""
    import torch
    from paper_1609_04661_gb300.train_denoiser import load_cnn
    net = load_cnn()
    mu = torch.empty((case["n"], case["n"]), device="cuda")

    def curve():
        out = []
        for t in range(1, T + 1):
            plan.solve(counts, case["I0"], t, mu_out=mu)
            out.append(_psnr(mu.cpu().numpy().astype("float64"), case["mu"]))
        return out

    plain = curve()
    plan.set_cnn(net)
    plan.set_options(denoiser=1, cnn_scale=int(net.scaled))
    try:
        for _ in range(2):
            plan.solve(counts, case["I0"], T, mu_out=mu)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(st)
        for _ in range(reps):
            plan.solve(counts, case["I0"], T, mu_out=mu)
        e1.record(st)
        torch.cuda.synchronize()
        learned_ips = reps * T / (e0.elapsed_time(e1) / 1e3)
        prof = plan.profile_iteration(reps=5)
        learned = curve()
    finally:
        plan.set_options(denoiser=0)
        plan.set_cnn(None)
        net.close()
    # the network judged by prox-TV (denoiser 2): both run every iteration
    # and the lower SURE risk estimate keeps one
    plan.set_cnn(net_j := load_cnn())
    plan.set_options(denoiser=2, cnn_scale=int(net_j.scaled))
    try:
        for _ in range(2):
            plan.solve(counts, case["I0"], T, mu_out=mu)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            plan.solve(counts, case["I0"], T, mu_out=mu)
        e1.record(st)
        torch.cuda.synchronize()
        judged_ips = reps * T / (e0.elapsed_time(e1) / 1e3)
        _, jst = plan.solve(counts, case["I0"], T, mu_out=mu, with_stats=True)
        judged = curve()
    finally:
        plan.set_options(denoiser=0)
        plan.set_cnn(None)
        net_j.close()
    peak, kind = _bf16_peak()
    flop = 2.0 * plan.N * CNN_FLOP_PER_PIXEL
    achieved = flop / (prof["cnn_pair"] * 1e-3) / 1e12
    reach = next((t + 1 for t, v in enumerate(learned) if v >= plain[-1]), None)
    reach_j = next((t + 1 for t, v in enumerate(judged) if v >= plain[-1]), None)
    return {"weights": "dncnn17_ellipse512_v64.bin (Gaussian-noise-trained, noise-level scaled, "
                       "sigma = sqrt(tau_r))",
            "learned_iters_per_s": learned_ips, "plain_iters_per_s": plain_iters_per_s,
            "plain_final_psnr_db": plain[-1], "plain_best_psnr_db": max(plain),
            "learned_final_psnr_db": learned[-1], "learned_best_psnr_db": max(learned),
            "learned_iterations_to_plain_final_psnr": reach,
            "psnr_db_plain": [round(v, 2) for v in plain], "psnr_db_learned": [round(v, 2) for v in learned],
            "judged": {"what": "denoiser 2: network and prox-TV every iteration, the lower SURE risk "
                               "estimate kept",
                       "iters_per_s": judged_ips, "final_psnr_db": judged[-1], "best_psnr_db": max(judged),
                       "iterations_to_plain_final_psnr": reach_j,
                       "network_kept_iterations": int(jst["learned_kept"]),
                       "psnr_db": [round(v, 2) for v in judged]},
            "kernel_ms": prof,
            "cnn_roofline": {"kernel": "CNN pair (2 images, 17 layers)", "bound": "tensor",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                             "peak_kind": f"{kind} cuBLAS bf16 burst",
                             "algorithmic_flop_per_iteration": flop}}


def _training(dg, steps: int = 20):
    """One Adam step of the 17-layer network on a batch of 32 patches of 64 x 64
    (the training batch of train_denoiser.py): forward, backward (data and
    weight gradients of every layer) and the update, timed with CUDA events on
    the launching stream.  Synthetic patches; the loss is read back each step
    as training does."""
    import numpy as np
    import torch
    B, H, W = 32, 64, 64
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 1.0, (B, H, W)).astype(np.float32)
    sig = np.exp(rng.uniform(np.log(0.005), np.log(0.1), B)).astype(np.float32)
    r = (x + sig[:, None, None] * rng.standard_normal((B, H, W))).astype(np.float32)
    rt, xt = torch.as_tensor(r).cuda(), torch.as_tensor(x).cuda()
    with dg.CNN(17, seed=3) as net:
        for _ in range(3):
            net.train_step(rt, xt, sig, 1e-4)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            net.train_step(rt, xt, sig, 1e-4)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    # forward, data gradient and weight gradient of the hidden layers, plus the end layers
    flop = 3.0 * B * H * W * CNN_FLOP_PER_PIXEL
    peak, kind = _bf16_peak()
    achieved = flop / (ms * 1e-3) / 1e12
    return {"workload": f"17-layer 64-channel network, {B} patches of {H}x{W}, Adam, loss read back each step",
            "ms_per_step": ms, "patches_per_s": B / (ms * 1e-3), "flop_per_step": flop,
            "tflops": achieved, "frac_of_bf16_peak": achieved / peak, "peak_kind": f"{kind} cuBLAS bf16 burst",
            "note": "64-wide patches fill half of each 128-pixel strip of the tensor-core kernels"}


def _ablation(plan, case, counts, T):
    """PSNR after t = 1..T iterations with and without the Onsager term and
    the damping (Sections 7.1 and 7.2), on the benchmark slice; and with the
    stronger damping eta = 0.5, which peaks early (near iteration 8) and
    then turns over."""
    import torch
    mu = torch.empty((case["n"], case["n"]), device="cuda")
    out = {}
    dx, ds = TV["damp_x"], TV["damp_s"]
    for name, ons, damp in [("onsager_damped", 1, (dx, ds)), ("onsager_undamped", 1, (1.0, 1.0)),
                            ("no_onsager_damped", 0, (dx, ds)), ("no_onsager_undamped", 0, (1.0, 1.0)),
                            ("onsager_damped_0.5", 1, (0.5, 0.5))]:
        plan.set_options(onsager=ons, damp_x=damp[0], damp_s=damp[1])
        curve = []
        for t in range(1, T + 1):
            plan.solve(counts, case["I0"], t, mu_out=mu)
            curve.append(_psnr(mu.cpu().numpy().astype("float64"), case["mu"]))
        best = max(range(T), key=lambda k: curve[k])
        out[name] = {"damp_x": damp[0], "damp_s": damp[1], "psnr_db_final": round(curve[-1], 2),
                     "psnr_db_best": round(curve[best], 2), "best_at_iteration": best + 1,
                     "psnr_db_at_10": round(curve[9], 2) if T >= 10 else None,
                     "psnr_db_curve": [round(v, 2) for v in curve]}
    plan.set_options(onsager=1, damp_x=TV["damp_x"], damp_s=TV["damp_s"])
    # the output step with the exact posterior moments instead of Laplace's
    # (Appendix A; the paper puts the difference at about 0.1 dB)
    try:
        out["exact_moments_damped"] = _exact_moments_curve(plan, case, counts, T, mu)
    except Exception as e:                      # an ablation entry never takes the bench line down
        out["exact_moments_damped"] = {"error": f"{type(e).__name__}: {e}"}
    finally:
        plan.set_options(output_moments=0)
    return out


def _exact_moments_curve(plan, case, counts, T, mu):
    import torch
    plan.set_options(output_moments=1)
    curve = []
    for t in range(1, T + 1):
        plan.solve(counts, case["I0"], t, mu_out=mu)
        curve.append(_psnr(mu.cpu().numpy().astype("float64"), case["mu"]))
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    plan.solve(counts, case["I0"], T, mu_out=mu)
    e1.record(st)
    torch.cuda.synchronize()
    best = max(range(T), key=lambda k: curve[k])
    return {"psnr_db_final": round(curve[-1], 2), "psnr_db_best": round(curve[best], 2),
            "best_at_iteration": best + 1, "psnr_db_at_10": round(curve[9], 2) if T >= 10 else None,
            "iters_per_s": T / (e0.elapsed_time(e1) * 1e-3)}


def _batched(dg, rank, world, dist, flush, steps, learned=False):
    """The 64-slice mixed batch (n in {256, 384, 512}, 32-128 views) through
    dgamp_ct_solve_batched; under torchrun each rank takes its largest-first
    share of the slices (strong scaling: the batch is fixed).  learned: the
    shipped network as denoiser, one network object per slice."""
    import numpy as np
    import torch
    import synth
    batch = synth.make_batch("mixed64")
    T = batch[0]["iters"]
    work = np.array([c["n_views"] * c["n_det"] * c["n"] for c in batch], dtype=np.int64)
    owner, _ = dg.schedule_lpt(work, world)
    mine = [c for c, q in zip(batch, owner) if q == rank]
    plans = [dg.Plan(c["n"], c["n_views"], c["n_det"], **TV) for c in mine]
    nets = []
    if learned:
        from paper_1609_04661_gb300.train_denoiser import load_cnn
        for p in plans:
            net = load_cnn()
            p.set_cnn(net)
            p.set_options(denoiser=1, cnn_scale=int(net.scaled))
            nets.append(net)
    counts = [torch.as_tensor(c["y"]).cuda() for c in mine]
    I0 = [c["I0"] for c in mine]
    mus = [torch.empty((c["n"], c["n"]), device="cuda") for c in mine]
    st = torch.cuda.current_stream()
    for _ in range(2):
        dg.solve_batched(plans, counts, I0, T, mu_out=mus)
    torch.cuda.synchronize()

    def timed(fn):
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([total], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total = float(t.item())
        return total / steps

    ms = timed(lambda: dg.solve_batched(plans, counts, I0, T, mu_out=mus))

    def serial():
        for p, c, i0, m in zip(plans, counts, I0, mus):
            p.solve(c, i0, T, mu_out=m)

    ms_serial = timed(serial)
    launches = sum(p.solve_launches(T) for p in plans)
    phase = None
    if not learned:
        # the same slices with every phase of an iteration as one launch over
        # all of them (dgamp_ct_batch_*), the iteration graph-captured once
        # (groups = 1), and split into groups whose launches run on parallel
        # graph branches
        runs = {}
        for groups in sorted({1, 2, 4, 8, 16, len(mine)}):
            with dg.Batch(plans, groups=groups) as bobj:
                for _ in range(2):
                    bobj.solve(counts, I0, T, mu_out=mus)
                torch.cuda.synchronize()
                ms_g = timed(lambda: bobj.solve(counts, I0, T, mu_out=mus))
                runs[groups] = {"ms_per_batch": ms_g, "iters_per_s": len(batch) * T / (ms_g / 1e3),
                                "slices_per_s": len(batch) / (ms_g / 1e3),
                                "gpu_launches_per_batch_rank0": bobj.launches(T),
                                "speedup_vs_stream_pool": ms / ms_g}
        best = min((g for g in runs if g > 1), key=lambda g: runs[g]["ms_per_batch"])
        phase = dict(runs[1], tuning="pj_seg 16, tile back-projection, cluster sinogram step, 10 TV steps per launch",
                     grouped=dict(runs[best], groups=best),
                     all_groups={str(g): round(r["iters_per_s"], 1) for g, r in runs.items()})
    for p in plans:
        p.close()
    for net in nets:
        net.close()
    return {"workload": "mixed64: 64 slices, n in {256,384,512}, views in {32,48,64,96,128}, bins ceil(1.42 n), "
                        "log10 I0 ~ U(4,6), 10 ellipses + rectangle each (seed 3000), 30 iterations, "
                        + ("learned denoiser (one network per slice)" if learned else "prox-TV"),
            "slices": len(batch), "iters_per_slice": T, "scaling": "strong",
            "ms_per_batch": ms, "iters_per_s": len(batch) * T / (ms / 1e3),
            "slices_per_s": len(batch) / (ms / 1e3),
            "one_stream_ms_per_batch": ms_serial, "concurrency_speedup": ms_serial / ms,
            "one_launch_per_phase": phase,
            "joseph_steps_per_batch": int(work.sum()), "gpu_launches_per_batch_rank0": int(launches)}


def _gpu_ms(fn, reps: int):
    """Mean CUDA-event time of fn() over reps calls on the current stream."""
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _variants(dg, plan, case, counts, T):
    """The paper's variants beyond the headline form (skipped with --no-variants).

    tv_metric: the headline solve with the prox-TV in the (V^T V)^{-1} norm
    (Section 6.3), its PSNR curve and iterations/s.  fan512_v102: the
    flat-detector fan-beam workload (Section 6 geometry, damping 0.5):
    plan time (||Phi~||_F^2 ray by ray), iterations/s, PSNR, and A
    and A^T alone with their compulsory bytes 4 (N + M) per launch."""
    import time
    import numpy as np
    import torch
    import synth
    out = {}
    mu = torch.empty((case["n"], case["n"]), device="cuda")
    try:
        plan.set_options(tv_metric=1)
        curve = []
        for t in range(1, T + 1):
            plan.solve(counts, case["I0"], t, mu_out=mu)
            curve.append(_psnr(mu.cpu().numpy().astype("float64"), case["mu"]))
        ms = _gpu_ms(lambda: plan.solve(counts, case["I0"], T, mu_out=mu), 1)
        out["tv_metric_damped"] = {"psnr_db_final": round(curve[-1], 2), "psnr_db_best": round(max(curve), 2),
                                   "psnr_db_at_5": round(curve[4], 2) if T >= 5 else None,
                                   "iters_per_s": T / (ms * 1e-3)}
    except Exception as e:                      # a variant never takes the bench line down
        out["tv_metric_damped"] = {"error": f"{type(e).__name__}: {e}"}
    finally:
        plan.set_options(tv_metric=0)
    try:
        c = synth.make_case("fan512_v102")
        f = c["fan"]
        n, nv, nd, Tf = c["n"], c["n_views"], c["n_det"], c["iters"]
        t0 = time.perf_counter()
        fp = dg.Plan(n, nv, nd, fan=f, **TV_HALF)
        plan_s = time.perf_counter() - t0
        y = torch.as_tensor(c["y"]).cuda()
        fmu = torch.empty((n, n), device="cuda")
        fp.solve(y, c["I0"], Tf, mu_out=fmu)                     # warm-up, graph capture
        ms = _gpu_ms(lambda: fp.solve(y, c["I0"], Tf, mu_out=fmu), 3)
        x = torch.rand((n, n), device="cuda")
        sino = torch.rand((nv, nd), device="cuda")
        img = torch.empty((n, n), device="cuda")
        zs = torch.empty((nv, nd), device="cuda")
        fp.project(x, out=zs)
        fp.backproject(sino, out=img)
        a_ms = _gpu_ms(lambda: fp.project(x, out=zs), 10)       # includes the image staging
        at_ms = _gpu_ms(lambda: fp.backproject(sino, out=img), 10)
        byts = 4.0 * (n * n + nv * nd)
        out["fan512_v102"] = {"iters_per_s": Tf / (ms * 1e-3), "iterations": Tf,
                              "psnr_db": round(_psnr(fmu.cpu().numpy().astype("float64"), c["mu"]), 2),
                              "plan_s": plan_s, "frob_sq": fp.frob_sq,
                              "project_ms": a_ms, "backproject_ms": at_ms,
                              "project_gbs": byts / (a_ms * 1e-3) / 1e9, "backproject_gbs": byts / (at_ms * 1e-3) / 1e9,
                              "kernel_ms": fp.profile_iteration(reps=3)}
        fp.close()
    except Exception as e:
        out["fan512_v102"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def _c5(dg):
    """The large mixed-precision workload: 128 slices of 1024 x 1024, 90 views,
    1449 bins, I0 = 1e5, sinograms and projector images in BF16 (storage = 1),
    learned denoiser judged by prox-TV (denoiser 2: both every iteration, the
    lower SURE risk estimate kept, the network only while 0 < D' < M/N),
    30 iterations; solved in groups of 8 concurrent slices (8 plans and 8
    networks reused).  Precision, on the last group's 8 slices: the relative
    error against the phantom of the BF16-storage and FP32-storage results,
    for the judged learned form (30 iterations) and for prox-TV alone (10 and
    30 iterations; at 90 views of 1024 x 1024 the scalar-variance iteration
    stops improving after about 10, so both are reported)."""
    import numpy as np
    import torch
    import synth
    from paper_1609_04661_gb300.train_denoiser import load_cnn
    batch = synth.make_batch("large128")
    c0 = batch[0]
    n, nv, nd, T = c0["n"], c0["n_views"], c0["n_det"], c0["iters"]
    G = 8
    nets = [load_cnn() for _ in range(G)]
    plans = [dg.Plan(n, nv, nd, storage=1, **TV_HALF) for _ in range(G)]
    for p, net in zip(plans, nets):
        p.set_cnn(net)
        p.set_options(denoiser=2, cnn_scale=int(net.scaled))
    counts = [torch.as_tensor(c["y"]).cuda() for c in batch]
    I0 = [c["I0"] for c in batch]
    mus = [torch.empty((n, n), device="cuda") for _ in range(G)]

    def run(g0, g1):
        for g in range(g0, g1, G):
            dg.solve_batched(plans, counts[g:g + G], I0[g:g + G], T, mu_out=mus)

    run(0, G)   # warm-up: graphs captured, workspaces sized
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    run(0, len(batch))
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    last = list(range(len(batch) - G, len(batch)))
    truth = [synth.rasterise(batch[k]["phantom"], n) for k in last]

    def err(img, k):
        a = img.cpu().numpy().astype(np.float64) if hasattr(img, "cpu") else img
        return round(float(np.linalg.norm(a - truth[k]) / np.linalg.norm(truth[k])), 4)

    learned = {"bf16": [err(mus[k], k) for k in range(G)]}
    for p in plans:
        p.set_options(storage=0)
    run(last[0], len(batch))
    learned["fp32"] = [err(mus[k], k) for k in range(G)]
    for p in plans:
        p.close()
    for net in nets:
        net.close()
    tv = {}
    for iters in (10, T):
        for stg, name in ((0, "fp32"), (1, "bf16")):
            with dg.Plan(n, nv, nd, storage=stg, **TV_HALF) as pl:
                tv[f"{name}_{iters}it"] = [err(pl.solve(counts[k], I0[k], iters), i) for i, k in enumerate(last)]
    return {"workload": "large128: 128 slices of 1024x1024, 10 seeded ellipses each (seed 3000, rho_max 0.01), "
                        "90 views, 1449 bins, I0=1e5, 30 iterations, damping 0.5, BF16 sinogram and projector-image storage, "
                        "FP32 sums, FP64 GAMP scalars, learned denoiser judged by prox-TV (denoiser 2), groups of 8 "
                        "concurrent slices",
            "slices": len(batch), "ms_per_batch": ms, "iters_per_s": len(batch) * T / (ms / 1e3),
            "slices_per_s": len(batch) / (ms / 1e3),
            "rel_error_vs_phantom_slices_120_127": {"learned_judged_30it": learned, "tv": tv}}


def _config(n_gpus):
    from synth import CASES
    n, nv, nd, ne, rmax, rect, I0, iters = CASES[WORKLOAD]
    return {"workload": f"{WORKLOAD}: {n}x{n} image of {ne} seeded random ellipses + rectangle object, "
                        f"parallel beam, {nv} views over 180 deg, {nd} detector bins, Poisson I0={I0:g}, "
                        f"{iters} iterations, prox-TV denoiser (K={TV['k_tv']}, c={TV['c_tv']}), damping eta_x={TV['damp_x']}, eta_s={TV['damp_s']}",
            "image": n, "views": nv, "detector_bins": nd, "I0": I0, "iters_per_step": iters,
            "l2": "flushed between steps (256 MiB write, outside the timed events)",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU"}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _psnr(mu, ref):
    import numpy as np
    mse = float(np.mean((mu - ref) ** 2))
    return 10.0 * math.log10(float(ref.max()) ** 2 / mse) if mse > 0 else float("inf")


# ------------------------------------------------------- oracle (CPU) leg --
def _oracle_sample(iters: int, warm: int, seed: int, ready=None):
    """Run the FP64 oracle on the workload; returns per-iteration seconds and
    the monotonic-clock stamps of the first and last timed iteration's ends.
    ready(), if given, is called after the set-up and before the solve."""
    import numpy as np  # noqa: F401
    import synth
    from oracle import gamp, precond
    from oracle.geometry import Geometry
    c = synth.make_case(WORKLOAD, seed=seed)
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    frob2 = precond.frobenius_sq(g)
    if ready is not None:
        ready()
    stamps = [time.monotonic()]
    gamp.ct_solve(c["y"], c["I0"], g, warm + iters, gamp.Options(**TV), frob2=frob2,
                  on_iter=lambda t, x: stamps.append(time.monotonic()))
    d = [b - a for a, b in zip(stamps[:-1], stamps[1:])]
    return {"per_iter": d[warm:], "t0": stamps[warm], "t1": stamps[-1]}


_ORACLE_ENV = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")


def _run_oracle_subprocess(iters: int, warm: int, seed: int = 1000):
    env = dict(os.environ, **_ORACLE_ENV)
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench._oracle_sample({iters}, {warm}, {seed})))")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])["per_iter"]


def _host_cores():
    """CPUs this process may run on (its affinity mask), not the machine's count."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _run_oracle_all_cores(iters: int, warm: int):
    """The same oracle sample on every host core at once, one single-threaded
    process per core on its own slice (seeds 1000 + k): the host's aggregate
    iterations/s when it solves independent slices in parallel.  Every child
    finishes its set-up, reports ready and waits for one shared start signal,
    so the timed loops overlap; the rate is all timed iterations over the span
    from the first timed start to the last timed end."""
    cores = _host_cores()
    env = dict(os.environ, **_ORACLE_ENV)
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"go = lambda: (print('READY', flush=True), sys.stdin.readline()); "
            f"print(json.dumps(bench._oracle_sample({iters}, {warm}, 1000 + int(sys.argv[1]), ready=go)))")
    procs = [subprocess.Popen([sys.executable, "-c", code, str(k)], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for k in range(cores)]
    for pr in procs:                                   # every child has finished its set-up
        line = pr.stdout.readline()
        if line.strip() != "READY":
            err = pr.stderr.read()
            for q in procs:
                q.kill()
            raise RuntimeError(f"oracle child failed before its timed loop: {line!r} {err[-2000:]}")
    for pr in procs:                                   # one start signal for all
        pr.stdin.write("go\n")
        pr.stdin.flush()
    results = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        results.append(json.loads(out.strip().splitlines()[-1]))
    total = sum(len(r["per_iter"]) for r in results)
    span = max(r["t1"] for r in results) - min(r["t0"] for r in results)
    return {"value": total / span, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{iters} timed iterations (after {warm}) of the {WORKLOAD} solve on each of {cores} slices "
                      f"(seeds 1000..{999 + cores}), one single-threaded FP64 numpy process per core, set-up done "
                      f"before one shared start signal; value = all timed iterations / the span from the first "
                      f"timed start to the last timed end; host CPU {_cpu_model()}"}


# Arm CPU part numbers (MIDR implementer 0x41) of the server cores this may run on
_ARM_PARTS = {0xd0c: "Arm Neoverse N1", 0xd40: "Arm Neoverse V1", 0xd49: "Arm Neoverse N2",
              0xd4f: "Arm Neoverse V2"}


def _cpu_model():
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except Exception:
        pass
    if "model name" in fields:
        return fields["model name"]
    part, impl = fields.get("cpu part"), fields.get("cpu implementer")
    if part:
        try:
            name = _ARM_PARTS.get(int(part, 16)) if impl and int(impl, 16) == 0x41 else None
        except ValueError:
            name = None
        return f"{name} ({impl}/{part})" if name else f"implementer {impl}, part {part}"
    return "unknown"


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    per_iter = _run_oracle_subprocess(args.steps, args.warmup)
    tot = sum(per_iter)
    value = len(per_iter) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(per_iter),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(_config(1), step="one D-GAMP-CT iteration of the workload"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed iterations (after {args.warmup}) of the "
                                       f"{WORKLOAD} solve, FP64 numpy oracle, one thread, "
                                       f"||Phi~||_F^2 precomputed; host CPU {_cpu_model()}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_all_cores": _run_oracle_all_cores(args.steps, args.warmup)}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU leg ----
def run_gpu(args):
    import numpy as np
    import torch
    import synth
    import paper_1609_04661_gb300 as dg
    from paper_1609_04661_gb300 import build as _build

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    dg.load()

    case = synth.make_case(WORKLOAD, seed=1000 + rank)
    T = case["iters"]
    plan = dg.Plan(case["n"], case["n_views"], case["n_det"], **TV)
    if args.tuning:
        # pin implementation choices (e.g. to profile the configuration the
        # plan-time timing picks when run without a profiler)
        plan.set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))})
    counts = torch.as_tensor(case["y"]).cuda()
    mu = torch.empty((case["n"], case["n"]), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.solve(counts, case["I0"], T, mu_out=mu)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(st)
        plan.solve(counts, case["I0"], T, mu_out=mu)
        ev[k][1].record(st)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps * T / (ms / 1e3)

    mu_h = mu.cpu().numpy().astype(np.float64)
    psnr = _psnr(mu_h, case["mu"])

    # e2e: host buffers through dgamp_ct_solve_host
    pin_c = torch.as_tensor(case["y"]).pin_memory()
    pin_mu = torch.empty((case["n"], case["n"]), dtype=torch.float32).pin_memory()
    c_np, mu_np = pin_c.numpy(), pin_mu.numpy()
    plan.solve_host(c_np, case["I0"], T, mu_out=mu_np)
    if dist is not None:
        dist.barrier()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.solve_host(c_np, case["I0"], T, mu_out=mu_np)
        e2e_s += time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * args.steps * T / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(c_np.nbytes), "d2h_bytes_per_step": int(mu_np.nbytes)}

    # per-kernel durations of one iteration, CUDA events on the launching stream
    prof = plan.profile_iteration(reps=10)
    iter_ms = sum(prof.values())
    hbm, peak_kind = _peaks()
    N, M = plan.N, plan.M
    # compulsory bytes per launch (FP32 images/sinograms, float2 TV duals, two images in the denoiser)
    algo = {"project": 4 * (N + M), "filter_z": 8 * M, "output_step": 16 * M, "filter_s": 8 * M,
            "sino_step": 20 * M,
            "backproject_update": 4 * (M + 2 * N), "probe_input": 8 * N,
            "tv_block_final": 8 * N + 16 * N + 16 * N}
    for kname in prof:
        if kname.startswith("tv_block") and kname != "tv_block_final":
            algo[kname] = 8 * N + 16 * N + (0 if kname == "tv_block0" else 16 * N)
    tv_ms = sum(v for k, v in prof.items() if k.startswith("tv_block"))
    shares = {k: v / iter_ms for k, v in prof.items()}
    # Dominant kernel = the blocked TV kernel (all its launches of one iteration).
    # The 512^2 working set is L2-resident, so it is bound by FP32 issue, not HBM:
    # algorithmic FLOP = 19 per Chambolle pixel-step (q: 3 adds, a scaled r, 1 sub;
    # grad: 2 subs; |grad|: 2 mul + add + sqrt; 1 + tau|g|: 2; p: 2 x (fma + div))
    # x K_TV steps x 2 images x N, plus 5 per pixel and image for x = r - lambda div p.
    # Peak = 152 SMs x 128 FP32 lanes x 2 FLOP x the median SM clock sampled here.
    tv_launches = [k for k in prof if k.startswith("tv_block")]
    tun = plan.tuning()
    traffic = (TV_TRAFFIC["bytes_per_iteration"] if TV_TRAFFIC is not None and
               (tun["tv_kb"], tun["tv_rows"], tun["tv_vrows"]) ==
               (TV_TRAFFIC["tv_kb"], TV_TRAFFIC["tv_rows"], TV_TRAFFIC["tv_vrows"]) else None)
    tv_flop = (19.0 * TV["k_tv"] * 2 + 5.0 * 2) * N
    # ALU peak: the library's FP32 FMA microbenchmark, measured here (TFLOP/s,
    # an FMA = 2 FLOP); the unit-count figure at the sampled clock beside it
    fp32_peak, sms = dg.binding.measure_fp32_peak(5)
    fp32x2_peak, _ = dg.binding.measure_fp32x2_peak(5)   # packed pairs: issue slots, not FMA rate
    clk_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_derived = sms * 128 * 2 * clk_mhz * 1e6 / 1e12
    peak_note = (f"FP32 FMA microbenchmark (dgamp_ct_measure_fp32_peak) in this run on {sms} SMs; "
                 f"unit-count figure {sms} SMs x 128 lanes x 2 FLOP x {clk_mhz:.0f} MHz = {alu_derived:.1f}")
    tv_tflops = tv_flop / (tv_ms * 1e-3) / 1e12
    tv_bytes = sum(algo[k] for k in tv_launches)
    roof = {"kernel": f"k_tv_steps ({len(tv_launches)} launches per iteration, KB={tun['tv_kb']}, "
                                f"{tun['tv_rows'] if tun['tv_vrows'] == 4 else 64} region rows, "
                                f"{tun['tv_vrows']} rows per thread)", "bound": "alu",
            "achieved": tv_tflops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tv_tflops / fp32_peak,
            "traffic": traffic,
            "traffic_note": "DRAM bytes of the TV launches of one iteration (ncu, cold cache), null unless the "
                            "plan chose the profiled configuration",
            "peak_kind": "measured: " + peak_note, "peak_derived": alu_derived,
            "algorithmic_flop_per_iteration": tv_flop, "launch_ms_per_iteration": tv_ms,
            "hbm_view": {"algorithmic_bytes_per_iteration": tv_bytes,
                         "achieved_gbs": tv_bytes / (tv_ms * 1e-3) / 1e9, "peak_gbs": hbm,
                         "peak_kind": f"{peak_kind} copy bandwidth"}}
    # A and A^T: Joseph ray steps (2 taps, 2 FMA = 4 FLOP each), against the
    # same FMA peak; and their compulsory bytes against HBM (the working set
    # sits in L2 at this size, so the HBM fraction stays small by nature)
    steps = float(case["n_views"]) * case["n_det"] * case["n"]

    def joseph_roof(kname, label, byts, traffic):
        ms_k = prof[kname]
        tfl = 4.0 * steps / (ms_k * 1e-3) / 1e12
        return {"kernel": label, "bound": "alu", "achieved": tfl, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": tfl / fp32_peak, "traffic": traffic, "peak_kind": "measured: " + peak_note,
                "ray_steps_per_launch": steps, "ray_steps_per_s": steps / (ms_k * 1e-3),
                "launch_ms": ms_k,
                "hbm_view": {"algorithmic_bytes_per_launch": byts, "achieved_gbs": byts / (ms_k * 1e-3) / 1e9,
                             "peak_gbs": hbm, "frac": byts / (ms_k * 1e-3) / 1e9 / hbm,
                             "peak_kind": f"{peak_kind} copy bandwidth"}}

    a_form = (tun["pj_band"], tun["pj_waves"]) if tun["pj_band"] else (0, tun["pj_seg"])
    if not tun["pj_band"]:
        a_label = f"k_project (A, {tun['pj_seg']} step segments)"
    elif tun["sino_fused"] == 2:
        a_label = (f"k_project_band (A as {tun['pj_band']}-line band partials, {tun['pj_waves']} wave(s); "
                   "the cluster sinogram kernel adds them)")
    else:
        a_label = f"k_project_band + k_band_sum (A, {tun['pj_band']}-line bands, {tun['pj_waves']} wave(s))"
    roof_a = joseph_roof("project", a_label, algo["project"],
                         A_TRAFFIC["bytes_per_launch"] if a_form == A_TRAFFIC["form"] else None)
    roof_at = joseph_roof("backproject_update",
                          "k_backproject_tile (A^T + update)" if tun["bp_mode"] == 1 else "k_backproject (A^T + update)",
                          algo["backproject_update"],
                          AT_TRAFFIC["bytes_per_launch"] if tun["bp_mode"] == AT_TRAFFIC["bp_mode"] else None)
    a_at_bytes = algo["project"] + algo["backproject_update"]
    a_at_ms = prof["project"] + prof["backproject_update"]
    learned = None
    if rank == 0 and not args.no_learned:
        learned = _learned_vs_plain(dg, plan, case, counts, T, value / world)
    batched = None if args.no_batched else _batched(dg, rank, world, dist, flush, 3)
    c5 = _c5(dg) if (not args.no_c5 and rank == 0) else None
    batched_learned = None if (args.no_batched or args.no_learned) else _batched(dg, rank, world, dist, flush, 1,
                                                                                   learned=True)
    ablation = _ablation(plan, case, counts, T) if rank == 0 and not args.no_learned else None
    training = _training(dg) if rank == 0 and not args.no_learned else None
    variants = _variants(dg, plan, case, counts, T) if (not args.no_variants and rank == 0) else None

    line = None
    if rank == 0:
        cpu = cpu_all = None
        if world == 1 and not args.no_cpu_baseline:
            per_iter = _run_oracle_subprocess(args.cpu_iters, 0)
            cpu = {"value": len(per_iter) / sum(per_iter), "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{len(per_iter)} of {T} iterations of the {WORKLOAD} solve (seed 1000), FP64 "
                             f"numpy oracle on one host thread ({_cpu_model()}), ||Phi~||_F^2 precomputed"}
            cpu_all = _run_oracle_all_cores(args.cpu_iters, 0)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _config(world), "roofline": roof, "cpu_baseline": cpu, "cpu_all_cores": cpu_all, "e2e": e2e,
                "clocks": clocks, "gpu_launches": int(args.steps * plan.solve_launches(T)),
                "psnr_db": psnr,
                "a_plus_at_gbs": a_at_bytes / (a_at_ms * 1e-3) / 1e9,
                "roofline_A": roof_a, "roofline_AT": roof_at, "fp32_fma_peak_tflops": fp32_peak,
                "fp32x2_fma_peak_tflops": fp32x2_peak,
                "iteration_ms": iter_ms, "tuning": tun, "kernel_ms": prof, "kernel_share": shares,
                "tv_share": tv_ms / iter_ms, "learned_vs_plain": learned, "batched": batched, "batched_learned": batched_learned, "large_bf16": c5,
                "ablation": ablation, "variants": variants, "training": training}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain section")
    ap.add_argument("--no-batched", action="store_true", help="skip the mixed-batch section")
    ap.add_argument("--no-c5", action="store_true", help="skip the 128-slice 1024x1024 BF16-storage workload (~1 min)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the (V^T V)^-1-norm prox-TV and the fan-beam workload")
    ap.add_argument("--tuning", default="", help="pin the headline plan's tuning, e.g. bp_mode=1,tv_kb=10")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
