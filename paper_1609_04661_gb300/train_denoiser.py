"""Train the learned D-GAMP-CT denoiser (GPU).

Two training sets, both built from training phantoms (seeds 2000 + k) in the
preconditioned space x_true = V mu_true (Eq. precondAMP):

* ``iterates`` (default): (r^t, x_true) pairs where r^t is the denoiser input
  of iteration t of a damped solve, with the noise level the solve reports,
  sigma = sqrt(tau_r^t); the network is told sigma (D_sigma(r) = r - sigma
  f(r / sigma)) and runs inside the solve with option cnn_scale = 1.  Round 1
  harvests prox-TV solves; each later round adds the iterates of solves with
  the network trained so far (whose trajectory differs) and trains on.
  ``--blind``: sigma = 1 instead.
* ``awgn``: the denoising problem that AMP poses, r = x + N(0, sigma^2)
  (the decoupling property behind Eq. MC_SURE), with sigma log-uniform.

Every array operation runs in the library's kernels through the C ABI (the
solve and its trace, V, the forward/backward passes and Adam); torch draws
the Gaussian noise of the awgn set and numpy the patch positions.

    python -m paper_1609_04661_gb300.train_denoiser --out weights.bin

Weight file: 8-byte magic b"DGCTCNN1", int32 layers, int32 flags (bit 0:
noise-level-scaled network, run it with options.cnn_scale = 1), int64
parameter count, uint32 CRC-32 of the parameter bytes, uint32 reserved, then
the float32 parameters in the library's flat order.
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import sys
import time
import zlib

import numpy as np

MAGIC = b"DGCTCNN1"
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "dncnn17_ellipse512_v64.bin")
PLAIN = dict(c_tv=3.0, k_tv=20, damp_x=0.5, damp_s=0.5)
WORKLOAD = ["ellipse512_v64"]   # the harvesting and evaluation workload (--workload)


def save_weights(path: str, params: np.ndarray, layers: int, scaled: bool) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    raw = p.tobytes()
    hdr = MAGIC + struct.pack("<iiqII", layers, 1 if scaled else 0, p.size, zlib.crc32(raw) & 0xFFFFFFFF, 0)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "wb") as f:
        f.write(hdr)
        f.write(raw)


def load_weights(path: str = DEFAULT_WEIGHTS):
    """Returns (layers, params float32, scaled); raises on a bad magic, size or checksum."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError(f"{path}: not a D-GAMP-CT CNN weight file")
    layers, flags, count, crc, _ = struct.unpack("<iiqII", data[8:32])
    raw = data[32:]
    if len(raw) != 4 * count or (zlib.crc32(raw) & 0xFFFFFFFF) != crc:
        raise ValueError(f"{path}: corrupt weight file")
    return layers, np.frombuffer(raw, dtype=np.float32).copy(), bool(flags & 1)


def load_cnn(path: str = DEFAULT_WEIGHTS):
    """A library CNN object holding the weights stored at `path`; ``net.scaled``
    tells whether it expects options.cnn_scale = 1."""
    from .binding import CNN
    layers, params, scaled = load_weights(path)
    net = CNN(layers)
    net.set_params(params)
    net.scaled = scaled
    return net


def harvest(n_phantoms: int, iters: int, patches_per_iter: int, patch: int, seed0: int = 2000,
            workload: str | None = None, scaled: bool = True, net=None, rng_seed: int = 7,
            max_mse: float = 1.0):
    """(r patches, x_true patches, sigma, diagnostics) on the GPU from damped
    solves of training phantoms: r^t is the denoiser input of iteration t
    and x_true = V mu_true.

    sigma = sqrt(tau_r^t) as GAMP reports it (scaled=True, the noise level
    the solve will hand the network), or 1 for a blind network.  GAMP's
    tau_r does not track the actual error of r^t on this operator (it runs
    far above it in the first iterations and below it later), so pairs from
    the method's own iterates teach the network what the reported level
    means along the trajectory.  net: harvest from solves with that network
    as the denoiser (noise-level scaled) instead of prox-TV.
    diagnostics: per iteration, the mean over phantoms of tau_r^t and of the
    actual mean squared error of r^t.  Iterates whose actual mean squared
    error exceeds max_mse (a solve that has diverged) are not harvested."""
    import torch
    import synth
    from .binding import Plan
    rng = np.random.default_rng(rng_seed)
    rs, xs, sg = [], [], []
    tau_tab, err_tab = np.zeros(iters), np.zeros(iters)
    plan = None
    for k in range(n_phantoms):
        c = synth.make_case(workload or WORKLOAD[0], seed=seed0 + k)
        if plan is None:
            opts = dict(PLAIN)
            if net is not None:
                opts.update(denoiser=1, cnn_scale=1)
            plan = Plan(c["n"], c["n_views"], c["n_det"], **opts)
            if net is not None:
                plan.set_cnn(net)
        y = torch.as_tensor(c["y"]).cuda()
        _, rt, tau_r = plan.solve_trace(y, c["I0"], iters)
        xt = plan.precond_image(torch.as_tensor(c["mu"], dtype=torch.float32).cuda(), inverse=False)
        n = c["n"]
        for t in range(iters):
            err = float(((rt[t] - xt) ** 2).mean())
            tau_tab[t] += tau_r[t] / n_phantoms
            err_tab[t] += err / n_phantoms
            if not (np.isfinite(tau_r[t]) and tau_r[t] > 0 and np.isfinite(err) and err <= max_mse):
                continue
            for _ in range(patches_per_iter):
                i, j = rng.integers(0, n - patch + 1, size=2)
                rs.append(rt[t, i:i + patch, j:j + patch])
                xs.append(xt[i:i + patch, j:j + patch])
                sg.append(np.sqrt(tau_r[t]) if scaled else 1.0)
    if net is not None:
        plan.set_cnn(None)
    plan.close()
    diag = {"tau_r": [float(f"{v:.3g}") for v in tau_tab], "mse_r": [float(f"{v:.3g}") for v in err_tab]}
    return torch.stack(rs).contiguous(), torch.stack(xs).contiguous(), np.asarray(sg, dtype=np.float32), diag


def psnr_curve(net, iters: int, seed: int = 1000, workload: str | None = None):
    """PSNR of mu after t = 1..iters damped iterations on one slice, with the
    network (noise-level scaled) or, for net=None, prox-TV."""
    import torch
    import synth
    from .binding import Plan
    c = synth.make_case(workload or WORKLOAD[0], seed=seed)
    opts = dict(PLAIN)
    if net is not None:
        opts.update(denoiser=1, cnn_scale=1)
    out = []
    with Plan(c["n"], c["n_views"], c["n_det"], **opts) as pl:
        if net is not None:
            pl.set_cnn(net)
        y = torch.as_tensor(c["y"]).cuda()
        peak = float(c["mu"].max()) ** 2
        for t in range(1, iters + 1):
            mu = pl.solve(y, c["I0"], t).cpu().numpy().astype(np.float64)
            mse = float(np.mean((mu - c["mu"]) ** 2))
            out.append(round(10 * np.log10(peak / mse), 2) if mse > 0 and np.isfinite(mse) else float("nan"))
        if net is not None:
            pl.set_cnn(None)
    return out


def harvest_clean(n_phantoms: int, patches: int, patch: int, seed0: int = 2000,
                  workload: str = "ellipse512_v64"):
    """x_true = V mu_true patches of training phantoms (GPU), [n_phantoms * patches][patch][patch]."""
    import torch
    import synth
    from .binding import Plan
    rng = np.random.default_rng(11)
    xs = []
    plan = None
    for k in range(n_phantoms):
        c = synth.make_case(workload, seed=seed0 + k)
        if plan is None:
            plan = Plan(c["n"], c["n_views"], c["n_det"], **PLAIN)
        xt = plan.precond_image(torch.as_tensor(c["mu"], dtype=torch.float32).cuda(), inverse=False)
        n = c["n"]
        for _ in range(patches):
            i, j = rng.integers(0, n - patch + 1, size=2)
            xs.append(xt[i:i + patch, j:j + patch])
    plan.close()
    return torch.stack(xs).contiguous()


def train(r, x, sigma, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 100,
          awgn=None, net=None):
    """Adam on the library's kernels.  awgn = (sigma_lo, sigma_hi) draws, every step,
    fresh r = x + sigma n with log-uniform sigma per patch (r and sigma unused).
    net: continue training that network instead of a fresh He-initialised one."""
    import torch
    from .binding import CNN
    if net is None:
        net = CNN(17, seed=seed)
    rng = np.random.default_rng(seed + 1)
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed + 2)
    n = x.shape[0]
    hist = []
    t0 = time.time()
    for s in range(steps):
        idx = rng.choice(n, size=batch, replace=False)
        ti = torch.as_tensor(idx, device=x.device)
        xb = x[ti].contiguous()
        if awgn is not None:
            sg = np.exp(rng.uniform(np.log(awgn[0]), np.log(awgn[1]), size=batch)).astype(np.float32)
            noise = torch.randn(xb.shape, generator=gen, device=x.device)
            rb = (xb + torch.as_tensor(sg, device=x.device)[:, None, None] * noise).contiguous()
        else:
            rb, sg = r[ti].contiguous(), sigma[idx]
        lr_s = lr * (0.5 if s > 0.6 * steps else 1.0) * (0.5 if s > 0.85 * steps else 1.0)
        loss = net.train_step(rb, xb, sg, lr_s)
        if s % log_every == 0 or s == steps - 1:
            hist.append((s, loss))
    return net, hist, time.time() - t0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--phantoms", type=int, default=40)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--patches", type=int, default=17, help="patches per phantom and iteration")
    ap.add_argument("--patch", type=int, default=64)
    ap.add_argument("--steps", type=int, default=4000, help="Adam steps per round")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--mode", choices=("awgn", "iterates"), default="iterates")
    ap.add_argument("--rounds", type=int, default=3,
                    help="iterates: round 1 harvests plain (prox-TV) solves; each later round adds the "
                         "iterates of solves with the network trained so far and trains on")
    ap.add_argument("--blind", action="store_true", help="iterates: sigma = 1 instead of sqrt(tau_r)")
    ap.add_argument("--sigma", type=float, nargs=2, default=(0.003, 1.0), help="awgn sigma range")
    ap.add_argument("--eval-iters", type=int, default=30, help="PSNR curve on the held-out slice (seed 1000)")
    ap.add_argument("--damp", type=float, default=PLAIN["damp_x"],
                    help="damping eta_x (and eta_s unless --damp-s) of the harvesting and evaluation solves")
    ap.add_argument("--damp-s", type=float, default=None)
    ap.add_argument("--tau-x0", type=float, default=1.0, help="initial tau_x of those solves (Algorithm 1)")
    ap.add_argument("--workload", default="ellipse512_v64", help="synth workload of the harvest and evaluation")
    args = ap.parse_args(argv)
    PLAIN.update(damp_x=args.damp, damp_s=args.damp if args.damp_s is None else args.damp_s,
                 tau_x0=args.tau_x0)
    WORKLOAD[0] = args.workload
    import torch
    from . import build
    build.build()
    t0 = time.time()
    rounds = []
    if args.mode == "awgn":
        x = harvest_clean(args.phantoms, args.iters * args.patches, args.patch)
        sg = np.asarray(args.sigma, dtype=np.float32)
        net, hist, t_t = train(None, x, sg, args.steps, args.batch, args.lr, awgn=tuple(args.sigma))
        rounds.append({"pairs": int(x.shape[0]), "loss": hist, "train_s": t_t})
        scaled = True
    else:
        scaled = not args.blind
        net, r, x, sg = None, None, None, None
        for k in range(args.rounds):
            th = time.time()
            rk, xk, sk, diag = harvest(args.phantoms, args.iters, args.patches, args.patch, scaled=scaled,
                                       net=net, rng_seed=7 + k)
            r = rk if r is None else torch.cat([r, rk])
            x = xk if x is None else torch.cat([x, xk])
            sg = sk if sg is None else np.concatenate([sg, sk])
            t_h = time.time() - th
            net, hist, t_t = train(r, x, sg, args.steps, args.batch, args.lr, seed=k, net=net)
            ev = psnr_curve(net, args.eval_iters) if scaled else None
            rounds.append({"round": k + 1, "harvested_from": "prox-TV" if k == 0 else "network",
                           "pairs": int(x.shape[0]), "sigma_range": [float(sg.min()), float(sg.max())],
                           "harvest_s": t_h, "train_s": t_t, "loss_first_last": [hist[0][1], hist[-1][1]],
                           "trajectory": diag, "heldout_psnr_db": ev})
            print(json.dumps(rounds[-1]), flush=True)
    save_weights(args.out, net.get_params(), net.layers, scaled=scaled)
    meta = {"mode": args.mode, "scaled": scaled, "patch": args.patch, "steps_per_round": args.steps,
            "batch": args.batch, "lr": args.lr, "total_s": time.time() - t0,
            "plain_heldout_psnr_db": psnr_curve(None, args.eval_iters), "rounds": len(rounds)}
    print(json.dumps(meta))
    torch.cuda.synchronize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
