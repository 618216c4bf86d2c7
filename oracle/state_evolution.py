"""State evolution of D-GAMP-CT (Section 4.4, Eqs. SEasym and SE_matches).

GAMP's state evolution tracks Algorithm 1 by a scalar recursion in which
the denoiser's input is the truth plus white Gaussian noise of variance
tau_r, and the output step sees messages P whose error against the true
Z has variance tau_p.  Per iteration, in the normalisation of Algorithm 1:

    tau_p = ||Phi~||_F^2 tau_x / M,
    P = Z + sqrt(tau_p) W, W ~ N(0, I)          (see the reading below),
    tau_s = mean_i tau_s,i(P_i, Y_i; tau_p)      (the output step's own -ds/dp),
    tau_r = N / (||Phi~||_F^2 tau_s),
    R = X + sqrt(tau_r) E, E ~ N(0, I),
    mse = ||D(R) - X||^2 / N                     (the error function E_in),
    D' = the MC divergence of D at R              (the sensitivity A_in, Eq. MC_SURE),
    tau_x = max(tau_r D', floor tau_r).

Reading: the paper's covariance K_p of (Z, P) makes Z - P independent of P
with variance tau_p; for line integrals with a spread far larger than tau_p
that is, to first order, P = Z + sqrt(tau_p) W with W independent of Z,
which is what this module draws.  Z and X are the true preconditioned
sinogram Phi~ x and image x = V mu; Y are the measured counts.  The
expectations over W and E are single draws (N and M are large), from a
seeded numpy generator.

The recursion is pinned by its reduction to the closed-form SE of the
i.i.d. Gaussian problem (oracle.gamp.state_evolution_gaussian); on CT data
it has no closed form (parity unpinned: there it is compared with the
algorithm, not with a known result).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SERecord:
    tau_p: float
    tau_s: float
    tau_r: float
    mse: float
    div: float
    tau_x: float


def state_evolution(z_true, x_true, frob2: float, gout, denoise_factory, T: int, tau_x0: float = 1.0,
                    tau_x_floor: float = 1e-6, eps_rel: float = 1e-3, seed: int = 0):
    """The recursion above for T iterations; gout(p, tau_p) -> (s, tau_s_i),
    denoise_factory(tau_r) -> D.  Returns one SERecord per iteration."""
    rng = np.random.default_rng(seed)
    z = np.asarray(z_true, dtype=np.float64).reshape(-1)
    x = np.asarray(x_true, dtype=np.float64)
    M, N = z.size, x.size
    tau_x = float(tau_x0)
    out = []
    for _ in range(T):
        tau_p = frob2 * tau_x / M
        p = z + np.sqrt(tau_p) * rng.standard_normal(M)
        _s, tsi = gout(p, tau_p)
        tau_s = float(np.mean(tsi))
        tau_r = N / (frob2 * tau_s)
        r = x + np.sqrt(tau_r) * rng.standard_normal(x.shape)
        D = denoise_factory(tau_r)
        xh = D(r)
        mse = float(np.mean((xh - x) ** 2))
        b = rng.standard_normal(x.shape)
        eps = eps_rel * max(float(np.max(np.abs(r))), 1e-6)
        div = float(np.sum(b * (D(r + eps * b) - xh))) / (N * eps)
        tau_x = max(tau_r * div, tau_x_floor * tau_r)
        out.append(SERecord(tau_p, tau_s, tau_r, mse, div, tau_x))
    return out


def ct_state_evolution(y, I0: float, geom, T: int, opts, mu_true, frob2: float | None = None, seed: int = 0):
    """The recursion for one CT slice with the operators, output step and
    prox-TV of oracle.gamp.ct_solve (parallel or fan beam)."""
    from . import fanbeam as _fan
    from . import gamp as _gamp
    from . import output_step as _out
    from . import precond as _pre
    from . import tv as _tv
    ops = _fan if isinstance(geom, _fan.FanGeometry) else _pre
    if frob2 is None:
        frob2 = ops.frobenius_sq(geom)
    x_true = _pre.v_forward(mu_true, geom)
    z_true = ops.project(x_true, geom).reshape(-1)
    yv = np.asarray(y, dtype=np.float64).reshape(-1)
    if not isinstance(opts, _gamp.Options):
        raise TypeError("opts must be oracle.gamp.Options")

    def gout(p, tau_p):
        if opts.exact_moments:
            s, tsi, _m, _v = _out.output_step_exact(p, yv, tau_p, I0)
        else:
            s, tsi, _z0, _v = _out.output_step(p, yv, tau_p, I0, truncate=opts.truncate_z)
        return s, tsi

    def denoise_factory(tau_r):
        lam = opts.c_tv * np.sqrt(tau_r)
        if opts.tv_metric:
            q_max = _pre.vtv_inverse_norm_bound(geom)
            return lambda r: _tv.tv_prox_metric(r, lam, opts.k_tv, lambda u: _pre.vtv_inverse(u, geom), q_max)
        return lambda r: _tv.tv_prox(r, lam, opts.k_tv)

    return state_evolution(z_true, x_true, frob2, gout, denoise_factory, T, tau_x0=opts.tau_x0,
                           tau_x_floor=opts.tau_x_floor, eps_rel=opts.eps_rel, seed=seed)
