"""The D-GAMP-CT loop (Algorithm 1) and the GAMP core it is built on (Section 3).

``gamp`` is Algorithm 1 with its operator, output step and denoiser passed
in, so the same loop runs both the CT problem (:func:`ct_solve`) and the
i.i.d.-Gaussian problem whose state evolution pins it (Section 4.4,
:func:`awgn_gaussian_problem`).  Per iteration t, in the paper's order:

  Step 1  z = Phi~ x;  tau_p = ||Phi~||_F^2 tau_x / M;  p = z - tau_p s_prev
  Step 2  (s, tau_s_i) = g_out(p, y, tau_p);  tau_s = mean(tau_s_i)
  Step 3  tau_r = N / (||Phi~||_F^2 tau_s);  r = x + tau_r Phi~^T s
  Step 4  x+ = D(r);  tau_x = tau_r * D'(r)   (D' by Eq. MC_SURE, K = 1);
          with several denoisers (Selected) each runs on r and the one with
          the lowest SURE estimate of the risk R(x, tau_r) of Section 4.3
          gives x+ and D'

Initialisation x = 0, tau_x = 1 (Algorithm 1, first line); the previous
s is taken as 0 (implied, not stated).  The result is mu = V^-1 x.

Readings (the paper is silent): the MC step is
eps = eps_rel * max(max|r|, 1e-6), the divergence estimate is
D' = b^T (D(r + eps b) - D(r)) / (N eps) -- or, for a denoiser that
provides its directional derivative (the learned network), the eps -> 0
limit b^T J_D(r) b / N that Eq. MC_SURE approaches -- and tau_x is floored at
1e-6 * tau_r (the paper has no guard for D' <= 0).  ``onsager=False`` drops
the tau_p s_prev term (Section 7.1); ``damp_x``/``damp_s`` blend the new x and
s with the previous ones (Section 7.2; 1.0 means no damping).
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np

from .geometry import Geometry
from . import output_step as _out
from . import philox as _philox
from . import precond as _pre
from . import tv as _tv
from . import cnn as _cnn
from . import fanbeam as _fan


@dataclasses.dataclass
class Options:
    c_tv: float = 1.0
    k_tv: int = 30
    eps_rel: float = 1e-3
    seed: int = 12345
    slice_id: int = 0
    onsager: bool = True
    damp_x: float = 1.0
    damp_s: float = 1.0
    tau_x_floor: float = 1e-6
    tau_x0: float = 1.0      # initial tau_x (Algorithm 1 uses 1)
    truncate_z: bool = False  # output step on z >= 0 instead of the whole line
    exact_moments: bool = False  # output step from the exact posterior moments, not Laplace's
    tv_metric: bool = False   # prox-TV in the (V^T V)^{-1} norm (Section 6.3) instead of l2


@dataclasses.dataclass
class IterLog:
    tau_x: float
    tau_p: float
    tau_s: float
    tau_r: float
    div: float
    eps: float
    risks: list | None = None   # SURE of each candidate (Selected), else None
    divs: list | None = None    # the divergence of each candidate (Selected), else None
    kept: int = 0               # index of the kept candidate (Selected)


def mc_divergence(denoise: Callable[[np.ndarray], np.ndarray], r: np.ndarray,
                  x_new: np.ndarray, b: np.ndarray, eps: float) -> float:
    """Eq. MC_SURE with one probe: b^T (D(r + eps b) - D(r)) / (N eps)."""
    d2 = denoise(r + eps * b)
    return float(b.reshape(-1) @ (d2 - x_new).reshape(-1)) / (b.size * eps)


def _divergence(D, r, x_new, b, eps) -> float:
    """D'(r): Eq. MC_SURE, or its eps -> 0 limit b^T J_D(r) b / N for a
    denoiser that provides its directional derivative (the learned network)."""
    jvp = getattr(D, "jvp", None)
    if jvp is not None:
        return float(np.vdot(b, jvp(r, b))) / r.size
    return mc_divergence(D, r, x_new, b, eps)


def sure_risk(r: np.ndarray, x_new: np.ndarray, div: float, tau_r: float) -> float:
    """Stein's unbiased estimate of the denoiser's risk R(x, tau_r) of
    Section 4.3, (1/N) E||D(x + sqrt(tau_r) psi) - x||^2, from its input r and
    output x_new alone: ||x_new - r||^2 / N - tau_r + 2 tau_r D'(r), with D'
    the (Monte-Carlo) divergence of Eq. MC_SURE (the estimate behind that
    equation's reference).  Unbiased when r = x + sqrt(tau_r) psi."""
    d = (np.asarray(x_new, dtype=np.float64) - np.asarray(r, dtype=np.float64)).reshape(-1)
    return float(d @ d) / d.size - tau_r + 2.0 * tau_r * div


class Selected:
    """Step 4 with several denoisers (the plain one first): every iteration
    runs each of them on r, with its own divergence, and keeps the one whose
    SURE risk estimate is lowest; a tie keeps the earlier one.  With the
    learned network second, prox-TV is its fallback and the judge of its
    error.

    ``max_div``: a candidate after the first is kept only if its divergence
    lies in (0, max_div).  tau_x = tau_r D' is a variance, so D' <= 0 (which
    the floor on tau_x would hide) is no estimate of it; and in Algorithm 1
    with a large tau_p the output step gives tau_s near 1/tau_p, so
    tau_r^{t+1} is about tau_r^t D' / delta (delta = M/N): a denoiser with
    D' >= delta makes tau_r grow from one iteration to the next, and the
    SURE estimate, which takes tau_r as the noise level of r, can then not
    be trusted."""

    def __init__(self, candidates, max_div=None):
        self.candidates = list(candidates)
        self.max_div = max_div


def gamp(Phi, PhiT, frob2: float, M: int, N: int, gout, denoise_factory,
         probe, T: int, opts: Options, shape=None, x0=None, log=None,
         on_iter=None):
    """Algorithm 1 with pluggable pieces.

    Phi(x) -> z, PhiT(s) -> image; gout(p, tau_p) -> (s, tau_s_i);
    denoise_factory(tau_r) -> D (a function of one image);
    probe(t, n) -> b (length n); on_iter(t, x) is called with each new x.
    Returns the final x.
    """
    x = np.zeros(shape if shape is not None else N) if x0 is None else np.array(x0, dtype=np.float64)
    tau_x = opts.tau_x0
    s_prev = np.zeros(M)
    for t in range(1, T + 1):
        # Step 1: estimate in the measurement domain
        z = Phi(x).reshape(-1)
        tau_p = frob2 * tau_x / M
        p = z - tau_p * s_prev if opts.onsager else z.copy()
        # Step 2: output step
        s, tau_s_i = gout(p, tau_p)
        if opts.damp_s != 1.0:
            s = opts.damp_s * s + (1.0 - opts.damp_s) * s_prev
        tau_s = float(np.mean(tau_s_i))
        # Step 3: estimate in the signal domain
        tau_r = N / (frob2 * tau_s)
        r = x + tau_r * PhiT(s).reshape(x.shape)
        # Step 4: denoising and divergence
        D = denoise_factory(tau_r)
        b = probe(t, r.size).reshape(r.shape)
        eps = opts.eps_rel * max(float(np.max(np.abs(r))), 1e-6)
        risks = divs = None
        kept = 0
        if isinstance(D, Selected):
            best = None
            risks, divs = [], []
            for k, Dk in enumerate(D.candidates):
                xk = Dk(r)
                dk = _divergence(Dk, r, xk, b, eps)
                rk = sure_risk(r, xk, dk, tau_r)
                risks.append(rk)
                divs.append(dk)
                eligible = k == 0 or D.max_div is None or 0.0 < dk < D.max_div
                if best is None or (eligible and rk < best[2]):
                    best = (xk, dk, rk)
                    kept = k
            x_new, div = best[0], best[1]
        else:
            x_new = D(r)
            div = _divergence(D, r, x_new, b, eps)
        tau_x = max(tau_r * div, opts.tau_x_floor * tau_r)
        if opts.damp_x != 1.0:
            x_new = opts.damp_x * x_new + (1.0 - opts.damp_x) * x
        if log is not None:
            log.append(IterLog(tau_x, tau_p, tau_s, tau_r, div, eps, risks, divs, kept))
        x = x_new
        s_prev = s
        if on_iter is not None:
            on_iter(t, x)
    return x


def ct_solve(y: np.ndarray, I0: float, geom: Geometry, T: int,
             opts: Options | None = None, return_x: bool = False, log=None,
             frob2: float | None = None, on_iter=None, cnn=None, cnn_bf16: bool = True,
             select: bool = False):
    """D-GAMP-CT on one slice (parity unpinned).

    The denoiser is prox-TV, or with ``cnn = (ws, bs, scaled)`` the learned
    residual network of ``oracle.cnn`` in its BF16-activation form
    (``cnn_bf16=False``: unrounded FP64 activations), run at
    sigma = sqrt(tau_r) (scaled) or sigma = 1 (blind).  With ``select`` both
    run every iteration and the lower SURE risk estimate decides
    (:class:`Selected`, prox-TV first; the network only with 0 < D' < M/N).  The full
    reconstruction has no closed form and the paper prints no synthetic
    result; it is checked only through its pinned parts and the tests'
    qualitative checks (error falls over the iterations, the Onsager term
    helps).  ``frob2`` may pass a precomputed ||Phi~||_F^2.
    """
    opts = opts or Options()
    yv = np.asarray(y, dtype=np.float64).reshape(-1)
    # parallel beam (Geometry) or flat-detector fan beam (FanGeometry): the
    # preconditioned operator Phi~ = A V^-1 of Eq. precondAMP_op either way
    ops = _fan if isinstance(geom, _fan.FanGeometry) else _pre
    if frob2 is None:
        frob2 = ops.frobenius_sq(geom)

    def Phi(x):
        return ops.project(x, geom)

    def PhiT(s):
        return ops.backproject(s.reshape(geom.n_views, geom.n_det), geom)

    if opts.exact_moments and opts.truncate_z:
        raise ValueError("exact posterior moments are computed on the whole line only")

    def gout(p, tau_p):
        if opts.exact_moments:
            s, tsi, _m, _v = _out.output_step_exact(p, yv, tau_p, I0)
        else:
            s, tsi, _z0, _v = _out.output_step(p, yv, tau_p, I0, truncate=opts.truncate_z)
        return s, tsi

    if select and cnn is None:
        raise ValueError("select needs the learned network (cnn)")

    def plain(tau_r):
        lam = opts.c_tv * np.sqrt(tau_r)
        if opts.tv_metric:
            q_max = _pre.vtv_inverse_norm_bound(geom)
            return lambda r: _tv.tv_prox_metric(r, lam, opts.k_tv,
                                                lambda u: _pre.vtv_inverse(u, geom), q_max)
        return lambda r: _tv.tv_prox(r, lam, opts.k_tv)

    def denoise_factory(tau_r):
        if cnn is None:
            return plain(tau_r)
        ws, bs, scaled = cnn
        sigma = float(np.sqrt(tau_r)) if scaled else 1.0
        learned = _cnn.Denoiser(sigma, ws, bs, bf16=cnn_bf16)
        return Selected([plain(tau_r), learned], max_div=geom.M / geom.N) if select else learned

    def probe(t, n):
        return _philox.probe_normals(n, opts.seed, t, opts.slice_id)

    x = gamp(Phi, PhiT, frob2, geom.M, geom.N, gout, denoise_factory, probe, T,
             opts, shape=(geom.n, geom.n), log=log, on_iter=on_iter)
    mu = _pre.v_inverse(x, geom)
    return (mu, x) if return_x else mu


# ----------------------------------------------------------- SE pin ----
def awgn_gaussian_problem(N: int, M: int, sigma2: float, seed: int):
    """i.i.d. Gaussian A (entries N(0, 1/M), Section 3), x ~ N(0, I), y = Ax + w."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, N)) / np.sqrt(M)
    x = rng.standard_normal(N)
    y = A @ x + np.sqrt(sigma2) * rng.standard_normal(M)
    return A, x, y


def awgn_gout(y, sigma2):
    """Gaussian channel output step: posterior of z given N(p, tau_p) and y = z + w."""
    def g(p, tau_p):
        s = (y - p) / (sigma2 + tau_p)
        return s, np.full_like(p, 1.0 / (sigma2 + tau_p))
    return g


def gaussian_prior_denoiser(tau_r):
    """MMSE denoiser for x ~ N(0, 1) seen through N(x, tau_r): r / (1 + tau_r)."""
    return lambda r: r / (1.0 + tau_r)


def state_evolution_gaussian(delta: float, sigma2: float, T: int):
    """Scalar SE (Section 4.4, Eq. SE_matches, beta = M/N = delta) for this problem.

    tau_r^t = sigma^2 + tau_x^t / delta, tau_x^{t+1} = tau_r^t / (1 + tau_r^t),
    tau_x^0 = 1 (Algorithm 1 initialisation).  Returns [tau_x^1, ..., tau_x^T].
    """
    tx = 1.0
    out = []
    for _ in range(T):
        tr = sigma2 + tx / delta
        tx = tr / (1.0 + tr)
        out.append(tx)
    return out
