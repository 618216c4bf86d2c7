"""Poisson output step of Algorithm 1, Step 2 (Section 4.2, Appendix A).

For each measurement the posterior of z given the Gaussian message
N(p, tau_p) and the count y ~ Poisson(I0 e^{-z}) (Eq. Poisson_CT with no
background term) is proportional to

    exp( -(z - p)^2 / (2 tau_p) + y log(I0 e^{-z}) - I0 e^{-z} ).

Laplace's method (Section 4.2 and Appendix A, after Tierney-Kadane) replaces
it by a Gaussian at its mode z0 with variance the inverse curvature there.
The appendix's algebra is garbled (the likelihood drops I0, a stray 1/M
appears, the stationarity and curvature equations have sign errors); this
oracle uses the corrected first-order reading:

* the mode solves psi(z) = (z - p)/tau_p + y - I0 e^{-z} = 0; psi is strictly
  increasing, so the root is unique;
* Var = 1 / (1/tau_p + I0 e^{-z0});
* s = (z0 - p)/tau_p (Eq. MMSEmm), tau_s_i = (1/tau_p)(1 - Var/tau_p)
  (Section 3, Eq. for tau_s), i.e. w/(1 + tau_p w) with w = I0 e^{-z0};
* tau_s = mean_i tau_s_i (Algorithm 1, Step 2).

The root is found for delta = z0 - p (a change of variable that keeps s free
of cancellation): psi(delta) = delta/tau_p + y - a e^{-delta},
a = exp(log I0 - p).  The bracket is [min(0, L - p), max(0, L - p)] with
L = log(I0/y) when y > 0, and [0, m - p + tau_p exp(log I0 - m)] with
m = max(p, log I0) when y = 0 (psi is negative at the left end and positive
at the right end in every case).  The search is Newton's method guarded by
bisection (a step that leaves the bracket, or that shrinks |psi| too slowly,
is replaced by the bracket midpoint), the classical safeguarded scheme.
The integrals run over the whole real line (the paper's restriction to
z >= 0 is not applied).
"""
from __future__ import annotations

import numpy as np


def _psi(delta, y, a, tau_p):
    with np.errstate(over="ignore", invalid="ignore"):
        w = a * np.exp(-delta)
        return delta / tau_p + y - w, 1.0 / tau_p + w, w


def laplace_mode_delta(p, y, tau_p, log_I0, max_iter: int = 100, tol: float = 1e-13):
    """delta = z0 - p for every measurement (vectorised safeguarded Newton)."""
    p = np.asarray(p, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    with np.errstate(over="ignore", divide="ignore"):
        a = np.exp(log_I0 - p)
        L = np.where(y > 0, log_I0 - np.log(np.where(y > 0, y, 1.0)), 0.0)
    m = np.maximum(p, log_I0)
    hi0 = m - p + tau_p * np.exp(log_I0 - m)
    lo = np.where(y > 0, np.minimum(0.0, L - p), 0.0)
    hi = np.where(y > 0, np.maximum(0.0, L - p), hi0)
    d = lo.copy()
    dx_old = hi - lo
    for _ in range(max_iter):
        f, df, _w = _psi(d, y, a, tau_p)
        lo = np.where(f < 0, d, lo)
        hi = np.where(f > 0, d, hi)
        with np.errstate(invalid="ignore", divide="ignore"):
            step = f / df
        newton = d - step
        bad = (~np.isfinite(newton)) | (newton <= lo) | (newton >= hi) \
            | (np.abs(2.0 * f) > np.abs(dx_old * df))
        nxt = np.where(bad, 0.5 * (lo + hi), newton)
        nxt = np.where(f == 0, d, nxt)
        dx_old = np.abs(nxt - d)
        done = dx_old <= tol * np.abs(nxt)
        d = nxt
        if np.all(done):
            break
    return d


def output_step(p, y, tau_p, I0, truncate: bool = False):
    """Algorithm 1, Step 2.  Returns (s, tau_s_i, z0, var) as fp64 arrays.

    ``truncate``: the posterior of z restricted to z >= 0 (a line integral of
    a non-negative attenuation map; the paper's integrals run over the whole
    line by default).  Its mode is max(z0, 0); where the bound is active the
    mode does not move with p, so s = -p / tau_p, var = 0 and
    tau_s_i = -ds/dp = 1 / tau_p."""
    log_I0 = float(np.log(I0))
    p = np.asarray(p, dtype=np.float64)
    d = laplace_mode_delta(p, y, tau_p, log_I0)
    z0 = p + d
    w = np.exp(log_I0 - z0)
    var = 1.0 / (1.0 / tau_p + w)
    s = d / tau_p
    tau_s_i = w / (1.0 + tau_p * w)
    if truncate:
        act = z0 < 0.0
        z0 = np.where(act, 0.0, z0)
        s = np.where(act, -p / tau_p, s)
        var = np.where(act, 0.0, var)
        tau_s_i = np.where(act, 1.0 / tau_p, tau_s_i)
    return s, tau_s_i, z0, var


def posterior_moments_quadrature(p, y, tau_p, I0, half_width: float = 12.0, n: int = 20001):
    """Exact posterior mean and variance of z by quadrature (test reference).

    Integrates the unnormalised posterior on a uniform grid of ``n`` points
    spanning +-half_width posterior standard deviations around the Laplace
    mode (the density is log-concave, so the mass outside is negligible).
    Scalar inputs only.
    """
    d = float(laplace_mode_delta(np.array([p]), np.array([y]), tau_p, np.log(I0))[0])
    z0 = p + d
    sd = np.sqrt(1.0 / (1.0 / tau_p + I0 * np.exp(-z0)))
    z = np.linspace(z0 - half_width * sd, z0 + half_width * sd, n)
    logpost = -(z - p) ** 2 / (2 * tau_p) + y * (np.log(I0) - z) - I0 * np.exp(-z)
    wgt = np.exp(logpost - logpost.max())
    mass = np.trapezoid(wgt, z)
    mean = np.trapezoid(wgt * z, z) / mass
    var = np.trapezoid(wgt * (z - mean) ** 2, z) / mass
    return mean, var


# ------------------------------------------------ exact posterior moments ---
# The output step without Laplace's approximation: s and tau_s_i from the
# exact posterior mean and variance of z (Appendix A, before its Laplace
# step; Section 3's s = (E[z] - p)/tau_p, tau_s_i = (1/tau_p)(1 - Var/tau_p)).
# Relative to the mode z0 = p + delta the log posterior is
#     l(t) = -t^2 / (2 tau_p) - w0 (e^{-t} - 1 + t),   w0 = I0 e^{-z0},
# (the mode condition cancels the linear terms): concave, l(0) = 0 and
# l(t) <= -t^2 / (2 tau_p).  The integrals run over [t_lo, t_hi] where
# l = -EXACT_LOGCUT on each side (found by bisection inside
# [0, +-sqrt(2 EXACT_LOGCUT tau_p)]), which holds all but e^-50 of the mass
# whatever the skew, by the trapezoid rule on a uniform grid.
EXACT_LOGCUT = 50.0


def _exact_l(t, tau_p, lw0):
    """l(t) with lw0 = log w0.  Near the mode (|t| < 1) w0 (expm1(-t) + t)
    keeps the t^2/2 behaviour exact; away from it the same term is
    exp(lw0 - t) + w0 (t - 1), which stays finite where w0 underflows."""
    with np.errstate(over="ignore", invalid="ignore"):
        w0 = np.exp(lw0)
        near = w0 * (np.expm1(-t) + t)
        far = np.exp(lw0 - t) + w0 * (t - 1.0)
    return -t * t / (2.0 * tau_p) - np.where(np.abs(t) < 1.0, near, far)


def _exact_edge(sign, tau_p, lw0, steps: int = 80):
    """t on side `sign` (+1 / -1) where l(t) = -EXACT_LOGCUT, by bisection."""
    lo = np.zeros_like(lw0)
    hi = sign * np.sqrt(2.0 * EXACT_LOGCUT * tau_p) * np.ones_like(lw0)
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        above = _exact_l(mid, tau_p, lw0) > -EXACT_LOGCUT
        lo = np.where(above, mid, lo)
        hi = np.where(above, hi, mid)
    return hi


def output_step_exact(p, y, tau_p, I0, n: int = 4001):
    """Algorithm 1, Step 2 with the exact posterior moments.  Returns
    (s, tau_s_i, mean, var) as fp64 arrays (mean and var of z)."""
    log_I0 = float(np.log(I0))
    p = np.asarray(p, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = laplace_mode_delta(p, y, tau_p, log_I0)
    lw0 = log_I0 - (p + d)                   # log of w0 = I0 e^{-z0}
    t_lo = _exact_edge(-1.0, tau_p, lw0)
    t_hi = _exact_edge(+1.0, tau_p, lw0)
    u = np.linspace(0.0, 1.0, n)
    mean = np.empty_like(p)
    var = np.empty_like(p)
    for i0 in range(0, p.size, 256):        # chunks: n grid points per measurement
        sl = slice(i0, min(p.size, i0 + 256))
        t = t_lo[sl, None] + (t_hi[sl] - t_lo[sl])[:, None] * u[None, :]
        wgt = np.exp(_exact_l(t, tau_p, lw0[sl, None]))
        mass = np.trapezoid(wgt, t, axis=1)
        m1 = np.trapezoid(wgt * t, t, axis=1) / mass
        var[sl] = np.trapezoid(wgt * (t - m1[:, None]) ** 2, t, axis=1) / mass
        mean[sl] = p[sl] + d[sl] + m1
    s = (mean - p) / tau_p
    tau_s_i = (1.0 - var / tau_p) / tau_p
    return s, tau_s_i, mean, var
