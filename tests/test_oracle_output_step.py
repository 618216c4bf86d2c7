"""Pins for the oracle's Poisson output step (Section 4.2, Appendix A)."""
import math

import numpy as np
import pytest

from oracle import output_step as out


def _batch(seed=7, n=4000):
    rng = np.random.default_rng(seed)
    I0 = 1e5
    z_true = rng.uniform(0.0, 14.0, n)
    y = rng.poisson(I0 * np.exp(-z_true)).astype(float)      # includes y = 0 rays
    p = z_true + rng.normal(0, 2.0, n)
    p[:20] = rng.uniform(-60, -20, 20)                        # far-off messages
    p[20:40] = rng.uniform(30, 60, 20)
    return p, y, I0


@pytest.mark.parametrize("tau_p", [1e-6, 1e-2, 1.0, 1e3])
def test_mode_solves_stationarity(tau_p):
    p, y, I0 = _batch()
    d = out.laplace_mode_delta(p, y, tau_p, math.log(I0))
    z0 = p + d
    w = np.exp(math.log(I0) - z0)
    resid = d / tau_p + y - w
    scale = np.abs(d / tau_p) + y + w
    assert np.all(np.isfinite(d))
    assert np.max(np.abs(resid) / scale) < 1e-10
    assert (y == 0).sum() > 10


def test_limits():
    p, y, I0 = _batch()
    keep = (y > 0) & (np.arange(p.size) >= 40)      # finite limits need ordinary messages
    p, y = p[keep], y[keep]
    # tau_p -> 0: the prior message dominates, z0 -> p and s tends to the
    # likelihood score d/dz log p(y|z) at z = p, i.e. I0 e^{-p} - y
    s, tsi, z0, var = out.output_step(p, y, 1e-12, I0)
    score = I0 * np.exp(-p) - y
    assert np.allclose(s, score, rtol=1e-3, atol=1e-6 * np.abs(score).max())
    assert np.max(np.abs(z0 - p)) < 1e-3
    # tau_p -> inf: the likelihood dominates, z0 -> log(I0 / y)
    s, tsi, z0, var = out.output_step(p, y, 1e10, I0)
    assert np.max(np.abs(z0 - np.log(I0 / y))) < 1e-5


def test_tau_s_is_minus_derivative_of_s():
    # Section 3: tau_s_i = -d g_out / d p_i; exact for the Laplace reading since dz0/dp = Var/tau_p.
    p, y, I0 = _batch(n=500)
    tau_p = 0.3
    h = 1e-6
    s1 = out.output_step(p + h, y, tau_p, I0)[0]
    s0 = out.output_step(p - h, y, tau_p, I0)[0]
    _, tsi, _, var = out.output_step(p, y, tau_p, I0)
    fd = -(s1 - s0) / (2 * h)
    assert np.allclose(fd, tsi, rtol=1e-5, atol=1e-7)     # FD rounding ~1e-9 / h
    assert np.allclose(tsi, (1 / tau_p) * (1 - var / tau_p), rtol=1e-10)


def test_laplace_matches_quadrature_as_counts_grow():
    # The posterior tends to a Gaussian as y grows, so the Laplace mode/variance
    # tend to the exact posterior mean/variance.
    errs = []
    for I0, z in [(1e2, 2.0), (1e4, 2.0), (1e6, 2.0), (1e8, 2.0)]:
        y = float(round(I0 * math.exp(-z)))
        p, tau_p = z + 0.3, 0.05
        mean_q, var_q = out.posterior_moments_quadrature(p, y, tau_p, I0)
        s, tsi, z0, var = out.output_step(np.array([p]), np.array([y]), tau_p, I0)
        errs.append((abs(z0[0] - mean_q) / math.sqrt(var_q), abs(var[0] / var_q - 1)))
    assert errs[-1][0] < 1e-3 and errs[-1][1] < 1e-2
    assert errs[0][0] > errs[1][0] > errs[2][0] > errs[3][0]


def test_gaussian_channel_limit_closed_form():
    # For large y the log-likelihood is ~ -(y/2)(z - L)^2 with L = log(I0/y), so
    # z0 -> (p/tau_p + y L)/(1/tau_p + y), the Gaussian-product mean.
    I0, y = 1e9, 1e7
    L = math.log(I0 / y)
    p, tau_p = L + 0.002, 1e-7
    _, _, z0, _ = out.output_step(np.array([p]), np.array([y]), tau_p, I0)
    ref = (p / tau_p + y * L) / (1 / tau_p + y)
    assert abs(z0[0] - ref) < 1e-6
