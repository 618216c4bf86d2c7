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


def test_truncated_mode_is_the_argmax_over_nonnegative_z():
    """The truncated reading: the mode of the posterior restricted to z >= 0 is
    found by brute force on a fine grid of [0, 20]; where the unconstrained
    mode is already >= 0 nothing changes."""
    I0, tau_p = 1e4, 0.5
    rng = np.random.default_rng(3)
    # rays through (almost) nothing: counts can exceed I0, pulling the mode below 0
    p = np.concatenate([rng.uniform(-3.0, 0.5, 40), rng.uniform(1.0, 8.0, 40)])
    u = np.concatenate([rng.uniform(-0.05, 0.02, 40), p[40:]])
    y = rng.poisson(I0 * np.exp(-u)).astype(float)
    s_f, tsi_f, z_f, _ = out.output_step(p, y, tau_p, I0)
    s_t, tsi_t, z_t, var_t = out.output_step(p, y, tau_p, I0, truncate=True)
    grid = np.linspace(0.0, 20.0, 400001)
    for k in range(p.size):
        logpost = -(grid - p[k]) ** 2 / (2 * tau_p) + y[k] * (np.log(I0) - grid) - I0 * np.exp(-grid)
        assert abs(z_t[k] - grid[np.argmax(logpost)]) <= 1e-4
    keep = z_f >= 0
    assert np.array_equal(z_t[keep], z_f[keep]) and np.array_equal(s_t[keep], s_f[keep])
    assert np.array_equal(tsi_t[keep], tsi_f[keep])
    act = ~keep
    assert act.sum() > 5
    assert np.all(var_t[act] == 0.0) and np.allclose(tsi_t[act], 1.0 / tau_p)


def test_truncated_tau_s_is_minus_derivative_of_s():
    """-ds/dp = tau_s_i holds on both branches of the truncated reading."""
    I0, tau_p = 1e4, 0.3
    rng = np.random.default_rng(5)
    p = rng.uniform(-2.0, 6.0, 200)
    y = rng.poisson(I0 * np.exp(-np.clip(p, 0.05, None))).astype(float)
    h = 1e-6
    s_p, *_ = out.output_step(p + h, y, tau_p, I0, truncate=True)
    s_m, *_ = out.output_step(p - h, y, tau_p, I0, truncate=True)
    _, tsi, z0, _ = out.output_step(p, y, tau_p, I0, truncate=True)
    away = np.abs(z0) > 1e-3             # not at the kink itself
    assert np.allclose(-(s_p - s_m)[away] / (2 * h), tsi[away], rtol=1e-5, atol=1e-6)
