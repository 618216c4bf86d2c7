"""Pins for the SURE risk estimate and the risk-judged choice of denoiser
(Section 4.3's risk R(x, tau_r) = (1/N) E||D(x + sqrt(tau_r) psi) - x||^2,
estimated from r alone with the divergence of Eq. MC_SURE).

Closed forms: for a linear denoiser D(r) = a r the risk is
(a - 1)^2 ||x||^2 / N + a^2 tau, and the mean of the estimate over the noise
must equal it; for soft thresholding the true risk is measured directly
with the clean signal known.  The choice is checked on the i.i.d. Gaussian
problem, where the MMSE denoiser must win against a poor one in either
order and the run must equal the MMSE-only run exactly.
"""
import numpy as np
import pytest

from oracle import gamp, philox


def _mc_mean(vals):
    vals = np.asarray(vals)
    return float(vals.mean()), float(vals.std(ddof=1) / np.sqrt(vals.size))


@pytest.mark.parametrize("a", [0.3, 0.8, 1.0, 1.4])
def test_sure_is_unbiased_for_a_linear_denoiser(a):
    rng = np.random.default_rng(5)
    n, tau, draws = 256, 0.7, 4000
    x = rng.standard_normal(n) * 1.5
    est = []
    for _ in range(draws):
        r = x + np.sqrt(tau) * rng.standard_normal(n)
        est.append(gamp.sure_risk(r, a * r, a, tau))     # D' = a exactly
    mean, se = _mc_mean(est)
    true = (a - 1.0) ** 2 * float(x @ x) / n + a * a * tau
    assert abs(mean - true) < 4 * se + 1e-12


def test_sure_with_mc_divergence_tracks_soft_threshold_risk():
    rng = np.random.default_rng(6)
    n, tau, thr, draws = 4096, 0.25, 0.6, 200
    x = np.where(rng.random(n) < 0.2, rng.standard_normal(n) * 3.0, 0.0)    # sparse signal
    D = lambda v: np.sign(v) * np.maximum(np.abs(v) - thr, 0.0)
    est, true = [], []
    for k in range(draws):
        r = x + np.sqrt(tau) * rng.standard_normal(n)
        xr = D(r)
        b = philox.probe_normals(n, 21, k + 1, 0)
        div = gamp.mc_divergence(D, r, xr, b, 1e-6)
        est.append(gamp.sure_risk(r, xr, div, tau))
        true.append(float(np.mean((xr - x) ** 2)))
    m_est, se_est = _mc_mean(est)
    m_true, se_true = _mc_mean(true)
    assert abs(m_est - m_true) < 4 * np.hypot(se_est, se_true)
    # and the estimate is not trivially the noise level
    assert abs(m_true - tau) > 10 * se_true


def _awgn_run(denoise_factory, seed=3, T=8):
    N, M, sigma2 = 2000, 1000, 0.01
    A, x, y = gamp.awgn_gaussian_problem(N, M, sigma2, seed)
    frob2 = float(np.sum(A * A))
    log = []
    xt = gamp.gamp(lambda v: A @ v, lambda s: A.T @ s, frob2, M, N, gamp.awgn_gout(y, sigma2), denoise_factory,
                   lambda t, n: philox.probe_normals(n, 40 + seed, t, 0), T, gamp.Options(eps_rel=1e-3), log=log)
    return xt, log


@pytest.mark.parametrize("order", ["mmse_first", "poor_first"])
def test_selection_keeps_the_lower_risk_denoiser(order):
    mmse = gamp.gaussian_prior_denoiser
    poor = lambda tau_r: (lambda r: 2.0 * r)      # D' = 2: its risk is ||r||^2/N + 3 tau_r

    def selected(tau_r):
        c = [mmse(tau_r), poor(tau_r)]
        return gamp.Selected(c if order == "mmse_first" else c[::-1])

    x_ref, log_ref = _awgn_run(mmse)
    x_sel, log_sel = _awgn_run(selected)
    assert np.array_equal(x_sel, x_ref)
    k = 0 if order == "mmse_first" else 1
    for a, b in zip(log_sel, log_ref):
        assert a.risks is not None and len(a.risks) == 2
        assert a.risks[k] < a.risks[1 - k]
        assert a.tau_x == b.tau_x and a.div == b.div


def test_selection_tie_keeps_the_first_denoiser():
    rng = np.random.default_rng(8)
    r = rng.standard_normal(64)
    # two candidates with identical outputs and divergences: the first is kept
    first = lambda v: 0.5 * v
    second = lambda v: 0.5 * v
    sel = gamp.Selected([first, second])
    assert sel.candidates[0] is first
    x_ref, _ = _awgn_run(lambda tau_r: first)
    x_sel, log = _awgn_run(lambda tau_r: gamp.Selected([first, second]))
    assert np.array_equal(x_sel, x_ref)
    assert all(lg.risks[0] == lg.risks[1] for lg in log)


def test_selection_skips_a_candidate_whose_divergence_is_too_large():
    # the MMSE denoiser has the lower risk, but its divergence 1/(1 + tau_r)
    # is not below max_div = 1e-12: the first candidate (a poor one) is kept
    mmse = gamp.gaussian_prior_denoiser
    poor = lambda tau_r: (lambda r: 2.0 * r)
    x_poor, _ = _awgn_run(poor, T=3)
    x_free, log_free = _awgn_run(lambda tau_r: gamp.Selected([poor(tau_r), mmse(tau_r)]), T=3)
    x_cap, log_cap = _awgn_run(lambda tau_r: gamp.Selected([poor(tau_r), mmse(tau_r)], max_div=1e-12), T=3)
    assert np.array_equal(x_cap, x_poor)
    # without the bound the MMSE candidate wins, so the bound is what decides
    assert all(lg.risks[1] < lg.risks[0] for lg in log_free)
    assert all(lg.div > 1e-12 for lg in log_free)
    assert not np.array_equal(x_free, x_poor)
