"""Pins of the oracle's exact-moment output step (the Poisson output step of
Algorithm 1, Step 2, with the posterior mean and variance of z computed
exactly instead of by Laplace's approximation; Appendix A).

* Against adaptive quadrature over the whole real line (scipy.integrate.quad,
  an independent integrator) in every regime: high counts, no counts, wide and
  narrow messages -- the skewed cases are where a window sized by the Laplace
  variance alone would miss the tail.
* The identity -ds/dp = tau_s_i: for a Gaussian message N(z; p, tau_p) and
  any likelihood, dE[z|p]/dp = Var[z|p]/tau_p, so with s = (E[z] - p)/tau_p
  the derivative of s is -(1/tau_p)(1 - Var/tau_p).  Checked by central
  differences, it ties the variance to the mean independently of how either
  is computed.
* The Gaussian limit: with many counts the posterior is nearly Gaussian and
  the exact moments approach Laplace's.
"""
import numpy as np
import pytest

from oracle import output_step as out

I0 = 1e5


def _quad_moments(p, y, tau_p):
    integrate = pytest.importorskip("scipy.integrate")
    d = float(out.laplace_mode_delta(np.array([p]), np.array([float(y)]), tau_p, np.log(I0))[0])
    z0 = p + d

    def lp(z):
        return -(z - p) ** 2 / (2 * tau_p) + y * (np.log(I0) - z) - I0 * np.exp(min(-z, 700.0))

    l0 = lp(z0)

    def f(z, m):
        e = lp(z) - l0
        return 0.0 if not e > -745.0 else np.exp(e) * (z - z0) ** m    # density underflowed: no mass

    mom = [integrate.quad(f, -np.inf, z0, args=(m,), epsabs=0, epsrel=1e-12, limit=1000)[0]
           + integrate.quad(f, z0, np.inf, args=(m,), epsabs=0, epsrel=1e-12, limit=1000)[0] for m in range(3)]
    mean = z0 + mom[1] / mom[0]
    return mean, mom[2] / mom[0] - (mom[1] / mom[0]) ** 2


@pytest.mark.parametrize("y", [0, 1, 30, 3000, 80000])
@pytest.mark.parametrize("tau_p", [1e-3, 1.0, 1e2, 1e4])
def test_exact_moments_match_adaptive_quadrature(y, tau_p):
    p = np.array([-4.0, 0.0, 4.0, 9.0])
    _s, _t, mean, var = out.output_step_exact(p, np.full(p.size, float(y)), tau_p, I0)
    for k in range(p.size):
        m_ref, v_ref = _quad_moments(float(p[k]), y, tau_p)
        assert abs(mean[k] - m_ref) <= 1e-8 * np.sqrt(v_ref)
        assert abs(var[k] - v_ref) <= 1e-8 * v_ref


@pytest.mark.parametrize("tau_p", [1e-2, 1.0, 1e2])
def test_exact_step_derivative_identity(tau_p):
    rng = np.random.default_rng(11)
    z = rng.uniform(0.0, 10.0, 40)
    y = rng.poisson(I0 * np.exp(-z)).astype(float)
    p = z + rng.normal(0.0, np.sqrt(tau_p), z.size)
    h = 1e-4 * np.sqrt(tau_p)
    s_plus = out.output_step_exact(p + h, y, tau_p, I0)[0]
    s_minus = out.output_step_exact(p - h, y, tau_p, I0)[0]
    tau_s_i = out.output_step_exact(p, y, tau_p, I0)[1]
    deriv = -(s_plus - s_minus) / (2 * h)
    assert np.allclose(deriv, tau_s_i, rtol=1e-5, atol=1e-9 / tau_p)


def test_exact_moments_reach_laplace_with_many_counts():
    """With y counts the likelihood's skew, and so the posterior mean's
    distance from the mode in units of its width, is at most of order
    1 / sqrt(y) (less where the Gaussian message dominates); the variance and
    tau_s_i agree to higher order."""
    z = np.array([0.5, 1.0, 2.0, 3.0, 6.0])
    y = np.round(I0 * np.exp(-z))
    tau_p = 1e-3
    p = z + 0.01
    _s, t_e, mean, var = out.output_step_exact(p, y, tau_p, I0)
    _s, t_l, z0, var_l = out.output_step(p, y, tau_p, I0)
    shift = np.abs(mean - z0) / np.sqrt(var_l)
    assert np.all(shift < 1.0 / np.sqrt(y))
    assert np.allclose(var, var_l, rtol=3.0 / y.min())
    assert np.allclose(t_e, t_l, rtol=3e-4)


@pytest.mark.parametrize("tau_p", [1e-2, 1.0, 1e4])
def test_exact_moments_with_no_information_are_the_message(tau_p):
    """y = 0 and a message far beyond the data (I0 e^{-z} underflows even in
    FP64): the likelihood is flat, so the posterior is the message itself,
    mean p and variance tau_p, and s = 0, tau_s_i = 0."""
    p = np.array([800.0, 2000.0])
    s, tsi, mean, var = out.output_step_exact(p, np.zeros(2), tau_p, I0)
    assert np.allclose(mean, p, rtol=0, atol=1e-9 * np.sqrt(tau_p))
    assert np.allclose(var, tau_p, rtol=1e-9)
    assert np.allclose(s, 0.0, atol=1e-9 / np.sqrt(tau_p))
    assert np.allclose(tsi, 0.0, atol=1e-9 / tau_p)
