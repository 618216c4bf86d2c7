"""Pins of the state-evolution oracle (Section 4.4).

The generic recursion, fed the AWGN channel and the linear MMSE denoiser of
the i.i.d. Gaussian problem, must reproduce that problem's closed-form SE
(tau_r = sigma^2 + tau_x / delta, tau_x+ = tau_r / (1 + tau_r)) to the
accuracy of its single Monte-Carlo draws.  On a CT slice the recursion is
compared with the algorithm's own scalars (no closed form exists there).
"""
import numpy as np

import synth
from oracle import gamp, precond, state_evolution as se
from oracle.geometry import Geometry


def test_reduces_to_the_gaussian_closed_form():
    N, M, sigma2, T = 20000, 10000, 0.01, 8
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N)
    z = rng.standard_normal(M) * np.sqrt(N / M)        # Ax for A_ij ~ N(0, 1/M): variance N/M
    frob2 = float(N)                                   # E ||A||_F^2 = M N / M

    def gout(p, tau_p):
        return np.zeros_like(p), np.full_like(p, 1.0 / (sigma2 + tau_p))

    rec = se.state_evolution(z, x, frob2, gout, gamp.gaussian_prior_denoiser, T, seed=4)
    want = np.array(gamp.state_evolution_gaussian(M / N, sigma2, T))
    taux = np.array([r.tau_x for r in rec])
    mse = np.array([r.mse for r in rec])
    tr = np.array([r.tau_r for r in rec])
    # the chain tau_p -> tau_s -> tau_r is exact for this deterministic channel:
    # tau_r+ = sigma^2 + tau_x N / M from the recursion's own tau_x
    assert np.allclose(tr[1:], sigma2 + taux[:-1] * N / M, rtol=1e-12)
    assert tr[0] == sigma2 + 1.0 * N / M
    # tau_x (MC divergence of the linear denoiser: ||b||^2 / N carries ~1%
    # sampling error) and the error function follow the closed form to that accuracy
    assert np.allclose(taux, want, rtol=3e-2)
    assert np.allclose(mse, want, rtol=3e-2)


def test_ct_recursion_meets_the_algorithms_tau_r():
    c = synth.make_case("ellipse64_v30")
    g = Geometry(c["n"], c["n_views"], c["n_det"])
    frob2 = precond.frobenius_sq(g)
    opts = gamp.Options(c_tv=3.0, k_tv=20)
    rec = se.ct_state_evolution(c["y"], c["I0"], g, 12, opts, c["mu"], frob2=frob2, seed=5)
    log = []
    gamp.ct_solve(c["y"], c["I0"], g, 12, opts, frob2=frob2, log=log)
    se_tr = np.array([r.tau_r for r in rec])
    alg_tr = np.array([lg.tau_r for lg in log])
    # iteration 1: tau_p is so large that tau_s,i ~ 1/tau_p whatever the messages
    assert abs(se_tr[0] / alg_tr[0] - 1) < 1e-6
    assert np.all(np.abs(se_tr[6:] / alg_tr[6:] - 1) < 0.05)
    assert rec[-1].mse < 1e-3 * rec[0].mse
