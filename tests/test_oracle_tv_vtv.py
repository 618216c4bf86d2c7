"""Pins of the oracle's prox-TV in the (V^T V)^{-1} norm (Section 6.3).

Each check rests on a fact other than the oracle's own formulas:
* Parseval on the padded grid for the covariance Q (its quadratic form from
  the spectra of the two images, never through the cropped filter);
* Q = I reduces the problem to the l2 prox, which Chambolle's 2004 projection
  (a different algorithm) solves;
* weak duality: any x and any feasible p bound the optimum from both sides,
  so a vanishing gap certifies the minimiser, with Q^{-1} formed densely;
* the dual ascent never decreases (the step is 1/L);
* the limits lambda -> 0 (x = r) and large lambda (x = the Q^{-1}-weighted
  mean of r, the only minimiser once TV must vanish).
"""
import numpy as np
import pytest

from oracle import precond as pre
from oracle import tv
from oracle.geometry import Geometry


def dense(op, n):
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(op(e.reshape(n, n)).reshape(-1))
    return np.array(cols).T


def primal(x, r, lam, Qinv):
    d = (x - r).reshape(-1)
    return 0.5 * d @ Qinv @ d + lam * tv.tv_value(x)


def dual(px, py, r, lam, Qd):
    d = tv.div(px, py).reshape(-1)
    return -0.5 * lam * lam * d @ Qd @ d - lam * r.reshape(-1) @ d


def phantom(n, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:n, 0:n]
    img = ((xx - n / 2) ** 2 + (yy - n / 2.5) ** 2 < (n / 3) ** 2).astype(float)
    img += 0.5 * ((xx > n // 4) & (xx < n // 2) & (yy > n // 2)).astype(float)
    return img + 0.1 * rng.standard_normal((n, n))


@pytest.mark.parametrize("n,nd", [(6, 9), (12, 17)])
def test_covariance_quadratic_form_is_parseval(n, nd):
    g = Geometry(n, 5, nd)
    rng = np.random.default_rng(n)
    u, v = rng.standard_normal((2, n, n))
    m = pre.image_pad(g)
    assert m >= 2 * n and m & (m - 1) == 0
    U = np.fft.fft2(np.pad(u, ((0, m - n), (0, m - n))))
    V = np.fft.fft2(np.pad(v, ((0, m - n), (0, m - n))))
    f = np.fft.fftfreq(m)
    rho = np.hypot(f[:, None], f[None, :])
    gain = np.maximum(rho, 1.0 / (2 * g.P))
    want = float(np.sum(gain * (U * np.conj(V)).real)) / (m * m)
    assert float(np.sum(u * pre.vtv_inverse(v, g))) == pytest.approx(want, rel=1e-12)
    Q = dense(lambda a: pre.vtv_inverse(a, g), n)
    assert np.allclose(Q, Q.T, atol=1e-14)
    ev = np.linalg.eigvalsh(Q)
    assert ev.min() > 0.0
    assert ev.max() <= pre.vtv_inverse_norm_bound(g) + 1e-12
    assert pre.vtv_inverse_norm_bound(g) == pytest.approx(np.sqrt(0.5))


@pytest.mark.parametrize("lam", [0.1, 0.2])
def test_identity_covariance_gives_the_l2_prox(lam):
    r = phantom(8, 3)
    a = tv.tv_prox_metric(r, lam, 20000, lambda u: u, 1.0)
    b = tv.tv_prox(r, lam, 40000)          # Chambolle 2004 converges more slowly
    assert np.max(np.abs(a - b)) < 1e-8 * np.max(np.abs(r))


@pytest.mark.parametrize("lam", [0.05, 0.3])
def test_duality_gap_certifies_the_minimiser(lam):
    n = 12
    g = Geometry(n, 7, 17)
    Qf = lambda u: pre.vtv_inverse(u, g)
    Q = dense(Qf, n)
    Qinv = np.linalg.inv(Q)
    r = phantom(n, 5)
    x, px, py, hist = tv.tv_prox_metric_dual(r, lam, 20000, Qf, pre.vtv_inverse_norm_bound(g))
    assert np.max(np.sqrt(px * px + py * py)) <= 1.0 + 1e-12
    P, D = primal(x, r, lam, Qinv), dual(px, py, r, lam, Q)
    assert P >= D - 1e-12                          # weak duality
    assert P - D < 1e-7 * abs(P)
    # the returned map is the same iteration
    x2 = tv.tv_prox_metric(r, lam, 20000, Qf, pre.vtv_inverse_norm_bound(g))
    assert np.array_equal(x, x2)
    # and x beats nearby points on the primal objective
    rng = np.random.default_rng(0)
    for _ in range(20):
        assert primal(x + 1e-3 * rng.standard_normal(x.shape), r, lam, Qinv) > P


def test_dual_ascent_is_monotone():
    n = 16
    g = Geometry(n, 9, 23)
    r = phantom(n, 7)
    _x, _px, _py, hist = tv.tv_prox_metric_dual(r, 0.2, 300, lambda u: pre.vtv_inverse(u, g),
                                                  pre.vtv_inverse_norm_bound(g))
    h = np.array(hist)
    assert np.all(np.diff(h) >= -1e-12 * np.abs(h[1:]).max())
    assert h[-1] > h[1] > h[0] == 0.0


def test_lambda_limits():
    n = 8
    g = Geometry(n, 5, 13)
    Qf = lambda u: pre.vtv_inverse(u, g)
    qb = pre.vtv_inverse_norm_bound(g)
    r = phantom(n, 11)
    assert np.array_equal(tv.tv_prox_metric(r, 0.0, 50, Qf, qb), r)
    # with lambda above the largest dual norm the minimiser is flat: the
    # constant c minimising (c1 - r)^T Q^{-1} (c1 - r)
    Qinv = np.linalg.inv(dense(Qf, n))
    one = np.ones(n * n)
    c = (one @ Qinv @ r.reshape(-1)) / (one @ Qinv @ one)
    x = tv.tv_prox_metric(r, 50.0, 40000, Qf, qb)
    assert np.max(np.abs(x - c)) < 1e-6
    assert tv.tv_value(x) < 1e-6
