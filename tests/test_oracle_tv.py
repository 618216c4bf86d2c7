"""Pins for the oracle's proximal TV denoiser (Section 6.3)."""
import numpy as np
import pytest

from oracle import tv


def test_zero_lambda_is_identity():
    r = np.random.default_rng(1).standard_normal((12, 9))
    assert np.array_equal(tv.tv_prox(r, 0.0, 50), r)


def test_constant_image_is_fixed_point():
    r = np.full((10, 10), 3.25)
    assert np.allclose(tv.tv_prox(r, 0.7, 40), r, atol=1e-14)


def test_div_is_negative_adjoint_of_grad():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((7, 11))
    px, py = rng.standard_normal((2, 7, 11))
    gx, gy = tv.grad(u)
    lhs = np.sum(gx * px + gy * py)
    rhs = -np.sum(u * tv.div(px, py))
    # boundary entries of p are not seen by grad's zero last difference; restrict p
    px[:, -1] = 0
    py[-1, :] = 0
    lhs = np.sum(gx * px + gy * py)
    rhs = -np.sum(u * tv.div(px, py))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_step_edge_closed_form():
    # Rows identical -> isotropic TV reduces to 1-D TV per row.  For a step of
    # height h between two halves of length m, the prox keeps the edge and moves
    # each plateau by lambda/m towards the other (h > 2 lambda / m).
    n, m, h, lam = 16, 8, 1.0, 1.2
    r = np.zeros((n, n))
    r[:, m:] = h
    x = tv.tv_prox(r, lam, 6000)
    assert np.allclose(x[:, :m], lam / m, atol=1e-6)
    assert np.allclose(x[:, m:], h - lam / m, atol=1e-6)


def test_objective_decreases_with_iterations():
    rng = np.random.default_rng(3)
    r = np.cumsum(rng.standard_normal((24, 24)), axis=1) * 0.1
    lam = 0.3
    obj = lambda x: 0.5 * np.sum((x - r) ** 2) + lam * tv.tv_value(x)
    vals = [obj(tv.tv_prox(r, lam, k)) for k in (5, 20, 80, 320)]
    assert vals[0] > vals[1] > vals[2] > vals[3]
    assert vals[3] < obj(r)
