"""Pins for the oracle's Radon preconditioner (Section 2.4, Eqs. PPFT/Aprecon/GramATA)."""
import math

import numpy as np
import pytest

from oracle import joseph, precond
from oracle.geometry import Geometry


def test_gain_definition():
    g = precond.detector_gain(16)
    assert g[0] == pytest.approx(math.sqrt(1 / 32))            # DC floor f0 = 1/(2P)
    assert g[8] == pytest.approx(math.sqrt(0.5))               # Nyquist
    assert g[3] == pytest.approx(math.sqrt(3 / 16)) and g[13] == pytest.approx(math.sqrt(3 / 16))


@pytest.mark.parametrize("geom", [Geometry(16, 3, 24), Geometry(20, 4, 29)])
def test_fft_filter_matches_direct_dft(geom):
    rng = np.random.default_rng(5)
    s = rng.standard_normal((geom.n_views, geom.n_det))
    T = precond.filter_matrix(geom)            # built from an O(P^2) cosine sum, no FFT
    ref = s @ T.T
    out = precond.filter_views(s, geom)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.allclose(T, T.T, rtol=0, atol=1e-13 * np.max(np.abs(T)))             # H = H^T (g real and even)


def test_frobenius_matches_dense_matrix():
    geom = Geometry(16, 12, 24)
    A = joseph.dense_matrix(geom)
    T = precond.filter_matrix(geom)
    HA = np.kron(np.eye(geom.n_views), T) @ A
    ref = float(np.sum(HA * HA))
    assert precond.frobenius_sq(geom) == pytest.approx(ref, rel=1e-12)


def test_preconditioned_operator_is_better_conditioned():
    # Eq. GramATA: A~^T A~ is close to a multiple of I; A^T A is not.
    geom = Geometry(16, 48, 24)
    A = joseph.dense_matrix(geom)
    T = precond.filter_matrix(geom)
    HA = np.kron(np.eye(geom.n_views), T) @ A
    ev_a = np.linalg.eigvalsh(A.T @ A)
    ev_p = np.linalg.eigvalsh(HA.T @ HA)
    assert ev_p[-1] / ev_p[0] < (ev_a[-1] / ev_a[0]) / 3
    spread = lambda e: np.percentile(e, 90) / np.percentile(e, 10)
    assert spread(ev_p) < 0.75 * spread(ev_a)
    # the un-normalised gain gives A~^T A~ ~ (N_theta / pi) I at the top of the spectrum
    assert ev_p[-1] == pytest.approx(geom.n_views / math.pi, rel=0.1)


def test_fourier_slice_consistency_of_1d_and_2d_filters():
    # A V^-1 mu ~= H A mu for a smooth, compact image (Eq. Aprecon).
    n = 64
    geom = Geometry(n, 16, 95)
    c = (n - 1) / 2
    X = np.arange(n)[None, :] - c
    Y = c - np.arange(n)[:, None]
    img = np.exp(-((X - 3) ** 2 + (Y + 2) ** 2) / (2 * 4.0 ** 2))
    a = joseph.forward_project(precond.v_inverse(img, geom), geom)
    b = precond.filter_views(joseph.forward_project(img, geom), geom)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.08


def test_image_filters_are_mutual_inverses_on_padded_grid():
    # V and V^-1 use reciprocal gains; on an image whose support is the top-left
    # quarter of the padded grid the composition is the identity up to the crop.
    geom = Geometry(32, 4, 47)
    rng = np.random.default_rng(6)
    img = np.zeros((32, 32))
    img[:8, :8] = rng.standard_normal((8, 8))
    back = precond.v_forward(precond.v_inverse(img, geom), geom)
    assert np.linalg.norm(back - img) / np.linalg.norm(img) < 0.3
