"""Pins for the oracle's Joseph system matrix (Eq. linCT, Section 2.1)."""
import math

import numpy as np
import pytest

import synth
from oracle import joseph
from oracle.geometry import Geometry

GEOMS = [
    Geometry(16, 12, 24),                # even detector count, incl. the 45-degree tie
    Geometry(16, 7, 23),                 # odd count, half-pixel detector offset
    Geometry(9, 5, 13, angles=(0.1, 1.0, 2.0, 2.9, -0.7)),  # arbitrary angles, odd image
]


@pytest.mark.parametrize("geom", GEOMS)
def test_forward_matches_bruteforce_matrix(geom):
    A = joseph.dense_matrix(geom)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((geom.n, geom.n))
    z = joseph.forward_project(x, geom).reshape(-1)
    assert np.max(np.abs(z - A @ x.reshape(-1))) <= 1e-13 * np.max(np.abs(z))


@pytest.mark.parametrize("geom", GEOMS)
def test_backproject_is_transpose(geom):
    A = joseph.dense_matrix(geom)
    rng = np.random.default_rng(2)
    s = rng.standard_normal((geom.n_views, geom.n_det))
    bp = joseph.back_project(s, geom).reshape(-1)
    assert np.max(np.abs(bp - A.T @ s.reshape(-1))) <= 1e-13 * np.max(np.abs(bp))


def test_adjoint_identity_large():
    geom = Geometry(96, 17, 139)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((geom.n, geom.n))
    s = rng.standard_normal((geom.n_views, geom.n_det))
    lhs = float(np.sum(joseph.forward_project(x, geom) * s))
    rhs = float(np.sum(x * joseph.back_project(s, geom)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_axis_aligned_views_are_column_and_row_sums():
    # n and n_det both even: bins line up with pixel centres at 0 and 90 degrees.
    geom = Geometry(16, 2, 16)        # theta = 0 and pi/2
    rng = np.random.default_rng(4)
    x = rng.uniform(size=(16, 16))
    z = joseph.forward_project(x, geom)
    # theta = 0: ray X = u_d is the column ix = d.
    assert np.allclose(z[0], x.sum(axis=0), rtol=0, atol=1e-12)
    # theta = pi/2: ray Y = u_d is the row iy = n-1-d (row 0 is the top).
    assert np.allclose(z[1], x.sum(axis=1)[::-1], rtol=0, atol=1e-12)


def test_gaussian_blob_matches_continuous_radon_transform():
    # The line integral of exp(-|v - v0|^2 / 2s^2) is sqrt(2 pi) s exp(-(u - u0)^2 / 2s^2)
    # with u0 = X0 cos(theta) + Y0 sin(theta): this pins signs and orientation.
    n, s = 64, 5.0
    geom = Geometry(n, 12, 95)
    c = (n - 1) / 2
    X = np.arange(n)[None, :] - c
    Y = c - np.arange(n)[:, None]
    X0, Y0 = 7.3, -4.1
    img = np.exp(-((X - X0) ** 2 + (Y - Y0) ** 2) / (2 * s * s))
    z = joseph.forward_project(img, geom)
    u = geom.det_offsets()[None, :]
    th = geom.thetas()[:, None]
    za = math.sqrt(2 * math.pi) * s * np.exp(-(u - X0 * np.cos(th) - Y0 * np.sin(th)) ** 2 / (2 * s * s))
    assert np.linalg.norm(z - za) / np.linalg.norm(za) < 5e-3
    # and a flipped Y convention would miss badly
    za_flip = math.sqrt(2 * math.pi) * s * np.exp(-(u - X0 * np.cos(th) + Y0 * np.sin(th)) ** 2 / (2 * s * s))
    assert np.linalg.norm(z - za_flip) / np.linalg.norm(za_flip) > 0.1


def test_ellipse_phantom_converges_to_analytic_integrals():
    ph = synth.random_phantom(32, 4, 7)
    errs = []
    for scale in (1, 2, 4):
        n = 32 * scale
        ells = tuple(synth.Ellipse(e.x0 * scale, e.y0 * scale, e.a * scale, e.b * scale, e.phi, e.rho)
                     for e in ph.ellipses)
        p2 = synth.Phantom(ells)
        geom = Geometry(n, 10, int(1.5 * n))
        img = synth.rasterise(p2, n, 8)
        z = joseph.forward_project(img, geom) / scale      # unit-length rescaling
        za = synth.analytic_sinogram(p2, geom.thetas(), geom.n_det) / scale
        errs.append(np.linalg.norm(z - za) / np.linalg.norm(za))
    assert errs[0] < 0.1
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]


@pytest.mark.parametrize("geom", GEOMS[:2])
def test_view_gram_is_tridiagonal(geom):
    for k in range(geom.n_views):
        G = joseph.view_gram(geom, k)
        band = np.abs(np.subtract.outer(np.arange(geom.n_det), np.arange(geom.n_det))) <= 1
        assert np.all(G[~band] == 0.0)
