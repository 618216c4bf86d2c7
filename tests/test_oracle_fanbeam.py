"""Pins of the fan-beam oracle (flat detector, Section 6 geometry).

* parallel rays through the generic-line Joseph taps reproduce the parallel
  oracle (itself pinned against analytic integrals and a dense matrix);
* a source and detector a million image widths away reduce the fan to the
  parallel geometry (magnified detector);
* the hat-function dense matrix, built pixel by pixel, equals the taps, and
  back-projection is its transpose;
* rotating the image by 90 degrees equals rotating the views by -90 degrees;
* ray sums of a smooth Gaussian blob match its closed-form line integral;
* the analytic fan sinogram of the synthetic inputs (an independent
  implementation of the same geometry) matches the projected phantom;
* ||Phi~||_F^2 summed over rays equals the sum over image columns.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fanbeam, joseph, precond
from oracle.geometry import Geometry


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_parallel_rays_reproduce_the_parallel_oracle():
    g = Geometry(9, 8, 13, angles=tuple(np.linspace(0, math.pi, 8, endpoint=False)))   # 45 deg tie included
    img = rnd((9, 9), 1)
    want = joseph.forward_project(img, g)
    got = np.zeros_like(want)
    flat = img.reshape(-1)
    for k, th in enumerate(g.thetas()):
        for d, u in enumerate(g.det_offsets()):
            idx, w = fanbeam.line_taps(9, (u * math.cos(th), u * math.sin(th)), (-math.sin(th), math.cos(th)))
            got[k, d] = np.sum(flat[idx] * w)
    assert np.max(np.abs(got - want)) < 1e-12


def test_far_source_is_parallel_beam():
    ang = tuple(np.linspace(0.1, 2 * math.pi, 6, endpoint=False))
    far = fanbeam.FanGeometry(16, 6, 23, 1e7, 1e7, det_spacing=2.0, angles=ang)   # magnification 2
    par = Geometry(16, 6, 23, angles=ang)
    img = rnd((16, 16), 2)
    a, b = fanbeam.forward_project(img, far), joseph.forward_project(img, par)
    assert np.max(np.abs(a - b)) < 1e-5 * np.max(np.abs(b))


def test_dense_matrix_and_transpose():
    g = fanbeam.FanGeometry(6, 5, 9, 9.0, 7.0, det_spacing=1.3)
    A = fanbeam.dense_matrix(g)
    x, s = rnd((6, 6), 3), rnd((5, 9), 4)
    assert np.allclose(fanbeam.forward_project(x, g).reshape(-1), A @ x.reshape(-1), atol=1e-12)
    assert np.allclose(fanbeam.back_project(s, g).reshape(-1), A.T @ s.reshape(-1), atol=1e-12)
    assert (A > 0).sum(axis=1).min() > 0          # every ray crosses the image


def test_rotating_the_image_rotates_the_views():
    ang = np.array([0.13, 0.9, 2.2, 4.0])
    g0 = fanbeam.FanGeometry(12, 4, 21, 20.0, 15.0, 1.1, angles=tuple(ang))
    g1 = fanbeam.FanGeometry(12, 4, 21, 20.0, 15.0, 1.1, angles=tuple(ang - math.pi / 2))
    img = rnd((12, 12), 5)
    a = fanbeam.forward_project(np.rot90(img), g0)
    b = fanbeam.forward_project(img, g1)
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b))


def test_gaussian_blob_ray_sums():
    # Joseph's linear interpolation errs by about h^2 / (8 sigma^2) of the peak
    n, sig, (x0, y0) = 64, 5.0, (4.3, -6.1)
    c = (n - 1) / 2
    X, Y = np.meshgrid(np.arange(n) - c, c - np.arange(n))
    img = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * sig * sig))
    g = fanbeam.FanGeometry(n, 7, 83, 109.0, 80.0, 1.5)
    z = fanbeam.forward_project(img, g)
    S, v = g.rays()
    vh = v / np.linalg.norm(v, axis=-1, keepdims=True)
    dist = (x0 - S[..., 0]) * vh[..., 1] - (y0 - S[..., 1]) * vh[..., 0]
    want = math.sqrt(2 * math.pi) * sig * np.exp(-dist ** 2 / (2 * sig * sig))
    assert np.max(np.abs(z - want)) < 6e-3 * want.max()


def test_synthetic_fan_sinogram_matches_the_projected_phantom():
    c = synth.make_case("fan64_v30")
    f = c["fan"]
    g = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"])
    assert np.allclose(g.thetas(), c["angles"])
    z = fanbeam.forward_project(c["mu"], g)
    err = np.linalg.norm(z - c["z"]) / np.linalg.norm(c["z"])
    assert err < 3e-2
    # the same phantom seen with the views mirrored is far off
    gm = fanbeam.FanGeometry(c["n"], c["n_views"], c["n_det"], f["src_dist"], f["det_dist"], f["det_spacing"],
                             angles=tuple(-c["angles"]))
    assert np.linalg.norm(fanbeam.forward_project(c["mu"], gm) - c["z"]) / np.linalg.norm(c["z"]) > 10 * err


def test_frobenius_norm_two_ways():
    g = fanbeam.FanGeometry(6, 4, 11, 10.0, 8.0, 1.2)
    by_rows = fanbeam.frobenius_sq(g)
    by_cols = 0.0
    for j in range(g.N):
        e = np.zeros(g.N)
        e[j] = 1.0
        by_cols += float(np.sum(fanbeam.project(e.reshape(6, 6), g) ** 2))
    assert by_rows == pytest.approx(by_cols, rel=1e-12)
    # Phi~^T is the transpose of Phi~
    x, s = rnd((6, 6), 6), rnd((4, 11), 7)
    assert np.sum(fanbeam.project(x, g) * s) == pytest.approx(np.sum(x * fanbeam.backproject(s, g)), rel=1e-12)


def test_geometry_must_enclose_the_image():
    with pytest.raises(ValueError):
        fanbeam.FanGeometry(64, 10, 96, 40.0, 92.0, 1.95)
    assert precond.image_pad(fanbeam.FanGeometry(64, 10, 96, 112.0, 92.0, 1.95)) == 128


def test_stored_fan_frobenius_is_the_oracles():
    """tests/golden/fan_frobenius.txt (written by make_fan_frobenius.py from
    the oracle alone): the small workload's entry is recomputed here."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fan_frobenius.txt")
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, v = line.split()
            vals[name] = float(v)
    assert set(vals) == {"fan64_v30", "fan512_v102"}
    n, nv, nd, _ne, _rm, _rect, _I0, _it, sd, dd, ds = synth.FAN_CASES["fan64_v30"]
    g = fanbeam.FanGeometry(n, nv, nd, sd, dd, ds)
    assert vals["fan64_v30"] == pytest.approx(fanbeam.frobenius_sq(g), rel=1e-12)
    assert vals["fan512_v102"] > 0


def test_synthetic_fan_lines_pass_through_source_and_bin():
    """synth.fan_lines (the synthetic counts' geometry, written apart from the
    oracle): every line (theta', u') contains the source and its bin's point
    on the detector, as the oracle's rays do."""
    ang = np.array([0.0, 0.7, 2.0, 3.9, 5.5])
    sd, dd, du, nd = 90.0, 70.0, 1.7, 23
    thp, up = synth.fan_lines(ang, nd, sd, dd, du)
    g = fanbeam.FanGeometry(40, len(ang), nd, sd, dd, du, angles=tuple(ang))
    S, v = g.rays()
    T = S + v
    for P in (S, T):
        resid = P[..., 0] * np.cos(thp) + P[..., 1] * np.sin(thp) - up
        assert np.max(np.abs(resid)) < 1e-9
