"""Radon preconditioner of Section 2.4 / 4.1 (Eqs. PPFT preconditioner, Aprecon).

The paper's right preconditioner is V = F^-1 C^{1/2} F with
C = diag(1/|rho|), so V^-1 applies the radial gain |rho|^{1/2}.  By the
Fourier slice theorem (Eq. Radon_op) a radial gain on the 2-D spectrum of the
image is the same gain on the 1-D detector-axis spectrum of every view, so

    Phi~ = S A V^-1 = H A,   Phi~^T = V^-1 A^T S^T = A^T H,

with H (per view) = crop o IFFT_P o diag(g) o FFT_P o zero-pad and
g_k = sqrt(max(|f_k|, f0)), f_k the signed frequency k/P in cycles per
detector bin.  g is real and even, so H is real-symmetric (Eq. precondAMP_op
then needs no separate transpose).

Readings where the paper is silent or singular:

* DC: C is singular at rho = 0; the gain is floored at f0 = 1/(2P), which
  touches only the DC bin.
* scale: the paper states A~^T A~ = I (Eq. GramATA) with no constant; the gain
  is kept un-normalised, so x = V mu does not change units with the view
  count.  GAMP absorbs the scale through ||Phi~||_F^2 (Algorithm 1).
* the image-domain map V^-1 used for the returned mu (Algorithm 1, return
  line) is the 2-D radial gain sqrt(max(rho, f0)) on an m x m zero-padded
  FFT, m the smallest power of two >= 2n (the paper gives no padding),
  cropped back to n x n; V uses the reciprocal gain.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Geometry
from . import joseph


def detector_gain(P: int) -> np.ndarray:
    """g_k = sqrt(max(|f_k|, 1/(2P))) for k = 0..P-1 (signed FFT frequencies)."""
    k = np.arange(P)
    f = np.where(k <= P // 2, k, k - P) / P
    return np.sqrt(np.maximum(np.abs(f), 1.0 / (2 * P)))


def filter_views(sino: np.ndarray, geom: Geometry) -> np.ndarray:
    """H applied to every view: zero-pad to P, FFT, times g, IFFT, crop."""
    sino = np.asarray(sino, dtype=np.float64).reshape(geom.n_views, geom.n_det)
    P = geom.P
    pad = np.zeros((geom.n_views, P))
    pad[:, :geom.n_det] = sino
    spec = np.fft.fft(pad, axis=1) * detector_gain(P)[None, :]
    return np.fft.ifft(spec, axis=1).real[:, :geom.n_det]


def filter_kernel_direct(P: int) -> np.ndarray:
    """h[m] = (1/P) sum_k g_k cos(2 pi k m / P), by an O(P^2) direct sum.

    Because g is real and even, H z[d] = sum_d' h[(d - d') mod P] z[d'] for
    zero-padded input; this is the circulant form of H, written without an FFT.
    """
    g = detector_gain(P)
    m = np.arange(P)
    k = np.arange(P)
    ang = 2.0 * math.pi * np.outer(m, k) / P
    return (np.cos(ang) @ g) / P


def filter_matrix(geom: Geometry) -> np.ndarray:
    """Dense T (n_det x n_det) with T[i, j] = h[(i - j) mod P]: H for one view."""
    h = filter_kernel_direct(geom.P)
    i = np.arange(geom.n_det)
    return h[(i[:, None] - i[None, :]) % geom.P]


def project(x: np.ndarray, geom: Geometry) -> np.ndarray:
    """z = Phi~ x = H A x (Algorithm 1, Step 1)."""
    return filter_views(joseph.forward_project(x, geom), geom)


def backproject(s: np.ndarray, geom: Geometry) -> np.ndarray:
    """Phi~^T s = A^T H s (Algorithm 1, Step 3)."""
    return joseph.back_project(filter_views(s, geom), geom)


def frobenius_sq(geom: Geometry) -> float:
    """||Phi~||_F^2 = sum_k trace(T^T T G_k), G_k = A_k A_k^T (Algorithm 1, Steps 1 and 3).

    T is the per-view matrix of H (the same for every view); G_k is
    tridiagonal, so only the band |i - j| <= 1 of T^T T contributes.  Both
    are built exactly, so this equals the squared Frobenius norm of the
    dense M x N matrix H A up to rounding.
    """
    T = filter_matrix(geom)
    TT = T.T @ T
    tot = 0.0
    for k in range(geom.n_views):
        G = joseph.view_gram(geom, k)
        tot += float(np.sum(TT * G))
    return tot


def _radial_gain_2d(m: int, P: int, inverse: bool) -> np.ndarray:
    fy = np.fft.fftfreq(m)[:, None]
    fx = np.fft.fftfreq(m)[None, :]
    rho = np.sqrt(fx * fx + fy * fy)
    g = np.sqrt(np.maximum(rho, 1.0 / (2 * P)))
    return 1.0 / g if inverse else g


def _image_filter(img: np.ndarray, geom: Geometry, inverse: bool) -> np.ndarray:
    n = geom.n
    m = 1 << (2 * n - 1).bit_length()      # smallest power of two >= 2n
    pad = np.zeros((m, m))
    pad[:n, :n] = img
    spec = np.fft.fft2(pad) * _radial_gain_2d(m, geom.P, inverse)
    return np.fft.ifft2(spec).real[:n, :n]


def v_inverse(x: np.ndarray, geom: Geometry) -> np.ndarray:
    """mu = V^-1 x (Algorithm 1, return line): radial gain sqrt(max(rho, f0))."""
    return _image_filter(np.asarray(x, dtype=np.float64), geom, inverse=False)


def v_forward(mu: np.ndarray, geom: Geometry) -> np.ndarray:
    """x = V mu (Eq. precondAMP): radial gain 1/sqrt(max(rho, f0))."""
    return _image_filter(np.asarray(mu, dtype=np.float64), geom, inverse=True)


# -------------------------------------------------- (V^T V)^{-1} ----
# The covariance that the preconditioner gives white noise seen through V^-1
# (Eq. r_input: r = x + tau_r V^-1 Phi^T s).  On the paper's Fourier grid
# V = F^-1 C^{1/2} F, so (V^T V)^{-1} = F^-1 C^-1 F, the radial gain |rho|.
# It is realised like V^-1: the gain max(rho, f0) (the square of V^-1's) on
# the same m x m zero-padded grid, cropped back to n x n.  The result Q is
# symmetric and positive definite (a principal block of a positive definite
# circulant), and ||Q|| <= the largest gain on the grid.

def _vtv_gain(m: int, P: int) -> np.ndarray:
    fy = np.fft.fftfreq(m)[:, None]
    fx = np.fft.fftfreq(m)[None, :]
    return np.maximum(np.sqrt(fx * fx + fy * fy), 1.0 / (2 * P))


def image_pad(geom: Geometry) -> int:
    """m, the side of the zero-padded grid of the image-domain filters."""
    return 1 << (2 * geom.n - 1).bit_length()


def vtv_inverse(u: np.ndarray, geom: Geometry) -> np.ndarray:
    """Q u with Q = (V^T V)^{-1}: zero-pad to m x m, FFT, times max(rho, f0),
    IFFT, crop."""
    n, m = geom.n, image_pad(geom)
    pad = np.zeros((m, m))
    pad[:n, :n] = np.asarray(u, dtype=np.float64)
    return np.fft.ifft2(np.fft.fft2(pad) * _vtv_gain(m, geom.P)).real[:n, :n]


def vtv_inverse_norm_bound(geom: Geometry) -> float:
    """The largest gain of Q on its grid, a bound on ||Q||."""
    return float(_vtv_gain(image_pad(geom), geom.P).max())
