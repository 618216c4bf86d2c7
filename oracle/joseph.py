"""System matrix A of Eq. (linCT): ray-driven Joseph interpolation.

The paper builds A with the ASTRA toolbox and leaves the pixel-ray weights
a_ij open (Section 2.1).  This oracle uses Joseph's method (Joseph 1982, IEEE
TMI 1:192), a published line-integral discretisation:

* a view whose rays run mostly along X (|sin theta| >= |cos theta|; the tie
  goes here) is marched column by column: in column ix the ray sits at
  Y = (u - X cos theta) / sin theta, i.e. at fractional row
  r = (n-1)/2 - Y, and contributes the linear interpolation between rows
  floor(r) and floor(r)+1, times the path length per column 1/|sin theta|;
* any other view is marched row by row: at row iy the ray sits at
  X = (u - Y sin theta) / cos theta, fractional column c = X + (n-1)/2,
  step weight 1/|cos theta|;
* an interpolation neighbour outside [0, n-1] contributes zero.

``back_project`` is the exact transpose (same weights, scattered), which is
what Algorithm 1 needs for Phi^T.  ``dense_matrix`` builds A entry by entry
from the hat-function form of the same definition, for brute-force checks on
tiny images.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Geometry


def _view_taps(geom: Geometry, theta: float):
    """Return (flat pixel index [2, nd, n], weight [2, nd, n]) of one view."""
    n, c = geom.n, geom.centre()
    u = geom.det_offsets()[:, None]               # (nd, 1)
    st, ct = math.sin(theta), math.cos(theta)
    steps = np.arange(n, dtype=np.float64)[None, :]  # (1, n)
    if abs(st) >= abs(ct):
        X = steps - c                               # column centres
        frac_row = c - (u - X * ct) / st            # (nd, n)
        i0 = np.floor(frac_row)
        f = frac_row - i0
        w = 1.0 / abs(st)
        rows = np.stack([i0, i0 + 1.0])             # (2, nd, n)
        cols = np.broadcast_to(steps, rows.shape)
        wts = np.stack([(1.0 - f) * w, f * w])
    else:
        Y = c - steps                               # row centres
        frac_col = (u - Y * st) / ct + c
        i0 = np.floor(frac_col)
        f = frac_col - i0
        w = 1.0 / abs(ct)
        cols = np.stack([i0, i0 + 1.0])
        rows = np.broadcast_to(steps, cols.shape)
        wts = np.stack([(1.0 - f) * w, f * w])
    ok = (rows >= 0) & (rows <= n - 1) & (cols >= 0) & (cols <= n - 1)
    idx = np.where(ok, rows * n + cols, 0).astype(np.int64)
    wts = np.where(ok, wts, 0.0)
    return idx, wts


def forward_project(img: np.ndarray, geom: Geometry) -> np.ndarray:
    """z = A img, shape [n_views][n_det] (Eq. linCT)."""
    flat = np.asarray(img, dtype=np.float64).reshape(-1)
    assert flat.size == geom.N
    out = np.zeros((geom.n_views, geom.n_det))
    for k, th in enumerate(geom.thetas()):
        idx, wts = _view_taps(geom, th)
        out[k] = (flat[idx] * wts).sum(axis=(0, 2))
    return out


def back_project(sino: np.ndarray, geom: Geometry) -> np.ndarray:
    """img = A^T sino, shape [n][n] (transpose of :func:`forward_project`)."""
    sino = np.asarray(sino, dtype=np.float64).reshape(geom.n_views, geom.n_det)
    acc = np.zeros(geom.N)
    for k, th in enumerate(geom.thetas()):
        idx, wts = _view_taps(geom, th)
        vals = wts * sino[k][None, :, None]
        acc += np.bincount(idx.reshape(-1), weights=vals.reshape(-1), minlength=geom.N)
    return acc.reshape(geom.n, geom.n)


def dense_matrix(geom: Geometry) -> np.ndarray:
    """Brute-force A (M x N), one (ray, pixel) pair at a time.

    For the ray's marching axis, pixel (ix, iy) gets weight
    step * max(0, 1 - |s - k|), where k is the pixel's index across the
    marching direction and s is the ray's fractional position in the pixel's
    own column (or row).  This is the hat-function reading of linear
    interpolation, evaluated independently of the floor/fraction taps above.
    """
    n, c = geom.n, geom.centre()
    A = np.zeros((geom.M, geom.N))
    us = geom.det_offsets()
    for k, th in enumerate(geom.thetas()):
        st, ct = math.sin(th), math.cos(th)
        for d, u in enumerate(us):
            row = k * geom.n_det + d
            for iy in range(n):
                for ix in range(n):
                    if abs(st) >= abs(ct):
                        s = c - (u - (ix - c) * ct) / st
                        wgt = max(0.0, 1.0 - abs(s - iy)) / abs(st)
                    else:
                        s = (u - (c - iy) * st) / ct + c
                        wgt = max(0.0, 1.0 - abs(s - ix)) / abs(ct)
                    A[row, iy * n + ix] = wgt
    return A


def view_matrix(geom: Geometry, k: int):
    """Sparse A_k (n_det x N): the rows of A that belong to view k."""
    import scipy.sparse as sp
    idx, wts = _view_taps(geom, geom.thetas()[k])
    nd, n = geom.n_det, geom.n
    rows = np.broadcast_to(np.arange(nd)[None, :, None], idx.shape)
    A = sp.coo_matrix((wts.reshape(-1), (rows.reshape(-1), idx.reshape(-1))),
                      shape=(nd, geom.N)).tocsr()
    A.sum_duplicates()
    return A


def view_gram(geom: Geometry, k: int) -> np.ndarray:
    """G_k = A_k A_k^T for view k, dense (n_det x n_det).

    Two rays of one view share a pixel only when their interpolation
    positions differ by less than 2, i.e. |d - d'| < 2|sin| (or 2|cos|) <= 2,
    so G_k is tridiagonal; the tests check that on the full product.
    """
    A = view_matrix(geom, k)
    return (A @ A.T).toarray()
