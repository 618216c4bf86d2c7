"""Fan-beam system matrix and its preconditioned operator (Sections 2.1, 2.4, 6).

The paper's experiments use a flat-detector fan beam (ASTRA, Section 6 and
Fig. 1(a)); its method (Eq. precondAMP_op: Phi~ = S A V^-1) holds for any A.
This module restates both for the fan-beam A, under these readings:

* geometry: at view angle theta the source sits at src_dist (sin, -cos),
  the detector centre at det_dist (-sin, cos) and bin d at the detector
  centre plus u_d (cos, sin), u_d = (d - (n_det-1)/2) det_spacing (all in
  pixel units; pixel centres as in :mod:`oracle.geometry`).  The central ray
  runs along (-sin theta, cos theta), the direction of the parallel-beam ray
  (theta, 0), so theta means the same in both geometries.  Views default to
  theta_k = 2 pi k / n_views (a full rotation).  The source and the
  detector lie outside the image's circumscribed circle, so each ray's
  line integral over the image is the integral over the whole line;
* A: Joseph's method (Joseph 1982) along each ray's own direction v: a ray
  with |v_x| >= |v_y| (ties included) is marched column by column, sitting in
  column ix at Y = S_y + (X - S_x) v_y / v_x and weighting the linear
  interpolation between the two nearest rows by |v| / |v_x|; any other ray is
  marched row by row with X = S_x + (Y - S_y) v_x / v_y and weight |v| / |v_y|;
  neighbours outside the image contribute zero.  For the parallel ray
  (S = u (cos, sin), v = (-sin, cos)) these are the parallel oracle's taps;
* the preconditioner is the image-domain V^-1 of :mod:`oracle.precond`
  (the paper's cone filter, Section 2.4; it names no resampling for fan
  beam), so Phi~ = A V^-1 and Phi~^T = V^-1 A^T (V^-1 is symmetric), and
  ||Phi~||_F^2 = sum_i ||V^-1 a_i||^2 over the rows a_i of A;
* the detector-axis length P that fixes V^-1's DC floor 1/(2P) is the
  smallest power of two >= 2 n_det, as for parallel beam.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import precond as _pre


@dataclasses.dataclass(frozen=True)
class FanGeometry:
    n: int
    n_views: int
    n_det: int
    src_dist: float
    det_dist: float
    det_spacing: float = 1.0
    angles: tuple | None = None

    def __post_init__(self):
        r = self.n / math.sqrt(2.0)
        if not (self.src_dist > r and self.det_dist > r and self.det_spacing > 0):
            raise ValueError("source and detector must lie outside the image's circumscribed circle")

    def thetas(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, dtype=np.float64)
        return np.arange(self.n_views, dtype=np.float64) * (2.0 * math.pi / self.n_views)

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def M(self) -> int:
        return self.n_views * self.n_det

    @property
    def P(self) -> int:
        p = 1
        while p < 2 * self.n_det:
            p *= 2
        return p

    def centre(self) -> float:
        return (self.n - 1) / 2.0

    def rays(self):
        """Source points S and directions v (to the bin), each [n_views][n_det][2]."""
        th = self.thetas()[:, None]
        u = (np.arange(self.n_det, dtype=np.float64) - (self.n_det - 1) / 2.0)[None, :] * self.det_spacing
        st, ct = np.sin(th), np.cos(th)
        T = np.stack([-self.det_dist * st + u * ct, self.det_dist * ct + u * st], axis=-1)
        S = np.broadcast_to(np.stack([self.src_dist * st, -self.src_dist * ct], axis=-1), T.shape)
        return S, T - S


def ray_taps(n: int, S, v):
    """Joseph taps of the lines through S[r] with directions v[r] (arrays
    [R][2]) on an n x n image: (flat pixel index [2, R, n], weight [2, R, n])."""
    c = (n - 1) / 2.0
    S = np.asarray(S, dtype=np.float64).reshape(-1, 2)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 2)
    sx, sy, vx, vy = (a[:, None] for a in (S[:, 0], S[:, 1], v[:, 0], v[:, 1]))
    L = np.hypot(vx, vy)
    steps = np.arange(n, dtype=np.float64)[None, :]
    by_col = np.abs(vx) >= np.abs(vy)                   # [R, 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        frac_c = c - (sy + ((steps - c) - sx) * vy / vx)    # fractional row in column `step`
        frac_r = sx + ((c - steps) - sy) * vx / vy + c      # fractional column in row `step`
        w = np.where(by_col, L / np.abs(vx), L / np.abs(vy))
    frac = np.where(by_col, frac_c, frac_r)
    i0 = np.floor(frac)
    f = frac - i0
    other = np.stack([i0, i0 + 1.0])                    # the interpolated index
    march = np.broadcast_to(steps, other.shape)         # the marched index
    rows = np.where(by_col[None], other, march)
    cols = np.where(by_col[None], march, other)
    wts = np.stack([(1.0 - f) * w, f * w])
    ok = (rows >= 0) & (rows <= n - 1) & (cols >= 0) & (cols <= n - 1)
    idx = np.where(ok, rows * n + cols, 0).astype(np.int64)
    return idx, np.where(ok, wts, 0.0)


def line_taps(n: int, S, v):
    """Taps of one line: (flat pixel index [2, n], weight [2, n])."""
    idx, wts = ray_taps(n, np.asarray(S)[None], np.asarray(v)[None])
    return idx[:, 0], wts[:, 0]


def forward_project(img: np.ndarray, geom: FanGeometry) -> np.ndarray:
    """z = A img, [n_views][n_det]."""
    flat = np.asarray(img, dtype=np.float64).reshape(-1)
    S, v = geom.rays()
    out = np.zeros((geom.n_views, geom.n_det))
    for k in range(geom.n_views):
        idx, wts = ray_taps(geom.n, S[k], v[k])
        out[k] = (flat[idx] * wts).sum(axis=(0, 2))
    return out


def back_project(sino: np.ndarray, geom: FanGeometry) -> np.ndarray:
    """A^T sino, [n][n] (the same taps, scattered)."""
    sino = np.asarray(sino, dtype=np.float64).reshape(geom.n_views, geom.n_det)
    S, v = geom.rays()
    acc = np.zeros(geom.N)
    for k in range(geom.n_views):
        idx, wts = ray_taps(geom.n, S[k], v[k])
        acc += np.bincount(idx.reshape(-1), weights=(wts * sino[k][None, :, None]).reshape(-1), minlength=geom.N)
    return acc.reshape(geom.n, geom.n)


def dense_matrix(geom: FanGeometry) -> np.ndarray:
    """A entry by entry from the hat-function reading of the same definition:
    pixel (ix, iy) on a column-marched ray gets |v|/|v_x| max(0, 1 - |s - iy|)
    with s the ray's fractional row in column ix (rows: likewise)."""
    n, c = geom.n, geom.centre()
    S, v = geom.rays()
    A = np.zeros((geom.M, geom.N))
    for k in range(geom.n_views):
        for d in range(geom.n_det):
            (sx, sy), (vx, vy) = S[k, d], v[k, d]
            L = math.hypot(vx, vy)
            for iy in range(n):
                for ix in range(n):
                    if abs(vx) >= abs(vy):
                        s = c - (sy + ((ix - c) - sx) * vy / vx)
                        wgt = max(0.0, 1.0 - abs(s - iy)) * L / abs(vx)
                    else:
                        s = sx + ((c - iy) - sy) * vx / vy + c
                        wgt = max(0.0, 1.0 - abs(s - ix)) * L / abs(vy)
                    A[k * geom.n_det + d, iy * n + ix] = wgt
    return A


def project(x: np.ndarray, geom: FanGeometry) -> np.ndarray:
    """Phi~ x = A V^-1 x (Eq. precondAMP_op)."""
    return forward_project(_pre.v_inverse(x, geom), geom)


def backproject(s: np.ndarray, geom: FanGeometry) -> np.ndarray:
    """Phi~^T s = V^-1 A^T s."""
    return _pre.v_inverse(back_project(s, geom), geom)


def frobenius_sq(geom: FanGeometry, views=None) -> float:
    """||Phi~||_F^2 = sum over rays of ||V^-1 a_i||^2, one filtered ray image
    at a time (over the rays of the given views only, when views is set)."""
    S, v = geom.rays()
    tot = 0.0
    for k in (range(geom.n_views) if views is None else views):
        idx, wts = ray_taps(geom.n, S[k], v[k])
        for d in range(geom.n_det):
            a = np.bincount(idx[:, d].reshape(-1), weights=wts[:, d].reshape(-1), minlength=geom.N)
            tot += float(np.sum(_pre.v_inverse(a.reshape(geom.n, geom.n), geom) ** 2))
    return tot
