"""Discretisation conventions (Section 2.1, Eqs. paramdiscrete and linCT).

The paper fixes a sqrt(N) x sqrt(N) pixel basis and a system matrix A of
size (N_dec * N_theta) x N.  It leaves the coordinates open; this oracle (and
the CUDA library, independently) reads them as follows:

* pixel (ix, iy) of an n x n image has centre X = ix - (n-1)/2,
  Y = (n-1)/2 - iy and unit size; arrays are indexed ``img[iy, ix]``;
* view k sits at theta_k = k*pi/n_views (evenly over 180 degrees, endpoint
  excluded) unless explicit angles are supplied;
* detector bin d sits at u_d = d - (n_det-1)/2 with unit spacing;
* ray (theta, u) is the line X cos(theta) + Y sin(theta) = u;
* the detector-axis FFT length P is the smallest power of two >= 2*n_det.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Geometry:
    n: int
    n_views: int
    n_det: int
    angles: tuple | None = None

    def thetas(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, dtype=np.float64)
        return np.arange(self.n_views, dtype=np.float64) * (math.pi / self.n_views)

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

    def det_offsets(self) -> np.ndarray:
        return np.arange(self.n_det, dtype=np.float64) - (self.n_det - 1) / 2.0

    def centre(self) -> float:
        return (self.n - 1) / 2.0
