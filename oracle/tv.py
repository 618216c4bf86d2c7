"""Proximal TV denoiser (Section 6.3), solved by Chambolle's dual projection.

The paper's plain denoiser in Section 6.3 is the l2 proximal map of total
variation:

    D_lambda(r) = argmin_x 1/2 ||x - r||^2 + lambda TV(x),

with isotropic TV(x) = sum_ij |grad x|_ij.  This oracle solves it with
Chambolle's 2004 projection algorithm (J. Math. Imaging Vis. 20:89), a
published method:

* grad: forward differences with Neumann boundary (the last difference in
  each direction is zero); div = -grad^T;
* p <- (p + tau grad(div p - r/lambda)) / (1 + tau |grad(div p - r/lambda)|),
  tau = 1/8, starting from p = 0, for a fixed number K of iterations;
* x = r - lambda div p.

The paper gives no rule for lambda; the D-GAMP-CT driver uses
lambda = c_tv * sqrt(tau_r) so that the threshold scales with the effective
noise standard deviation of r (Eq. rGAMP).  K is fixed, not run to
convergence, so a second implementation with the same K computes the same map.
"""
from __future__ import annotations

import numpy as np

TAU = 0.125


def grad(u: np.ndarray):
    gx = np.zeros_like(u)
    gy = np.zeros_like(u)
    gx[:, :-1] = u[:, 1:] - u[:, :-1]
    gy[:-1, :] = u[1:, :] - u[:-1, :]
    return gx, gy


def div(px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Negative adjoint of :func:`grad`."""
    d = np.zeros_like(px)
    d[:, 0] += px[:, 0]
    d[:, 1:-1] += px[:, 1:-1] - px[:, :-2]
    d[:, -1] += -px[:, -2]
    d[0, :] += py[0, :]
    d[1:-1, :] += py[1:-1, :] - py[:-2, :]
    d[-1, :] += -py[-2, :]
    return d


def tv_prox(r: np.ndarray, lam: float, n_iter: int) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    if lam <= 0.0 or n_iter <= 0:
        return r.copy()
    px = np.zeros_like(r)
    py = np.zeros_like(r)
    for _ in range(n_iter):
        q = div(px, py) - r / lam
        gx, gy = grad(q)
        nrm = np.sqrt(gx * gx + gy * gy)
        den = 1.0 + TAU * nrm
        px = (px + TAU * gx) / den
        py = (py + TAU * gy) / den
    return r - lam * div(px, py)


def tv_value(x: np.ndarray) -> float:
    gx, gy = grad(x)
    return float(np.sum(np.sqrt(gx * gx + gy * gy)))
