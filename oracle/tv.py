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

:func:`tv_prox_metric` is the same prox in the norm of the preconditioned
space (Section 6.3's prox_{(V^T V)} TV); its reading and algorithm are stated
beside it.
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


# ------------------------------------------- prox_{(V^T V)} TV (Sec. 6.3) ----
# Section 4.3 lets the denoiser use the norm of the preconditioned space, and
# Section 6.3 compares the l2 prox-TV with the one in the (V^T V)^{-1} norm.
# Reading: the norm is the Mahalanobis distance whose covariance is
# Q = (V^T V)^{-1}, the covariance that white noise takes on through V^-1
# (Eq. r_input), so
#
#     D_lambda(r) = argmin_x 1/2 (x - r)^T Q^{-1} (x - r) + lambda TV(x).
#
# Q = I is the l2 prox above.  Writing lambda |grad x|_i as the largest
# lambda p_i . (grad x)_i over |p_i| <= 1 and minimising over x first gives
# x(p) = r + lambda Q div p and the dual problem
#
#     max_{|p_i| <= 1}  -lambda^2/2 <div p, Q div p> - lambda <r, div p>,
#
# whose gradient in p is lambda grad x(p).  It is solved by projected gradient
# ascent (Chambolle 2005, EMMCVPR; Beck and Teboulle 2009, IEEE TIP 18:2419,
# for the dual TV problem), here with Q inside x(p):
#
#     x_k = r + lambda Q div p_k,
#     p_{k+1} = Proj_{|p_i| <= 1}(p_k + theta/lambda grad x_k),
#
# from p_0 = 0 for a fixed number K of steps, returning x(p_K).  The step
# theta = 1 / (8 q_max), with ||grad||^2 <= 8 and ||Q|| <= q_max, is 1/L for
# the dual's gradient, so the dual objective never decreases.  Only Q is
# applied, never Q^{-1}, which the cropped realisation does not give as a
# filter.

def tv_prox_metric(r: np.ndarray, lam: float, n_iter: int, Q, q_max: float) -> np.ndarray:
    """argmin_x 1/2 (x-r)^T Q^{-1} (x-r) + lam TV(x) by n_iter dual steps.

    Q is a callable applying the covariance (symmetric positive definite,
    norm at most q_max) to an image."""
    r = np.asarray(r, dtype=np.float64)
    if lam <= 0.0 or n_iter <= 0:
        return r.copy()
    theta = 1.0 / (8.0 * q_max)
    px = np.zeros_like(r)
    py = np.zeros_like(r)
    for _ in range(n_iter):
        x = r + lam * Q(div(px, py))
        gx, gy = grad(x)
        px = px + (theta / lam) * gx
        py = py + (theta / lam) * gy
        nrm = np.maximum(np.sqrt(px * px + py * py), 1.0)
        px = px / nrm
        py = py / nrm
    return r + lam * Q(div(px, py))


def tv_prox_metric_dual(r: np.ndarray, lam: float, n_iter: int, Q, q_max: float):
    """The same iteration, returning (x, px, py, dual objective per step), for
    the certificate checks."""
    r = np.asarray(r, dtype=np.float64)
    theta = 1.0 / (8.0 * q_max)
    px = np.zeros_like(r)
    py = np.zeros_like(r)
    hist = []
    for _ in range(n_iter):
        d = div(px, py)
        qd = Q(d)
        hist.append(-0.5 * lam * lam * float(np.sum(d * qd)) - lam * float(np.sum(r * d)))
        gx, gy = grad(r + lam * qd)
        px = px + (theta / lam) * gx
        py = py + (theta / lam) * gy
        nrm = np.maximum(np.sqrt(px * px + py * py), 1.0)
        px = px / nrm
        py = py / nrm
    return r + lam * Q(div(px, py)), px, py, hist
