"""Seeded synthetic inputs for the D-GAMP-CT hot path.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds none of the reconstruction method's arithmetic: no projector, no
preconditioner, no GAMP step.  It draws random ellipse/rectangle phantoms,
rasterises them, evaluates their *analytic* parallel-beam line integrals (the
continuous Radon transform of each shape, a textbook closed form), and draws
Poisson transmission counts from those integrals.

Conventions (the paper leaves them open; Section 2.1 only fixes a sqrt(N) x
sqrt(N) pixel grid and the ray model of Eq. (BeerLaw)):

* image array ``img[iy, ix]`` with ``n`` rows and columns, pixel size 1;
  pixel centre ``X = ix - (n-1)/2``, ``Y = (n-1)/2 - iy`` (row 0 at the top);
* view ``k`` at angle ``theta_k = k*pi/n_views`` unless angles are given;
* detector bin ``d`` at offset ``u_d = d - (n_det-1)/2``;
* ray ``(theta, u)`` is the line ``X cos(theta) + Y sin(theta) = u``.

The measurement model is Eq. (Poisson_CT) of Section 2.1 with no background
term: ``y_i ~ Poisson(I0 * exp(-z_i))`` where ``z_i`` is the line integral.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Ellipse", "Rect", "Phantom", "random_phantom", "rasterise",
    "analytic_sinogram", "poisson_counts", "view_angles", "make_case",
    "CASES", "FAN_CASES", "fan_lines", "analytic_fan_sinogram", "fan_view_angles",
]


@dataclasses.dataclass(frozen=True)
class Ellipse:
    x0: float          # centre, pixel units (X axis)
    y0: float          # centre, pixel units (Y axis, up)
    a: float           # semi-axis along direction phi
    b: float           # semi-axis perpendicular to phi
    phi: float         # rotation, radians
    rho: float         # attenuation per pixel length


@dataclasses.dataclass(frozen=True)
class Rect:
    x0: float
    y0: float
    hx: float          # half side along direction phi
    hy: float          # half side perpendicular to phi
    phi: float
    rho: float


@dataclasses.dataclass(frozen=True)
class Phantom:
    """Additive ellipses, then an optional rectangle painted on top.

    Painting replaces whatever lies under the rectangle by ``rect.rho``; the
    line integral stays analytic because every shape's chord along a line is
    one interval, so the covered part of each ellipse chord is an interval
    intersection.
    """
    ellipses: tuple
    rect: Rect | None = None


def view_angles(n_views: int) -> np.ndarray:
    """theta_k = k*pi/n_views, k = 0..n_views-1 (endpoint excluded)."""
    return np.arange(n_views, dtype=np.float64) * (math.pi / n_views)


def random_phantom(n: int, n_ellipses: int, seed: int, rho_max: float = 0.02,
                   with_rect: bool = False, rect_rho: float = 0.05) -> Phantom:
    """Draw the ellipse phantom recipe used by every workload.

    Centres uniform in a disk of radius 0.6*n/2, semi-axes U(0.05, 0.4)*n/2,
    rotation U(0, pi), density U(0, rho_max).  The optional rectangle has
    half sides U(0.05, 0.2)*n/2, rotation U(0, pi), a centre uniform in a disk
    of radius 0.4*n/2 and density ``rect_rho``; it is painted last.
    """
    rng = np.random.default_rng(seed)
    half = n / 2.0
    ells = []
    for _ in range(n_ellipses):
        rad = 0.6 * half * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        a, b = rng.uniform(0.05, 0.4, size=2) * half
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, rho_max)
        ells.append(Ellipse(rad * math.cos(ang), rad * math.sin(ang),
                            float(a), float(b), float(phi), float(rho)))
    rect = None
    if with_rect:
        rad = 0.4 * half * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        hx, hy = rng.uniform(0.05, 0.2, size=2) * half
        phi = rng.uniform(0.0, math.pi)
        rect = Rect(rad * math.cos(ang), rad * math.sin(ang), float(hx),
                    float(hy), float(phi), float(rect_rho))
    return Phantom(tuple(ells), rect)


# ---------------------------------------------------------------- raster ----
def _inside_ellipse(e: Ellipse, X, Y):
    c, s = math.cos(e.phi), math.sin(e.phi)
    dx, dy = X - e.x0, Y - e.y0
    xr = c * dx + s * dy
    yr = -s * dx + c * dy
    return (xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0


def _inside_rect(r: Rect, X, Y):
    c, s = math.cos(r.phi), math.sin(r.phi)
    dx, dy = X - r.x0, Y - r.y0
    xr = c * dx + s * dy
    yr = -s * dx + c * dy
    return (np.abs(xr) <= r.hx) & (np.abs(yr) <= r.hy)


def rasterise(ph: Phantom, n: int, supersample: int = 4) -> np.ndarray:
    """Pixel averages of the phantom by ``supersample``^2 point samples."""
    c = (n - 1) / 2.0
    ss = supersample
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    img = np.zeros((n, n), dtype=np.float64)
    ix = np.arange(n, dtype=np.float64)
    for oy in offs:
        for ox in offs:
            X = (ix[None, :] - c) + ox
            Y = (c - ix[:, None]) + oy
            X = np.broadcast_to(X, (n, n))
            Y = np.broadcast_to(Y, (n, n))
            val = np.zeros((n, n))
            for e in ph.ellipses:
                val += e.rho * _inside_ellipse(e, X, Y)
            if ph.rect is not None:
                m = _inside_rect(ph.rect, X, Y)
                val = np.where(m, ph.rect.rho, val)
            img += val
    return img / (ss * ss)


# ------------------------------------------------------------- analytic ----
def _line_frame(theta, u):
    """Point on the line closest to the origin and unit direction."""
    ct, st = np.cos(theta), np.sin(theta)
    return u * ct, u * st, -st, ct


def _ellipse_interval(e: Ellipse, theta, u):
    """Chord [t1, t2] of line (theta, u) through the ellipse (t2<t1 = empty)."""
    px, py, dx, dy = _line_frame(theta, u)
    c, s = math.cos(e.phi), math.sin(e.phi)
    qx, qy = px - e.x0, py - e.y0
    qxr, qyr = (c * qx + s * qy) / e.a, (-s * qx + c * qy) / e.b
    dxr, dyr = (c * dx + s * dy) / e.a, (-s * dx + c * dy) / e.b
    A = dxr * dxr + dyr * dyr
    B = qxr * dxr + qyr * dyr
    C = qxr * qxr + qyr * qyr - 1.0
    disc = B * B - A * C
    ok = disc > 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t1 = np.where(ok, (-B - sq) / A, 0.0)
    t2 = np.where(ok, (-B + sq) / A, -1.0)
    return t1, t2


def _rect_interval(r: Rect, theta, u):
    px, py, dx, dy = _line_frame(theta, u)
    c, s = math.cos(r.phi), math.sin(r.phi)
    qx, qy = px - r.x0, py - r.y0
    q = [c * qx + s * qy, -s * qx + c * qy]
    d = [c * dx + s * dy, -s * dx + c * dy]
    h = [r.hx, r.hy]
    lo = np.full(np.broadcast(theta, u).shape, -np.inf)
    hi = np.full_like(lo, np.inf)
    for k in range(2):
        dk = np.broadcast_to(d[k], lo.shape)
        qk = np.broadcast_to(q[k], lo.shape)
        par = np.abs(dk) < 1e-15
        inside = np.abs(qk) <= h[k]
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (-h[k] - qk) / dk
            tb = (h[k] - qk) / dk
        lo = np.where(par, np.where(inside, lo, np.inf), np.maximum(lo, np.minimum(ta, tb)))
        hi = np.where(par, np.where(inside, hi, -np.inf), np.minimum(hi, np.maximum(ta, tb)))
    return lo, hi


def analytic_sinogram(ph: Phantom, angles: np.ndarray, n_det: int) -> np.ndarray:
    """Exact line integrals ``z[view, bin]`` of the phantom (fp64)."""
    u = np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0
    th = np.asarray(angles, dtype=np.float64)[:, None]
    return _line_integrals(ph, th, u[None, :])


def _line_integrals(ph: Phantom, th, uu) -> np.ndarray:
    """Line integrals along the lines (th, uu) (broadcast together)."""
    th, uu = np.broadcast_arrays(np.asarray(th, dtype=np.float64), np.asarray(uu, dtype=np.float64))
    z = np.zeros(th.shape)
    if ph.rect is not None:
        r1, r2 = _rect_interval(ph.rect, th, uu)
    for e in ph.ellipses:
        t1, t2 = _ellipse_interval(e, th, uu)
        chord = np.maximum(t2 - t1, 0.0)
        if ph.rect is not None:
            cov = np.maximum(np.minimum(t2, r2) - np.maximum(t1, r1), 0.0)
            chord = chord - np.where(t2 > t1, cov, 0.0)
        z += e.rho * chord
    if ph.rect is not None:
        z += ph.rect.rho * np.maximum(r2 - r1, 0.0)
    return z


def fan_lines(angles: np.ndarray, n_det: int, src_dist: float, det_dist: float,
              det_spacing: float):
    """Each fan-beam ray as a line (theta', u') of the parallel convention.

    Flat-detector fan beam: at view angle theta the source sits at
    src_dist (sin theta, -cos theta), the detector centre at
    det_dist (-sin theta, cos theta), and bin d at the detector centre plus
    u_d (cos theta, sin theta), u_d = (d - (n_det-1)/2) det_spacing.  The
    central ray therefore runs along (-sin theta, cos theta), the direction of
    the parallel-beam ray (theta, 0).  Returns theta', u' of shape
    [n_views][n_det] with X cos theta' + Y sin theta' = u' the ray's line."""
    th = np.asarray(angles, dtype=np.float64)[:, None]
    u = (np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0)[None, :] * det_spacing
    sx, sy = src_dist * np.sin(th), -src_dist * np.cos(th)
    tx = -det_dist * np.sin(th) + u * np.cos(th)
    ty = det_dist * np.cos(th) + u * np.sin(th)
    dx, dy = tx - sx, ty - sy
    nrm = np.hypot(dx, dy)
    dx, dy = dx / nrm, dy / nrm
    # direction (-sin theta', cos theta') = (dx, dy)
    thp = np.arctan2(-dx, dy)
    up = sx * np.cos(thp) + sy * np.sin(thp)
    return thp, up


def analytic_fan_sinogram(ph: Phantom, angles: np.ndarray, n_det: int, src_dist: float,
                          det_dist: float, det_spacing: float) -> np.ndarray:
    """Exact line integrals of the phantom along the fan-beam rays (fp64)."""
    thp, up = fan_lines(angles, n_det, src_dist, det_dist, det_spacing)
    return _line_integrals(ph, thp, up)


def poisson_counts(z: np.ndarray, I0: float, seed: int) -> np.ndarray:
    """y ~ Poisson(I0 * exp(-z)), float32 (integer valued, exact below 2^24)."""
    rng = np.random.default_rng(seed)
    lam = I0 * np.exp(-np.asarray(z, dtype=np.float64))
    return rng.poisson(lam).astype(np.float32)


# ---------------------------------------------------------------- cases ----
#: name -> (n, n_views, n_det, n_ellipses, rho_max, with_rect, I0, iters)
CASES = {
    # 64x64, 5 ellipses, 30 views over 180 deg, 95 bins, I0 = 1e4, 20 iterations
    "ellipse64_v30": (64, 30, 95, 5, 0.02, False, 1e4, 20),
    # 512x512, 10 ellipses + rectangle object, 64 views, 729 bins, I0 = 1e5, 30 iterations
    "ellipse512_v64": (512, 64, 729, 10, 0.02, True, 1e5, 30),
}


#: fan-beam workloads (flat detector, views evenly over 360 degrees, see
#: fan_lines): name -> (n, n_views, n_det, n_ellipses, rho_max, with_rect,
#: I0, iters, src_dist, det_dist, det_spacing), distances in pixels
FAN_CASES = {
    # 64x64, 5 ellipses, 30 views, 96 bins of 1.95 px, source 112 px and
    # detector 92 px from the centre (field of view radius 46 px)
    "fan64_v30": (64, 30, 96, 5, 0.02, False, 1e4, 20, 112.0, 92.0, 1.95),
    # 512x512, 10 ellipses + rectangle, 102 views (a tenth of 1024), 736 bins
    # of 1.95 px, source 900 px and detector 740 px from the centre: the
    # proportions of a clinical fan-beam scanner at 0.66 mm pixels
    "fan512_v102": (512, 102, 736, 10, 0.02, True, 1e5, 30, 900.0, 740.0, 1.95),
}


def fan_view_angles(n_views: int) -> np.ndarray:
    """theta_k = 2 pi k / n_views (a full rotation)."""
    return np.arange(n_views, dtype=np.float64) * (2.0 * math.pi / n_views)


def make_case(name: str, seed: int = 1000):
    """Phantom, counts and geometry for one named workload.

    Returns a dict with ``mu`` (rasterised phantom, fp64 [n][n]), ``z``
    (analytic sinogram, fp64 [n_views][n_det]), ``y`` (float32 counts),
    ``I0``, ``n``, ``n_views``, ``n_det``, ``iters``; a fan-beam workload
    also has ``angles`` and ``fan`` (src_dist, det_dist, det_spacing).
    """
    if name in FAN_CASES:
        n, nv, nd, ne, rmax, rect, I0, iters, sd, dd, ds = FAN_CASES[name]
        ph = random_phantom(n, ne, seed, rho_max=rmax, with_rect=rect)
        ang = fan_view_angles(nv)
        z = analytic_fan_sinogram(ph, ang, nd, sd, dd, ds)
        y = poisson_counts(z, I0, seed + 7)
        return dict(name=name, phantom=ph, mu=rasterise(ph, n), z=z, y=y, I0=I0, n=n, n_views=nv,
                    n_det=nd, iters=iters, seed=seed, angles=ang,
                    fan=dict(src_dist=sd, det_dist=dd, det_spacing=ds))
    n, nv, nd, ne, rmax, rect, I0, iters = CASES[name]
    ph = random_phantom(n, ne, seed, rho_max=rmax, with_rect=rect)
    ang = view_angles(nv)
    z = analytic_sinogram(ph, ang, nd)
    y = poisson_counts(z, I0, seed + 7)
    return dict(name=name, phantom=ph, mu=rasterise(ph, n), z=z, y=y, I0=I0,
                n=n, n_views=nv, n_det=nd, iters=iters, seed=seed)


# Mixed batch of independent slices: image side, view count, detector bins
# ceil(1.42 n) and dose drawn per slice (the paper reconstructs slice by
# slice; a batch stands in for a volume or a queue of scans of varying size).
BATCHES = {
    # 64 slices, n in {256, 384, 512}, views in {32, 48, 64, 96, 128},
    # log10 I0 ~ U(4, 6), 10 ellipses + rectangle object each, 30 iterations
    "mixed64": dict(count=64, sides=(256, 384, 512), views=(32, 48, 64, 96, 128), log10_I0=(4.0, 6.0),
                    n_ellipses=10, with_rect=True, iters=30),
    # 128 slices of 1024 x 1024, 90 views, 1449 bins, I0 = 1e5, 10 ellipses
    # each.  Densities are halved (rho_max 0.01 per pixel): the same objects
    # as the 512 x 512 workloads on a grid of half the pixel size, so that the
    # line integrals (and the photon counts) span the same range.
    "large128": dict(count=128, sides=(1024,), views=(90,), bins=1449, log10_I0=(5.0, 5.0),
                     n_ellipses=10, with_rect=False, iters=30, rho_max=0.01),
}


def make_batch(name: str = "mixed64", seed: int = 3000, with_mu: bool = False, count: int | None = None):
    """Slices of a named batch: a list of dicts like :func:`make_case` (``mu``
    only with ``with_mu``; rasterising is the slow part).  Slice k's phantom
    uses seed ``seed + 1 + k`` and its counts ``seed + 1 + k + 7``."""
    spec = BATCHES[name]
    k_total = spec["count"] if count is None else int(count)
    rng = np.random.default_rng(seed)
    out = []
    for k in range(k_total):
        n = int(rng.choice(spec["sides"]))
        nv = int(rng.choice(spec["views"]))
        nd = int(spec["bins"]) if "bins" in spec else int(math.ceil(1.42 * n))
        I0 = float(10.0 ** rng.uniform(*spec["log10_I0"]))
        ph = random_phantom(n, spec["n_ellipses"], seed + 1 + k, rho_max=spec.get("rho_max", 0.02),
                            with_rect=spec["with_rect"])
        z = analytic_sinogram(ph, view_angles(nv), nd)
        y = poisson_counts(z, I0, seed + 1 + k + 7)
        out.append(dict(name=f"{name}[{k}]", phantom=ph, mu=rasterise(ph, n) if with_mu else None, z=z, y=y,
                        I0=I0, n=n, n_views=nv, n_det=nd, iters=spec["iters"], seed=seed + 1 + k))
    return out
