"""CPU emulations of the index logic of two GPU paths, against the oracle.

These restate, in numpy, the integer and index arithmetic of kernels that are
checked on the GPU by their parity tests; here they pin the design on the CPU:

* the fan-beam gather (fanbeam.cu, k_fan_backproject): candidate rays found
  by projecting the segments (X, Y-1)-(X, Y+1) and (X-1, Y)-(X+1, Y) through
  the source in FP32, widened by one bin, and tested with the projector's
  32.32 positions (taken from the library's own host constants,
  dgamp_ct_fan_ray_constants), must find every tap of A, so the gather is
  A's exact transpose;
* the metric prox-TV launch sequence (tv_metric.cu): a dual step from p = 0,
  then per step the three FFT passes with the MC pair packed as the real and
  imaginary parts of one complex image, then the dual step, must give the
  oracle's tv_prox_metric for both images;
* the banded projector's work split (joseph.cu, project_band_chunks and
  k_project_band): the chunks of each orientation's (view, bin) list cover
  every ray once, and no chunk spans more views than the block's shared
  table holds (8), for every occupancy the plan may see.
"""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import fanbeam, precond, tv

f32 = np.float32


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04661_gb300 import build, binding
    build.build()
    return C.CDLL(binding.LIB_PATH), binding


def _constants(lib, n, nv, nd, sd, dd, du):
    L, binding = lib
    fg = binding.FanGeometry(binding.Geometry(n, nv, nd, None), sd, dd, du)
    R = nv * nd
    p0, ps = np.zeros(R, np.int64), np.zeros(R, np.int64)
    w, col = np.zeros(R, np.float32), np.zeros(R, np.int32)
    L.dgamp_ct_fan_ray_constants.restype = C.c_int
    assert L.dgamp_ct_fan_ray_constants(C.byref(fg), *[a.ctypes.data_as(C.c_void_p) for a in (p0, ps, w, col)]) == 0
    return p0, ps, w, col


def _tap(pos):
    return pos >> 32, ((pos & 0xFFFFFFFF) >> 9) / 2.0 ** 23


@pytest.mark.parametrize("n,nv,nd,sd,dd,du", [(24, 7, 37, 40.0, 30.0, 1.3), (16, 9, 33, 13.4, 13.4, 0.9),
                                                (20, 5, 41, 1e7, 1e7, 2.0)])
def test_fan_gather_finds_every_tap(lib, n, nv, nd, sd, dd, du):
    p0, ps, w, col = _constants(lib, n, nv, nd, sd, dd, du)
    g = fanbeam.FanGeometry(n, nv, nd, sd, dd, du)
    c = 0.5 * (n - 1)
    # A from the projector's integer taps
    A = np.zeros((nv * nd, n * n))
    for i in range(nv * nd):
        for s in range(n):
            i0, f = _tap(int(p0[i]) + s * int(ps[i]))
            for q, wt in ((i0, 1 - f), (i0 + 1, f)):
                if 0 <= q < n:
                    A[i, q * n + s if col[i] else s * n + q] += wt * float(w[i])
    assert np.abs(A - fanbeam.dense_matrix(g)).max() < 1e-5 * np.abs(A).max()
    # the gather's candidate search, in FP32 as on the GPU
    th = g.thetas()
    found = np.zeros_like(A, dtype=bool)
    for k in range(nv):
        st, ct = math.sin(th[k]), math.cos(th[k])
        eux, euy, ecx, ecy = f32(ct), f32(st), f32(-st), f32(ct)

        def binf(x, y):
            x, y = f32(x), f32(y)
            along = x * ecx + (y * ecy + f32(sd))
            across = x * eux + y * euy
            return f32(sd + dd) * across / (along * f32(du)) + f32(0.5 * (nd - 1))

        def cands(x1, y1, x2, y2):
            b1, b2 = binf(x1, y1), binf(x2, y2)
            bl = min(max(min(b1, b2), -2.0), nd + 1.0)
            bh = max(min(max(b1, b2), nd + 1.0), -2.0)
            return max(0, math.floor(bl) - 1), min(nd - 1, math.ceil(bh) + 1)

        for iy in range(n):
            for ix in range(n):
                X, Y = ix - c, c - iy
                for (lo, hi), want_col in ((cands(X, Y - 1, X, Y + 1), 1), (cands(X - 1, Y, X + 1, Y), 0)):
                    for d in range(lo, hi + 1):
                        i = k * nd + d
                        if col[i] != want_col:
                            continue
                        i0, _ = _tap(int(p0[i]) + (ix if want_col else iy) * int(ps[i]))
                        k_across = iy if want_col else ix
                        if i0 in (k_across, k_across - 1):
                            found[i, iy * n + ix] = True
    assert np.all(found[A != 0])                  # no tap of A is missed (extra zero-weight hits are harmless)
    assert found.sum() >= (A != 0).sum() > 0


@pytest.mark.parametrize("n,K", [(7, 1), (9, 3), (12, 5)])
def test_metric_tv_launch_sequence(n, K):
    from oracle.geometry import Geometry
    g = Geometry(n, 5, 2 * n + 1)
    m = precond.image_pad(g)
    r = np.random.default_rng(n).standard_normal((2, n, n))
    lam = 0.3
    fy = np.fft.fftfreq(m)
    f0 = 1.0 / (2 * g.P)
    theta = f32(1.0 / (8.0 * max(math.sqrt(0.5), f0)))
    p = np.zeros((2, n, n, 2))
    X = np.zeros((2, n, n))
    Cs = np.zeros((n, m), complex)
    for i in range(4 * K):
        phase = 3 if i == 0 else (i - 1) % 4
        if phase == 3:
            src = r if i == 0 else X
            for im in range(2):
                gx = np.zeros((n, n))
                gy = np.zeros((n, n))
                gx[:, :-1] = src[im][:, 1:] - src[im][:, :-1]
                gy[:-1, :] = src[im][1:, :] - src[im][:-1, :]
                q = np.zeros((n, n, 2)) if i == 0 else p[im].copy()
                q[..., 0] += theta / lam * gx
                q[..., 1] += theta / lam * gy
                p[im] = q / np.maximum(np.hypot(q[..., 0], q[..., 1]), 1.0)[..., None]
        elif phase == 0:
            d = np.zeros((n, m), complex)
            for im in range(2):
                px, py = p[im][..., 0], p[im][..., 1]
                dv = px.copy() + py
                dv[:, 1:] -= px[:, :-1]
                dv[1:, :] -= py[:-1, :]
                d[:, :n] += dv if im == 0 else 1j * dv
            Cs = np.fft.fft(d, axis=1)
        elif phase == 1:
            col = np.zeros((m, m), complex)
            col[:n] = Cs
            gain = np.maximum(np.hypot(fy[:, None], fy[None, :]), f0)
            Cs = (np.fft.ifft(np.fft.fft(col, axis=0) * gain, axis=0) * m)[:n]
        else:
            row = np.fft.ifft(Cs, axis=1) * m
            X[0] = r[0] + lam / (m * m) * row[:, :n].real
            X[1] = r[1] + lam / (m * m) * row[:, :n].imag
    for im in range(2):
        ref = tv.tv_prox_metric(r[im], lam, K, lambda u: precond.vtv_inverse(u, g), precond.vtv_inverse_norm_bound(g))
        assert np.abs(X[im] - ref).max() < 1e-6


# ------------------------------------------------ banded projector split ----
BAND_MAX_VIEWS = 8          # kBandMaxViews: the block's shared view table


def _band_chunks(total, n0, nv, nd):
    """Chunks per band of each orientation, as project_band_chunks picks them."""
    def fit(want, nvo):
        if nvo == 0:
            return 0
        want = max(want, (nvo + BAND_MAX_VIEWS - 2) // (BAND_MAX_VIEWS - 1))
        return min(max(want, 1), nvo * nd)
    c0 = fit(int(math.floor(total * n0 / nv + 0.5)), n0)
    return c0, fit(total - c0, nv - n0)


@pytest.mark.parametrize("n,nv,nd", [(512, 64, 729), (37, 13, 55), (96, 37, 140), (16, 4096, 24), (300, 5, 1100),
                                     (1024, 90, 1449), (2, 3, 3), (16, 2, 4096), (50, 1, 73)])
@pytest.mark.parametrize("band", [16, 32])
def test_band_split_covers_every_ray_once(n, nv, nd, band):
    nb = (n + band - 1) // band
    for n0 in sorted({0, nv // 2, nv - (nv // 3), nv}):
        for bps in (1, 2, 3):
            for waves in (1, 2):
                total = max(2, waves * bps * 152 // nb)
                c0, c1 = _band_chunks(total, n0, nv, nd)
                assert c0 + c1 <= 65535
                for nvo, C in ((n0, c0), (nv - n0, c1)):
                    tot = nvo * nd
                    assert (C == 0) == (nvo == 0)
                    covered = 0
                    for ci in range(C):
                        lo, hi = tot * ci // C, tot * (ci + 1) // C
                        assert lo == covered and hi > lo
                        covered = hi
                        assert (hi - 1) // nd - lo // nd + 1 <= BAND_MAX_VIEWS
                    assert covered == tot
