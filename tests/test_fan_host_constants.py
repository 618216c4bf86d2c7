"""The fan-beam ray constants the library builds on the host
(dgamp_ct_fan_ray_constants, no device needed) against the oracle's Joseph
taps: for every ray and step, the same marching axis, the same left tap,
the fraction and the path length per step to FP32 accuracy."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import fanbeam

GEOMS = [
    (24, 7, 37, 40.0, 30.0, 1.3, None),
    (64, 30, 96, 112.0, 92.0, 1.95, None),
    (20, 5, 41, 1e7, 1e7, 2.0, None),
    (18, 8, 30, 35.0, 28.0, 1.7, tuple(np.linspace(0, math.pi, 8, endpoint=False))),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04661_gb300 import build, binding
    build.build()
    return C.CDLL(binding.LIB_PATH), binding


@pytest.mark.parametrize("n,nv,nd,sd,dd,du,ang", GEOMS)
def test_host_constants_give_the_oracle_taps(lib, n, nv, nd, sd, dd, du, ang):
    L, binding = lib
    g = binding.Geometry(n, nv, nd, None)
    keep = None
    if ang is not None:
        keep = np.ascontiguousarray(ang, dtype=np.float64)
        g.angles = keep.ctypes.data_as(C.POINTER(C.c_double))
    fg = binding.FanGeometry(g, sd, dd, du)
    R = nv * nd
    p0, ps = np.zeros(R, np.int64), np.zeros(R, np.int64)
    w, col = np.zeros(R, np.float32), np.zeros(R, np.int32)
    f = L.dgamp_ct_fan_ray_constants
    f.restype = C.c_int
    args = [a.ctypes.data_as(C.c_void_p) for a in (p0, ps, w, col)]
    assert f(C.byref(fg), *args) == 0
    geom = fanbeam.FanGeometry(n, nv, nd, sd, dd, du, angles=ang)
    S, v = geom.rays()
    steps = np.arange(n, dtype=np.int64)
    for k in range(nv):
        idx, wts = fanbeam.ray_taps(n, S[k], v[k])          # [2, nd, n]
        for d in range(nd):
            i = k * nd + d
            by_col = abs(v[k, d, 0]) >= abs(v[k, d, 1])
            assert col[i] == int(by_col)
            pos = p0[i] + steps * ps[i]
            i0 = pos >> 32
            frac = (pos & 0xFFFFFFFF) / 2.0 ** 32
            wo = math.hypot(*v[k, d]) / (abs(v[k, d, 0]) if by_col else abs(v[k, d, 1]))
            assert w[i] == pytest.approx(wo, rel=1e-6)
            # the oracle's interpolated index of tap 0 at every step whose
            # left tap lies inside the image
            other = idx[0, d] // n if by_col else idx[0, d] % n
            inside = wts[0, d] > 0
            assert np.array_equal(i0[inside], other[inside])
            assert np.allclose(frac[inside], 1.0 - wts[0, d][inside] / wo, atol=1e-6)


def test_host_constants_reject_bad_arguments(lib):
    L, binding = lib
    f = L.dgamp_ct_fan_ray_constants
    f.restype = C.c_int
    buf = np.zeros(16, np.int64)
    p = buf.ctypes.data_as(C.c_void_p)
    assert f(None, p, p, p, p) == -1
    fg = binding.FanGeometry(binding.Geometry(8, 2, 4, None), 100.0, 100.0, 0.0)
    assert f(C.byref(fg), p, p, p, p) == -1
