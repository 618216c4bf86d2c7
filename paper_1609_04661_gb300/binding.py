"""Thin ctypes binding of libdgampct.so (include/dgamp_ct.h).

Argument marshalling only: every call forwards device pointers of torch
tensors and the current CUDA stream to the C ABI; all arithmetic runs in the
library's CUDA kernels.  Importing this module does not touch the GPU; a
missing library raises immediately (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgampct.so")

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED_GEOMETRY", -3: "OOM", -4: "CUDA", -5: "TIMEOUT",
          -6: "NONFINITE"}

#: every symbol include/dgamp_ct.h declares
EXPORTS = (
    "dgamp_ct_default_options", "dgamp_ct_plan", "dgamp_ct_plan_destroy", "dgamp_ct_set_options",
    "dgamp_ct_plan_info", "dgamp_ct_project", "dgamp_ct_backproject", "dgamp_ct_filter",
    "dgamp_ct_output_step", "dgamp_ct_denoise_tv", "dgamp_ct_denoise_div", "dgamp_ct_probe",
    "dgamp_ct_precond_image", "dgamp_ct_solve", "dgamp_ct_solve_host", "dgamp_ct_solve_launches",
    "dgamp_ct_strerror", "dgamp_ct_last_cuda_error", "dgamp_ct_profile_iteration",
    "dgamp_ct_output_step_noalloc", "dgamp_ct_get_tuning", "dgamp_ct_set_tuning",
    "dgamp_ct_cnn_create", "dgamp_ct_cnn_destroy", "dgamp_ct_cnn_num_params", "dgamp_ct_cnn_set_params",
    "dgamp_ct_cnn_get_params", "dgamp_ct_cnn_denoise", "dgamp_ct_cnn_denoise_jvp", "dgamp_ct_cnn_gradients", "dgamp_ct_cnn_train_step",
    "dgamp_ct_cnn_test_timeout", "dgamp_ct_plan_set_cnn", "dgamp_ct_solve_trace", "dgamp_ct_solve_batched", "dgamp_ct_schedule_lpt",
    "dgamp_ct_plan_fan", "dgamp_ct_fan_ray_constants", "dgamp_ct_measure_fp32_peak", "dgamp_ct_measure_fp32x2_peak",
    "dgamp_ct_batch_create", "dgamp_ct_batch_destroy", "dgamp_ct_batch_solve", "dgamp_ct_batch_launches",
)


class DgampError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {ERRORS.get(code, code)}"
        if code == -4 and _lib is not None:
            msg += f" (cudaError {_lib.dgamp_ct_last_cuda_error()})"
        super().__init__(msg)


class Geometry(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_views", C.c_int32), ("n_det", C.c_int32),
                ("angles", C.POINTER(C.c_double))]


class FanGeometry(C.Structure):
    """dgamp_ct_fan_geometry (flat-detector fan beam)."""
    _fields_ = [("base", Geometry), ("src_dist", C.c_double), ("det_dist", C.c_double),
                ("det_spacing", C.c_double)]


class Tuning(C.Structure):
    """dgamp_ct_tuning."""
    _fields_ = [("filter_mode", C.c_int32), ("tv_kb", C.c_int32), ("tv_rows", C.c_int32),
                ("sino_fused", C.c_int32), ("bp_mode", C.c_int32), ("pj_seg", C.c_int32),
                ("tv_vrows", C.c_int32), ("pj_band", C.c_int32), ("pj_waves", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("denoiser", C.c_int32), ("k_tv", C.c_int32), ("c_tv", C.c_double),
                ("eps_rel", C.c_double), ("seed", C.c_uint64), ("slice_id", C.c_int32),
                ("onsager", C.c_int32), ("damp_x", C.c_double), ("damp_s", C.c_double),
                ("tau_x_floor", C.c_double), ("use_graph", C.c_int32), ("cnn_scale", C.c_int32),
                ("tau_x0", C.c_double), ("truncate_z", C.c_int32), ("storage", C.c_int32),
                ("output_moments", C.c_int32), ("tv_metric", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("tau_x", C.POINTER(C.c_double)), ("tau_p", C.POINTER(C.c_double)),
                ("tau_s", C.POINTER(C.c_double)), ("tau_r", C.POINTER(C.c_double)),
                ("div", C.POINTER(C.c_double)), ("iters_done", C.c_int32),
                ("newton_capped", C.c_int32), ("tau_x_floored", C.c_int32),
                ("risk_plain", C.POINTER(C.c_double)), ("risk_learned", C.POINTER(C.c_double)),
                ("kept_learned", C.POINTER(C.c_int32)), ("learned_kept", C.c_int32)]


_STAT_ARRAYS = ("tau_x", "tau_p", "tau_s", "tau_r", "div")


def _new_stats(iters: int):
    """A Stats record with host arrays for every per-iteration field."""
    arrays = {k: np.zeros(iters) for k in _STAT_ARRAYS + ("risk_plain", "risk_learned")}
    p = {k: a.ctypes.data_as(C.POINTER(C.c_double)) for k, a in arrays.items()}
    arrays["kept_learned"] = np.zeros(iters, dtype=np.int32)
    kept = arrays["kept_learned"].ctypes.data_as(C.POINTER(C.c_int32))
    st = Stats(*[p[k] for k in _STAT_ARRAYS], 0, 0, 0, p["risk_plain"], p["risk_learned"], kept, 0)
    return st, arrays


def _stats_dict(st, arrays):
    arrays.update(iters_done=st.iters_done, newton_capped=st.newton_capped, tau_x_floored=st.tau_x_floored,
                  learned_kept=st.learned_kept)
    return arrays


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1609_04661_gb300.build` "
                          "(the CUDA library is required; there is no CPU path)")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "dgamp_ct_default_options": (C.c_int, [C.POINTER(Options)]),
        "dgamp_ct_plan": (C.c_int, [C.POINTER(Geometry), C.POINTER(Options), C.POINTER(vp)]),
        "dgamp_ct_plan_destroy": (None, [vp]),
        "dgamp_ct_plan_fan": (C.c_int, [C.POINTER(FanGeometry), C.POINTER(Options), C.POINTER(vp)]),
        "dgamp_ct_fan_ray_constants": (C.c_int, [C.POINTER(FanGeometry), vp, vp, vp, vp]),
        "dgamp_ct_set_options": (C.c_int, [vp, C.POINTER(Options)]),
        "dgamp_ct_plan_info": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(i32)]),
        "dgamp_ct_project": (C.c_int, [vp, vp, vp, C.c_int, vp]),
        "dgamp_ct_backproject": (C.c_int, [vp, vp, vp, C.c_int, vp]),
        "dgamp_ct_filter": (C.c_int, [vp, vp, vp, vp]),
        "dgamp_ct_output_step": (C.c_int, [vp, vp, vp, vp, dbl, dbl, vp, vp, vp]),
        "dgamp_ct_denoise_tv": (C.c_int, [vp, vp, dbl, vp, vp]),
        "dgamp_ct_denoise_div": (C.c_int, [vp, vp, dbl, i32, vp, vp, vp]),
        "dgamp_ct_probe": (C.c_int, [vp, i32, i64, vp, vp, vp]),
        "dgamp_ct_precond_image": (C.c_int, [vp, vp, vp, C.c_int, vp]),
        "dgamp_ct_solve": (C.c_int, [vp, vp, dbl, i32, vp, vp, C.POINTER(Stats), vp]),
        "dgamp_ct_solve_host": (C.c_int, [vp, vp, dbl, i32, vp, C.POINTER(Stats), vp]),
        "dgamp_ct_solve_launches": (i64, [vp, i32]),
        "dgamp_ct_strerror": (C.c_char_p, [C.c_int]),
        "dgamp_ct_last_cuda_error": (C.c_int, []),
        "dgamp_ct_profile_iteration": (C.c_int, [vp, i32, C.POINTER(dbl), i32, C.POINTER(i32), vp]),
        "dgamp_ct_output_step_noalloc": (C.c_int, [vp, vp, vp, i64, dbl, dbl, vp, vp, vp]),
        "dgamp_ct_get_tuning": (C.c_int, [vp, C.POINTER(Tuning)]),
        "dgamp_ct_set_tuning": (C.c_int, [vp, C.POINTER(Tuning)]),
        "dgamp_ct_cnn_create": (C.c_int, [i32, C.c_uint64, C.POINTER(vp)]),
        "dgamp_ct_cnn_destroy": (None, [vp]),
        "dgamp_ct_cnn_num_params": (i64, [vp]),
        "dgamp_ct_cnn_set_params": (C.c_int, [vp, vp, i64]),
        "dgamp_ct_cnn_get_params": (C.c_int, [vp, vp, i64]),
        "dgamp_ct_cnn_denoise": (C.c_int, [vp, vp, vp, i32, i32, i32, vp, vp]),
        "dgamp_ct_cnn_denoise_jvp": (C.c_int, [vp, vp, vp, C.c_float, i32, i32, vp, vp, vp]),
        "dgamp_ct_solve_batched": (C.c_int, [i32, vp, vp, vp, i32, vp, vp, vp]),
        "dgamp_ct_schedule_lpt": (C.c_int, [i32, vp, i32, vp, vp]),
        "dgamp_ct_cnn_gradients": (C.c_int, [vp, vp, vp, vp, i32, i32, i32, C.POINTER(dbl), vp, vp]),
        "dgamp_ct_cnn_train_step": (C.c_int, [vp, vp, vp, vp, i32, i32, i32, C.c_float, C.POINTER(dbl), vp]),
        "dgamp_ct_plan_set_cnn": (C.c_int, [vp, vp]),
        "dgamp_ct_cnn_test_timeout": (C.c_int, [vp, i32]),
        "dgamp_ct_measure_fp32_peak": (C.c_int, [i32, C.POINTER(dbl), C.POINTER(i32), vp]),
        "dgamp_ct_measure_fp32x2_peak": (C.c_int, [i32, C.POINTER(dbl), C.POINTER(i32), vp]),
        "dgamp_ct_batch_create": (C.c_int, [i32, vp, i32, vp]),
        "dgamp_ct_batch_destroy": (None, [vp]),
        "dgamp_ct_batch_solve": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
        "dgamp_ct_batch_launches": (i64, [vp, i32]),
        "dgamp_ct_solve_trace": (C.c_int, [vp, vp, dbl, i32, vp, vp, C.POINTER(dbl), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_options(**over) -> Options:
    o = Options()
    _check(load().dgamp_ct_default_options(C.byref(o)), "default_options")
    for k, v in over.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _check(rc: int, what: str):
    if rc != OK:
        raise DgampError(rc, what)


def _ptr(t, n_expect=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if n_expect is not None and t.numel() != n_expect:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n_expect}")
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def measure_fp32_peak(reps: int = 5):
    """Measured FP32 FMA throughput of the current GPU (dgamp_ct_measure_fp32_peak):
    returns (TFLOP/s, SM count)."""
    tf = C.c_double()
    sms = C.c_int32()
    _check(load().dgamp_ct_measure_fp32_peak(int(reps), C.byref(tf), C.byref(sms), _stream()),
           "dgamp_ct_measure_fp32_peak")
    return tf.value, sms.value


def measure_fp32x2_peak(reps: int = 5):
    """The same with packed FP32 pairs (dgamp_ct_measure_fp32x2_peak): (TFLOP/s, SM count)."""
    tf = C.c_double()
    sms = C.c_int32()
    _check(load().dgamp_ct_measure_fp32x2_peak(int(reps), C.byref(tf), C.byref(sms), _stream()),
           "dgamp_ct_measure_fp32x2_peak")
    return tf.value, sms.value


def output_step_noalloc(z, y, s_prev, I0: float, tau_p: float, s_out, tau_s_out):
    """dgamp_ct_output_step_noalloc: the output step with no plan and no allocation.

    For callers that cannot allocate device memory while running; every
    buffer is the caller's (``s_out`` float32 like ``z``; ``tau_s_out`` one
    float64 CUDA element).  Calls share one library-owned scratch array, so
    calls that overlap on the GPU must be serialised by the caller.
    """
    import torch
    M = z.numel()
    if not (isinstance(tau_s_out, torch.Tensor) and tau_s_out.is_cuda and tau_s_out.dtype == torch.float64):
        raise TypeError("tau_s_out must be a float64 CUDA tensor")
    _check(load().dgamp_ct_output_step_noalloc(
        _ptr(z, M, "z"), _ptr(y, M, "y"), _ptr(s_prev, M, "s_prev") if s_prev is not None else None,
        int(M), float(I0), float(tau_p), _ptr(s_out, M, "s_out"), C.c_void_p(tau_s_out.data_ptr()), _stream()),
        "dgamp_ct_output_step_noalloc")
    return s_out, tau_s_out


class Plan:
    """One geometry's plan (dgamp_ct_plan).  Tensors are float32 CUDA tensors."""

    def __init__(self, n: int, n_views: int, n_det: int, angles=None, fan=None, **options):
        """fan: None (parallel beam) or dict(src_dist=, det_dist=, det_spacing=)
        for the flat-detector fan beam of dgamp_ct_plan_fan."""
        self._lib = load()
        self.n, self.n_views, self.n_det = int(n), int(n_views), int(n_det)
        g = Geometry(self.n, self.n_views, self.n_det, None)
        self._angles = None
        if angles is not None:
            self._angles = np.ascontiguousarray(angles, dtype=np.float64)
            g.angles = self._angles.ctypes.data_as(C.POINTER(C.c_double))
        self.options = default_options(**options)
        self.fan = fan is not None
        h = C.c_void_p()
        if fan is None:
            _check(self._lib.dgamp_ct_plan(C.byref(g), C.byref(self.options), C.byref(h)), "dgamp_ct_plan")
        else:
            fg = FanGeometry(g, float(fan["src_dist"]), float(fan["det_dist"]), float(fan.get("det_spacing", 1.0)))
            _check(self._lib.dgamp_ct_plan_fan(C.byref(fg), C.byref(self.options), C.byref(h)),
                   "dgamp_ct_plan_fan")
        self._h = h
        fr = C.c_double()
        P = C.c_int32()
        _check(self._lib.dgamp_ct_plan_info(h, C.byref(fr), C.byref(P)), "plan_info")
        self.frob_sq = fr.value
        self.fft_len = P.value

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.dgamp_ct_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def N(self):
        return self.n * self.n

    @property
    def M(self):
        return self.n_views * self.n_det

    def tuning(self):
        """The plan's implementation choices (dgamp_ct_tuning): {"filter_mode": 0 FFT | 1 Toeplitz,
        "tv_kb": steps per TV launch, "tv_rows": rows of a TV block's region, "sino_fused": 1 if the
        solve runs H A x, the output step and H s as one kernel, "bp_mode": 0 pixel-driven | 1
        ray-driven A^T, "pj_seg": warps splitting the steps of 32 rays in A, "tv_vrows": rows of a TV
        region per thread (2, 4 or 8), "pj_band": 0 for that ray-group A or the lines of a shared-memory
        band of the banded A (16 or 32), "pj_waves": full waves of blocks of the banded A (1 or 2)}."""
        t = Tuning()
        _check(self._lib.dgamp_ct_get_tuning(self._h, C.byref(t)), "get_tuning")
        return {name: getattr(t, name) for name, _ in Tuning._fields_}

    def set_tuning(self, **choices):
        """Set some of the tuning's fields by name; the others keep their values."""
        t = Tuning(*([-1] * len(Tuning._fields_)))
        for k, v in choices.items():
            if k not in dict(Tuning._fields_):
                raise TypeError(f"unknown tuning field {k!r}")
            setattr(t, k, int(v))
        _check(self._lib.dgamp_ct_set_tuning(self._h, C.byref(t)), "set_tuning")

    def set_options(self, **options):
        """Change some options; if the library rejects them the plan keeps its
        previous options (here and in the library)."""
        o = Options.from_buffer_copy(self.options)
        for k, v in options.items():
            if k not in dict(Options._fields_):
                raise TypeError(f"unknown option {k!r}")
            setattr(o, k, v)
        _check(self._lib.dgamp_ct_set_options(self._h, C.byref(o)), "set_options")
        self.options = o

    def _img(self, like=None):
        import torch
        return torch.empty((self.n, self.n), dtype=torch.float32, device="cuda")

    def _sino(self):
        import torch
        return torch.empty((self.n_views, self.n_det), dtype=torch.float32, device="cuda")

    # -- single steps --
    def project(self, img, precond: bool = False, out=None):
        out = self._sino() if out is None else out
        _check(self._lib.dgamp_ct_project(self._h, _ptr(img, self.N, "img"), _ptr(out, self.M, "out"),
                                          int(precond), _stream()), "dgamp_ct_project")
        return out

    def backproject(self, sino, precond: bool = False, out=None):
        out = self._img() if out is None else out
        _check(self._lib.dgamp_ct_backproject(self._h, _ptr(sino, self.M, "sino"), _ptr(out, self.N, "out"),
                                              int(precond), _stream()), "dgamp_ct_backproject")
        return out

    def filter(self, sino, out=None):
        out = self._sino() if out is None else out
        _check(self._lib.dgamp_ct_filter(self._h, _ptr(sino, self.M, "sino"), _ptr(out, self.M, "out"),
                                         _stream()), "dgamp_ct_filter")
        return out

    def output_step(self, z, y, s_prev, I0: float, tau_p: float):
        import torch
        s = self._sino()
        ts = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(self._lib.dgamp_ct_output_step(
            self._h, _ptr(z, self.M, "z"), _ptr(y, self.M, "y"),
            _ptr(s_prev, self.M, "s_prev") if s_prev is not None else None,
            float(I0), float(tau_p), _ptr(s, self.M, "s"), C.c_void_p(ts.data_ptr()), _stream()),
            "dgamp_ct_output_step")
        return s, ts

    def denoise_tv(self, r, lam: float):
        x = self._img()
        _check(self._lib.dgamp_ct_denoise_tv(self._h, _ptr(r, self.N, "r"), float(lam), _ptr(x, self.N, "x"),
                                             _stream()), "dgamp_ct_denoise_tv")
        return x

    def denoise_div(self, r, tau_r: float, t: int):
        import torch
        x = self._img()
        dv = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(self._lib.dgamp_ct_denoise_div(self._h, _ptr(r, self.N, "r"), float(tau_r), int(t),
                                              _ptr(x, self.N, "x"), C.c_void_p(dv.data_ptr()), _stream()),
               "dgamp_ct_denoise_div")
        return x, dv

    def probe(self, t: int, n: int, words: bool = False):
        import torch
        b = torch.empty(n, dtype=torch.float32, device="cuda")
        w = torch.empty(n, dtype=torch.int32, device="cuda") if words else None
        _check(self._lib.dgamp_ct_probe(self._h, int(t), int(n), C.c_void_p(b.data_ptr()),
                                        C.c_void_p(w.data_ptr()) if w is not None else None, _stream()),
               "dgamp_ct_probe")
        return (b, w) if words else b

    def precond_image(self, img, inverse: bool = True, out=None):
        out = self._img() if out is None else out
        _check(self._lib.dgamp_ct_precond_image(self._h, _ptr(img, self.N, "img"), _ptr(out, self.N, "out"),
                                                int(inverse), _stream()), "dgamp_ct_precond_image")
        return out

    # -- the loop --
    def solve(self, counts, I0: float, iters: int, with_stats: bool = False, mu_out=None, x_out=None):
        mu = self._img() if mu_out is None else mu_out
        st, arrays = None, None
        if with_stats:
            st, arrays = _new_stats(iters)
        rc = self._lib.dgamp_ct_solve(self._h, _ptr(counts, self.M, "counts"), float(I0), int(iters),
                                      _ptr(mu, self.N, "mu_out"),
                                      _ptr(x_out, self.N, "x_out") if x_out is not None else None,
                                      C.byref(st) if st is not None else None, _stream())
        _check(rc, "dgamp_ct_solve")
        if with_stats:
            return mu, _stats_dict(st, arrays)
        return mu

    def solve_host(self, counts: np.ndarray, I0: float, iters: int, mu_out: np.ndarray | None = None):
        c = np.ascontiguousarray(counts, dtype=np.float32)
        if c.size != self.M:
            raise ValueError("counts has the wrong size")
        mu = np.empty((self.n, self.n), dtype=np.float32) if mu_out is None else mu_out
        rc = self._lib.dgamp_ct_solve_host(self._h, c.ctypes.data_as(C.c_void_p), float(I0), int(iters),
                                           mu.ctypes.data_as(C.c_void_p), None, _stream())
        _check(rc, "dgamp_ct_solve_host")
        return mu

    def profile_iteration(self, reps: int = 5):
        """Mean per-kernel durations (ms) of one iteration, in launch order."""
        k_tv = max(int(self.options.k_tv), 0)
        metric = bool(self.options.tv_metric) and k_tv > 0 and self.options.c_tv > 0
        cap = 8 + (4 * k_tv + 1 if metric else k_tv)
        arr = (C.c_double * cap)()
        cnt = C.c_int32()
        _check(self._lib.dgamp_ct_profile_iteration(self._h, int(reps), arr, cap, C.byref(cnt), _stream()),
               "dgamp_ct_profile_iteration")
        if self.fan:
            names = ["vinv_stage_project", "output_step", "backproject", "vinv_update", "probe_input"]
        else:
            fused = self.tuning()["sino_fused"] and not self.options.output_moments
            sino = ["sino_step"] if fused else ["filter_z", "output_step", "filter_s"]
            names = ["project"] + sino + ["backproject_update", "probe_input"]
        if self.options.denoiser == 2:
            k = cnt.value - len(names) - 4      # the TV launches
            names += ["cnn_pair", "probe_tv"] + [f"tv_block{i}" for i in range(k - 1)] + ["tv_block_final"]
            names += ["select_sums", "select_final"]
        elif self.options.denoiser == 1:
            names += ["cnn_pair", "denoise_final"]
        elif metric:
            # prox-TV in the (V^T V)^{-1} norm: a dual step from p = 0, then per
            # step x(p) in three FFT passes and a dual step, the last one final
            names += ["tvm_dual0"]
            for s in range(1, k_tv + 1):
                names += [f"tvm_rows_fwd{s}", f"tvm_cols{s}", f"tvm_rows_inv{s}"]
                names += [f"tvm_dual{s}"] if s < k_tv else ["tv_final"]
        else:
            k = cnt.value - len(names) - 1
            names += [f"tv_block{i}" for i in range(k)] + ["tv_block_final"]
        return dict(zip(names, [arr[i] for i in range(cnt.value)]))

    def set_cnn(self, net):
        """Attach a learned denoiser (a CNN) or detach it (None); use with options.denoiser = 1 (the network) or 2 (the network judged by prox-TV)."""
        _check(self._lib.dgamp_ct_plan_set_cnn(self._h, net._h if net is not None else None), "plan_set_cnn")
        self._cnn = net

    def solve_trace(self, counts, I0: float, iters: int):
        """Solve and return (mu, r^t for t = 1..iters as [iters][n][n], tau_r^t)."""
        import torch
        mu = self._img()
        rt = torch.empty((iters, self.n, self.n), dtype=torch.float32, device="cuda")
        tr = np.zeros(iters)
        _check(self._lib.dgamp_ct_solve_trace(self._h, _ptr(counts, self.M, "counts"), float(I0), int(iters),
                                              _ptr(mu), _ptr(rt), tr.ctypes.data_as(C.POINTER(C.c_double)),
                                              _stream()), "dgamp_ct_solve_trace")
        return mu, rt, tr

    def solve_launches(self, iters: int) -> int:
        return int(self._lib.dgamp_ct_solve_launches(self._h, int(iters)))


class CNN:
    """The learned residual denoiser (dgamp_ct_cnn_*): D_sigma(r) = r - sigma f(r/sigma)."""

    def __init__(self, layers: int = 17, seed: int = 0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.dgamp_ct_cnn_create(int(layers), int(seed), C.byref(h)), "dgamp_ct_cnn_create")
        self._h = h
        self.layers = int(layers)
        self.num_params = int(self._lib.dgamp_ct_cnn_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dgamp_ct_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(self._lib.dgamp_ct_cnn_set_params(self._h, a.ctypes.data_as(C.c_void_p), a.size), "cnn_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.dgamp_ct_cnn_get_params(self._h, a.ctypes.data_as(C.c_void_p), a.size), "cnn_get_params")
        return a

    @staticmethod
    def _sig(sigma, batch):
        s = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.float32), (batch,)))
        return s

    def denoise(self, r, sigma):
        import torch
        B, H, W = (1,) + tuple(r.shape) if r.dim() == 2 else tuple(r.shape)
        out = torch.empty_like(r)
        s = self._sig(sigma, B)
        _check(self._lib.dgamp_ct_cnn_denoise(self._h, _ptr(r), s.ctypes.data_as(C.c_void_p), B, H, W, _ptr(out),
                                              _stream()), "cnn_denoise")
        return out

    def denoise_jvp(self, r, b, sigma: float):
        """(D_sigma(r), J_D(r) b) for one [H][W] image on the device."""
        import torch
        H, W = tuple(r.shape)
        out, jb = torch.empty_like(r), torch.empty_like(r)
        _check(self._lib.dgamp_ct_cnn_denoise_jvp(self._h, _ptr(r), _ptr(b, H * W, "b"), float(sigma), H, W,
                                                  _ptr(out), _ptr(jb), _stream()), "cnn_denoise_jvp")
        return out, jb

    def gradients(self, r, x, sigma):
        B, H, W = tuple(r.shape)
        s = self._sig(sigma, B)
        loss = C.c_double()
        g = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.dgamp_ct_cnn_gradients(self._h, _ptr(r), _ptr(x), s.ctypes.data_as(C.c_void_p), B, H, W,
                                                C.byref(loss), g.ctypes.data_as(C.c_void_p), _stream()),
               "cnn_gradients")
        return loss.value, g

    def test_timeout(self, on: bool):
        """Timeout test switch (dgamp_ct_cnn_test_timeout): while on, every
        tensor-core convolution of this network times out on purpose (a 1 ms
        wait on a barrier nothing arrives at) and computes nothing."""
        _check(self._lib.dgamp_ct_cnn_test_timeout(self._h, 1 if on else 0), "cnn_test_timeout")

    def train_step(self, r, x, sigma, lr: float):
        B, H, W = tuple(r.shape)
        s = self._sig(sigma, B)
        loss = C.c_double()
        _check(self._lib.dgamp_ct_cnn_train_step(self._h, _ptr(r), _ptr(x), s.ctypes.data_as(C.c_void_p), B, H, W,
                                                 C.c_float(lr), C.byref(loss), _stream()), "cnn_train_step")
        return loss.value


def schedule_lpt(work, queues: int):
    """Largest-first assignment of jobs to queues (dgamp_ct_schedule_lpt):
    returns (queue of each job, total work per queue)."""
    lib = load()
    w = np.ascontiguousarray(work, dtype=np.int64)
    q = np.empty(w.size, dtype=np.int32)
    load_ = np.empty(int(queues), dtype=np.int64)
    _check(lib.dgamp_ct_schedule_lpt(int(w.size), w.ctypes.data_as(C.c_void_p), int(queues),
                                     q.ctypes.data_as(C.c_void_p), load_.ctypes.data_as(C.c_void_p)),
           "dgamp_ct_schedule_lpt")
    return q, load_


def solve_batched(plans, counts, I0, iters: int, mu_out=None, with_stats: bool = False):
    """dgamp_ct_solve_batched over a list of plans: one slice per plan, each with
    its own counts tensor and I0; returns the list of mu (and per-slice stats)."""
    n = len(plans)
    if len(counts) != n or len(I0) != n:
        raise ValueError("plans, counts and I0 must have the same length")
    lib = load()
    mus = [p._img() for p in plans] if mu_out is None else list(mu_out)
    P = (C.c_void_p * n)(*[p._h.value if isinstance(p._h, C.c_void_p) else p._h for p in plans])
    Cn = (C.c_void_p * n)(*[_ptr(c, p.M, "counts").value for c, p in zip(counts, plans)])
    Mu = (C.c_void_p * n)(*[_ptr(m, p.N, "mu_out").value for m, p in zip(mus, plans)])
    i0 = np.ascontiguousarray(I0, dtype=np.float64)
    st, arrays = None, None
    if with_stats:
        made = [_new_stats(iters) for _ in range(n)]
        arrays = [a for _, a in made]
        st = (Stats * n)(*[r for r, _ in made])
    rc = lib.dgamp_ct_solve_batched(n, P, Cn, i0.ctypes.data_as(C.c_void_p), int(iters), Mu,
                                    st if st is not None else None, _stream())
    _check(rc, "dgamp_ct_solve_batched")
    if with_stats:
        return mus, [_stats_dict(st[k], arrays[k]) for k in range(n)]
    return mus


class Batch:
    """A batch of slices run one launch per phase (dgamp_ct_batch_*): holds the
    plans (which must stay open) and solves them together."""

    def __init__(self, plans, groups: int = 1):
        """groups: slices split largest-first into that many groups whose launches
        run on parallel branches of the iteration graph (1: one launch per phase)."""
        self._lib = load()
        self.plans = list(plans)
        n = len(self.plans)
        P = (C.c_void_p * n)(*[p._h.value if isinstance(p._h, C.c_void_p) else p._h for p in self.plans])
        h = C.c_void_p()
        _check(self._lib.dgamp_ct_batch_create(n, P, int(groups), C.byref(h)), "dgamp_ct_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dgamp_ct_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def launches(self, iters: int) -> int:
        return int(self._lib.dgamp_ct_batch_launches(self._h, int(iters)))

    def solve(self, counts, I0, iters: int, mu_out=None, with_stats: bool = False):
        n = len(self.plans)
        if len(counts) != n or len(I0) != n:
            raise ValueError("counts and I0 must have one entry per slice")
        mus = [p._img() for p in self.plans] if mu_out is None else list(mu_out)
        Cn = (C.c_void_p * n)(*[_ptr(c, p.M, "counts").value for c, p in zip(counts, self.plans)])
        Mu = (C.c_void_p * n)(*[_ptr(m, p.N, "mu_out").value for m, p in zip(mus, self.plans)])
        i0 = np.ascontiguousarray(I0, dtype=np.float64)
        st, arrays = None, None
        if with_stats:
            made = [_new_stats(iters) for _ in range(n)]
            arrays = [a for _, a in made]
            st = (Stats * n)(*[r for r, _ in made])
        rc = self._lib.dgamp_ct_batch_solve(self._h, Cn, i0.ctypes.data_as(C.c_void_p), int(iters), Mu,
                                            st if st is not None else None, _stream())
        _check(rc, "dgamp_ct_batch_solve")
        if with_stats:
            return mus, [_stats_dict(st[k], arrays[k]) for k in range(n)]
        return mus


def flatten_params(ws, bs) -> np.ndarray:
    """Reference-layout parameter vector (per layer W[ky][kx][ci][co] then b) as float32."""
    parts = []
    for w, b in zip(ws, bs):
        parts.append(np.asarray(w, dtype=np.float32).reshape(-1))
        parts.append(np.asarray(b, dtype=np.float32).reshape(-1))
    return np.concatenate(parts)


def unflatten_params(flat: np.ndarray, layers: int = 17, channels: int = 64):
    ws, bs, off = [], [], 0
    for l in range(layers):
        cin = 1 if l == 0 else channels
        cout = 1 if l == layers - 1 else channels
        n = 9 * cin * cout
        ws.append(np.asarray(flat[off:off + n], dtype=np.float64).reshape(3, 3, cin, cout))
        off += n
        bs.append(np.asarray(flat[off:off + cout], dtype=np.float64))
        off += cout
    return ws, bs
