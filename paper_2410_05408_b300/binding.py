"""Thin ctypes binding of ``libgl.so`` (C-ABI in include/gl.h).

Argument marshalling only: every step of the light-curve path runs in the CUDA
kernels of the library.  The functions keep the C names.  Arrays may be torch
tensors (CUDA or CPU) or numpy arrays; they must already have the dtype the ABI
names (float64, int64 offsets, int32 nsuper) and be contiguous - nothing is
converted silently.  If the library has not been built, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgl.so")

GL_OK = 0
GL_EINVAL = -1
GL_ENOMEM = -2
GL_ECUDA = -3
GL_ETIMEOUT = -4
GL_ENUMERIC = -5
GL_FP64 = 0
GL_FP32C = 1

EXPORTED = ("gl_context_create", "gl_context_destroy", "gl_last_error", "gl_lightcurve_batch",
            "gl_flux_sky", "gl_q_to_u", "gl_sync", "gl_launch_count", "gl_profile_enable",
            "gl_profile_read", "gl_lightcurve_batch_noalloc", "gl_counts_enable",
            "gl_counts_read", "gl_graphs_enable", "gl_graph_launches", "gl_autotune",
            "gl_configure",
            "gl_flux_sphere", "gl_mlp_param_count", "gl_mlp_create", "gl_mlp_destroy",
            "gl_mlp_set_params", "gl_mlp_get_params", "gl_mlp_get_grads", "gl_mlp_forward",
            "gl_mlp_loss_grad", "gl_mlp_adam", "gl_mlp_status", "gl_lightcurve_surrogate",
            "gl_surrogate_features", "gl_surrogate_targets", "gl_loglike", "gl_item_pipeline",
            "gl_flux_sky_simpson", "gl_lightcurve_locked", "gl_munu_to_feta",
            "gl_feta_to_munu", "gl_munu_prior", "gl_ensemble_init", "gl_ensemble_sweep",
            "gl_mlp_init", "gl_surrogate_train", "gl_surrogate_error_table",
            "gl_surrogate_save", "gl_surrogate_load", "gl_mlp_wait_probe",
            "gl_debug_alloc_limit", "gl_mlp_profile", "gl_mlp_profile_read")

SUR_BINS = 16   # GL_SURROGATE_BINS
GL_EIO = -6


class TrainConfig(ctypes.Structure):
    """gl_train_config: the schedule, batch and shuffle seed of a training run."""
    _fields_ = [("epochs", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("lr", ctypes.c_float), ("lr_end", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}

COUNT_NAMES = ("exposures", "kept", "in_window", "kepler", "items", "item_kepler", "full",
               "partial")

GL_NOALLOC_MAX_SETS = 4096

GL_KERNEL_SETUP = 0
GL_KERNEL_CURVE = 1
GL_KERNEL_SKY = 2
GL_KERNEL_SPHERE = 3
GL_KERNEL_QUAD = 4
GL_KERNEL_SIMPSON = 5
GL_KERNEL_WINDOW = 6
GL_KERNEL_ITEMS = 7
GL_KERNEL_STEP = 8
PROFILE_OFF, PROFILE_EAGER, PROFILE_GRAPH = 0, 1, 2
GL_MLP_KERNEL_GEMM_FWD, GL_MLP_KERNEL_GEMM_BWD, GL_MLP_KERNEL_WGRAD = 0, 1, 2
GL_MLP_KERNEL_IN, GL_MLP_KERNEL_OUT = 3, 4

PARAM_NAMES = ("t0", "period", "a_rs", "b", "ecc", "omega", "k", "f", "eta", "xi", "u1", "u2")


class GLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gl error {code}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = ([("n_sets", ctypes.c_int64)] + [(n, ctypes.c_void_p) for n in PARAM_NAMES] +
                [("g", ctypes.c_void_p), ("zeta", ctypes.c_void_p)])


def _params(params: dict) -> "_Params":
    """Marshal a parameter dict (PARAM_NAMES, plus optional "g" and "zeta" for a
    triaxial shape) into the C struct."""
    n_sets = int(len(params["t0"]))
    return _Params(n_sets, *[_ptr(params[n], "float64") for n in PARAM_NAMES],
                   _ptr(params.get("g"), "float64"), _ptr(params.get("zeta"), "float64"))


class _TuneReport(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("tile", ctypes.c_int), ("nodes", ctypes.c_int),
                ("ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("max_abs_err", ctypes.c_double), ("candidates", ctypes.c_int),
                ("admissible", ctypes.c_int), ("quad_ctas_per_sm", ctypes.c_int),
                ("exposure_block", ctypes.c_int)]


GL_FIT_DIM = 10
FIT_NAMES = ("t0", "period", "a_rs", "b", "k", "mu", "nu", "xi", "q1", "q2")


class _Ensemble(ctypes.Structure):
    _fields_ = [("n_walkers", ctypes.c_int64), ("walkers", ctypes.c_void_p),
                ("logpost", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("n_times", ctypes.c_int64), ("data", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("exptime", ctypes.c_double),
                ("nsuper", ctypes.c_int), ("a", ctypes.c_double), ("prec", ctypes.c_int)]


class _SurStats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int64), ("exposures", ctypes.c_int64),
                ("fallback", ctypes.c_int64)]


class _Times(ctypes.Structure):
    _fields_ = [("t", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("n_times", ctypes.c_int64), ("n_total", ctypes.c_int64),
                ("exptime", ctypes.c_void_p), ("nsuper", ctypes.c_void_p),
                ("nsuper_all", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libgl.so; raises FileNotFoundError if it was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(f"{LIB_PATH} is missing: build it with "
                                    "paper_2410_05408_b300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.gl_context_create.argtypes = [ctypes.POINTER(vp), i32]
        lib.gl_context_create.restype = i32
        lib.gl_context_destroy.argtypes = [vp]
        lib.gl_context_destroy.restype = i32
        lib.gl_last_error.argtypes = [vp]
        lib.gl_last_error.restype = ctypes.c_char_p
        lib.gl_lightcurve_batch.argtypes = [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Times),
                                            vp, i32, vp]
        lib.gl_lightcurve_batch.restype = i32
        lib.gl_lightcurve_locked.argtypes = [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Times),
                                             vp, i32, vp]
        lib.gl_lightcurve_locked.restype = i32
        for name in ("gl_munu_to_feta", "gl_feta_to_munu", "gl_munu_prior"):
            getattr(lib, name).argtypes = [vp, i64, vp, vp, vp, vp, vp]
            getattr(lib, name).restype = i32
        lib.gl_ensemble_init.argtypes = [vp, ctypes.POINTER(_Ensemble), vp]
        lib.gl_ensemble_init.restype = i32
        lib.gl_ensemble_sweep.argtypes = [vp, ctypes.POINTER(_Ensemble), vp, vp, vp]
        lib.gl_ensemble_sweep.restype = i32
        lib.gl_flux_sky.argtypes = [vp, i64] + [vp] * 10 + [i32, vp]
        lib.gl_flux_sky.restype = i32
        lib.gl_flux_sky_simpson.argtypes = [vp, i64] + [vp] * 10 + [i32, i32, vp]
        lib.gl_flux_sky_simpson.restype = i32
        lib.gl_lightcurve_surrogate.argtypes = [vp, vp, ctypes.POINTER(_Params),
                                                ctypes.POINTER(_Times), vp, vp, ctypes.c_double,
                                                vp, ctypes.POINTER(_SurStats)]
        lib.gl_lightcurve_surrogate.restype = i32
        lib.gl_surrogate_features.argtypes = [vp, i64] + [vp] * 12 + [vp]
        lib.gl_surrogate_features.restype = i32
        lib.gl_surrogate_targets.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        lib.gl_surrogate_targets.restype = i32
        lib.gl_loglike.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
        lib.gl_loglike.restype = i32
        lib.gl_mlp_param_count.argtypes = []
        lib.gl_mlp_param_count.restype = i64
        lib.gl_mlp_create.argtypes = [ctypes.POINTER(vp), i32]
        lib.gl_mlp_create.restype = i32
        lib.gl_mlp_destroy.argtypes = [vp]
        lib.gl_mlp_destroy.restype = i32
        for fn in ("gl_mlp_set_params", "gl_mlp_get_params", "gl_mlp_get_grads"):
            getattr(lib, fn).argtypes = [vp, vp, i64]
            getattr(lib, fn).restype = i32
        lib.gl_mlp_forward.argtypes = [vp, i64, vp, vp, vp]
        lib.gl_mlp_forward.restype = i32
        lib.gl_mlp_loss_grad.argtypes = [vp, i64, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        lib.gl_mlp_loss_grad.restype = i32
        lib.gl_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, vp]
        lib.gl_mlp_adam.restype = i32
        lib.gl_mlp_status.argtypes = [vp]
        lib.gl_mlp_status.restype = i32
        lib.gl_mlp_init.argtypes = [vp, ctypes.c_uint64]
        lib.gl_mlp_init.restype = i32
        lib.gl_mlp_wait_probe.argtypes = [vp, i32]
        lib.gl_mlp_wait_probe.restype = i32
        lib.gl_mlp_profile.argtypes = [vp, i32]
        lib.gl_mlp_profile.restype = i32
        lib.gl_mlp_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(i64)]
        lib.gl_mlp_profile_read.restype = i32
        lib.gl_debug_alloc_limit.argtypes = [vp, i64]
        lib.gl_debug_alloc_limit.restype = i32
        lib.gl_surrogate_train.argtypes = [vp, i64, vp, vp, ctypes.POINTER(TrainConfig), i64, i64,
                                           ctypes.POINTER(ctypes.c_double), vp]
        lib.gl_surrogate_train.restype = i32
        lib.gl_surrogate_error_table.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        lib.gl_surrogate_error_table.restype = i32
        lib.gl_surrogate_save.argtypes = [vp, ctypes.c_char_p, vp, ctypes.POINTER(TrainConfig), i64]
        lib.gl_surrogate_save.restype = i32
        lib.gl_surrogate_load.argtypes = [vp, ctypes.c_char_p, vp, ctypes.POINTER(TrainConfig),
                                          ctypes.POINTER(i64)]
        lib.gl_surrogate_load.restype = i32
        lib.gl_flux_sphere.argtypes = [vp, i64] + [vp] * 7 + [i32, vp]
        lib.gl_flux_sphere.restype = i32
        lib.gl_q_to_u.argtypes = [i64, vp, vp, vp, vp]
        lib.gl_q_to_u.restype = i32
        lib.gl_sync.argtypes = [vp, vp]
        lib.gl_sync.restype = i32
        lib.gl_launch_count.argtypes = [vp]
        lib.gl_launch_count.restype = i64
        lib.gl_autotune.argtypes = [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Times), vp, i32,
                                    vp, ctypes.POINTER(_TuneReport)]
        lib.gl_autotune.restype = i32
        lib.gl_configure.argtypes = [vp, i32, i32, i32, i32, i32]
        lib.gl_configure.restype = i32
        lib.gl_counts_enable.argtypes = [vp, i32]
        lib.gl_counts_enable.restype = i32
        lib.gl_counts_read.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i32]
        lib.gl_counts_read.restype = i32
        lib.gl_graphs_enable.argtypes = [vp, i32]
        lib.gl_graphs_enable.restype = i32
        lib.gl_graph_launches.argtypes = [vp]
        lib.gl_graph_launches.restype = i64
        lib.gl_item_pipeline.argtypes = [vp, i32, i64]
        lib.gl_item_pipeline.restype = i32
        lib.gl_lightcurve_batch_noalloc.argtypes = [ctypes.POINTER(_Params),
                                                    ctypes.POINTER(_Times), vp, i32, vp]
        lib.gl_lightcurve_batch_noalloc.restype = i32
        lib.gl_profile_enable.argtypes = [vp, i32]
        lib.gl_profile_enable.restype = i32
        lib.gl_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]
        lib.gl_profile_read.restype = i32
        _lib = lib
        return lib


_TORCH = None   # (torch.Tensor, {dtype name: torch dtype}) once torch is imported
_NP_DTYPES = {n: np.dtype(n) for n in ("float64", "int64", "int32", "float32")}


def _torch():
    global _TORCH
    if _TORCH is None:
        import torch
        _TORCH = (torch.Tensor, {"float64": torch.float64, "int64": torch.int64,
                                 "int32": torch.int32, "float32": torch.float32})
    return _TORCH


def _ptr(a, dtype: str):
    """Raw pointer of a contiguous tensor/array of the given dtype (None stays None).
    (Called ~20 times per light-curve call: the checks are kept cheap.)"""
    if a is None:
        return None
    tensor, want = _TORCH if _TORCH is not None else _torch()
    if isinstance(a, tensor):
        if a.dtype is not want[dtype] or not a.is_contiguous():
            raise TypeError(f"expected contiguous {dtype} tensor, got {a.dtype}")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if a.dtype != _NP_DTYPES[dtype] or not a.flags.c_contiguous:
            raise TypeError(f"expected contiguous {dtype} numpy array, got {a.dtype}")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, rc):
    if rc != GL_OK:
        msg = load().gl_last_error(ctx)
        raise GLError(rc, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream   # torch.cuda.Stream


def gl_context_create(device: int = 0):
    lib = load()
    h = ctypes.c_void_p()
    rc = lib.gl_context_create(ctypes.byref(h), int(device))
    if rc != GL_OK:
        raise GLError(rc, f"gl_context_create(device={device}) failed")
    return h


def gl_context_destroy(ctx) -> int:
    return load().gl_context_destroy(ctx)


def gl_last_error(ctx) -> str:
    s = load().gl_last_error(ctx)
    return s.decode() if s else ""


def gl_lightcurve_batch(ctx, params: dict, t, out, precision: int = GL_FP32C, offsets=None,
                        exptime=None, nsuper=None, nsuper_all: int = 1, stream=None,
                        check: bool = True, locked: bool = False) -> int:
    """Marshal arrays into gl_params / gl_times and call the library.

    ``params`` maps PARAM_NAMES to float64 arrays of n_sets entries (plus optional
    "g", "zeta"); ``exptime`` is a float64 array of n_sets; ``nsuper`` an int32
    array or None (then ``nsuper_all``); ``offsets`` int64 of n_sets + 1 or None for
    a shared grid.  ``locked`` calls gl_lightcurve_locked (tidally locked bodies).
    """
    lib = load()
    n_sets = int(len(params["t0"]))
    p = _params(params)
    n_t = int(len(t))
    n_total = int(len(out))
    tm = _Times(_ptr(t, "float64"), _ptr(offsets, "int64"), 0 if offsets is not None else n_t,
                n_total, _ptr(exptime, "float64"), _ptr(nsuper, "int32"), int(nsuper_all))
    fn = lib.gl_lightcurve_locked if locked else lib.gl_lightcurve_batch
    rc = fn(ctx, ctypes.byref(p), ctypes.byref(tm), _ptr(out, "float64"), int(precision),
            _stream_ptr(stream))
    if check:
        _check(ctx, rc)
    return rc


def gl_lightcurve_batch_noalloc(params: dict, t, out, precision: int = GL_FP32C, offsets=None,
                                exptime=None, nsuper=None, nsuper_all: int = 1,
                                stream=None) -> int:
    """Allocation-free light curves (see include/gl.h): every array must be a
    CUDA tensor on the current device.  Returns the C status code."""
    lib = load()
    n_sets = int(len(params["t0"]))
    p = _params(params)
    tm = _Times(_ptr(t, "float64"), _ptr(offsets, "int64"),
                0 if offsets is not None else int(len(t)), int(len(out)),
                _ptr(exptime, "float64"), _ptr(nsuper, "int32"), int(nsuper_all))
    return lib.gl_lightcurve_batch_noalloc(ctypes.byref(p), ctypes.byref(tm),
                                           _ptr(out, "float64"), int(precision),
                                           _stream_ptr(stream))


def gl_autotune(ctx, params: dict, t, out, precision: int = GL_FP32C, offsets=None,
                exptime=None, nsuper=None, nsuper_all: int = 1, stream=None) -> dict:
    """Run the library's autotuner on this batch; returns its report as a dict."""
    lib = load()
    n_sets = int(len(params["t0"]))
    p = _params(params)
    tm = _Times(_ptr(t, "float64"), _ptr(offsets, "int64"),
                0 if offsets is not None else int(len(t)), int(len(out)),
                _ptr(exptime, "float64"), _ptr(nsuper, "int32"), int(nsuper_all))
    rep = _TuneReport()
    _check(ctx, lib.gl_autotune(ctx, ctypes.byref(p), ctypes.byref(tm), _ptr(out, "float64"),
                                int(precision), _stream_ptr(stream), ctypes.byref(rep)))
    return {f: getattr(rep, f) for f, _ in rep._fields_}


def gl_configure(ctx, precision: int, threads: int = 0, nodes: int = 0,
                 quad_ctas: int = 0, exposure_block: int = 0) -> None:
    """Set the light-curve configuration of a precision directly (0 = default)."""
    _check(ctx, load().gl_configure(ctx, int(precision), int(threads), int(nodes),
                                    int(quad_ctas), int(exposure_block)))


def gl_flux_sky(ctx, x0, y0, z, k, f, eta, xi, u1, u2, out, precision: int = GL_FP32C,
                stream=None, check: bool = True) -> int:
    lib = load()
    n = int(len(out))
    rc = lib.gl_flux_sky(ctx, n, *[_ptr(a, "float64") for a in (x0, y0, z, k, f, eta, xi, u1, u2)],
                         _ptr(out, "float64"), int(precision), _stream_ptr(stream))
    if check:
        _check(ctx, rc)
    return rc


def gl_flux_sky_simpson(ctx, x0, y0, z, k, f, eta, xi, u1, u2, out, n_intervals: int,
                        precision: int = GL_FP32C, stream=None, check: bool = True) -> int:
    lib = load()
    n = int(len(out))
    rc = lib.gl_flux_sky_simpson(ctx, n, *[_ptr(a, "float64") for a in
                                           (x0, y0, z, k, f, eta, xi, u1, u2)],
                                 _ptr(out, "float64"), int(n_intervals), int(precision),
                                 _stream_ptr(stream))
    if check:
        _check(ctx, rc)
    return rc


def gl_munu(ctx, op: str, a, b, c, d, stream=None) -> None:
    """op: "to_feta" ((mu, nu) -> (f, eta)), "to_munu" ((f, eta) -> (mu, nu)) or
    "prior" ((u, w) -> (mu, nu)); four device float64 arrays of equal length."""
    fn = {"to_feta": "gl_munu_to_feta", "to_munu": "gl_feta_to_munu",
          "prior": "gl_munu_prior"}[op]
    _check(ctx, getattr(load(), fn)(ctx, int(len(a)), *[_ptr(x, "float64") for x in (a, b, c, d)],
                                    _stream_ptr(stream)))


class Ensemble:
    """Device-resident stretch-move ensemble (gl_ensemble_init / gl_ensemble_sweep):
    walkers (n x GL_FIT_DIM), logpost, box bounds and data are torch CUDA tensors
    kept by the caller; sweep() takes the 3 n uniforms of one sweep."""

    def __init__(self, ctx, walkers, lo, hi, t, data, sigma, exptime: float, nsuper: int,
                 precision: int = GL_FP32C, a: float = 2.0):
        import torch
        self.ctx = ctx
        self.walkers = walkers
        self.logpost = torch.empty(walkers.shape[0], dtype=torch.float64, device=walkers.device)
        self._keep = (lo, hi, t, data, sigma)
        self.e = _Ensemble(int(walkers.shape[0]), _ptr(walkers, "float64"),
                           _ptr(self.logpost, "float64"), _ptr(lo, "float64"),
                           _ptr(hi, "float64"), _ptr(t, "float64"), int(len(t)),
                           _ptr(data, "float64"), _ptr(sigma, "float64"), float(exptime),
                           int(nsuper), float(a), int(precision))

    def init(self, stream=None):
        _check(self.ctx.handle, load().gl_ensemble_init(self.ctx.handle, ctypes.byref(self.e),
                                                        _stream_ptr(stream)))

    def sweep(self, rnd, accepted=None, stream=None):
        _check(self.ctx.handle, load().gl_ensemble_sweep(
            self.ctx.handle, ctypes.byref(self.e), _ptr(rnd, "float64"),
            None if accepted is None else accepted.data_ptr(), _stream_ptr(stream)))


def gl_flux_sphere(ctx, x0, y0, z, p, u1, u2, out, precision: int = GL_FP32C, stream=None,
                   check: bool = True) -> int:
    lib = load()
    n = int(len(out))
    rc = lib.gl_flux_sphere(ctx, n, *[_ptr(a, "float64") for a in (x0, y0, z, p, u1, u2)],
                            _ptr(out, "float64"), int(precision), _stream_ptr(stream))
    if check:
        _check(ctx, rc)
    return rc


def gl_lightcurve_surrogate(ctx, mlp, params: dict, t, out, bound_table, bound_limit: float,
                            exptime=None, nsuper_all: int = 1, offsets=None, stream=None) -> dict:
    """Surrogate light curves (device buffers, uniform nsuper); returns the stats."""
    lib = load()
    n_sets = int(len(params["t0"]))
    p = _params(params)
    tm = _Times(_ptr(t, "float64"), _ptr(offsets, "int64"),
                0 if offsets is not None else int(len(t)), int(len(out)),
                _ptr(exptime, "float64"), None, int(nsuper_all))
    st = _SurStats()
    _check(ctx, lib.gl_lightcurve_surrogate(ctx, mlp.handle, ctypes.byref(p), ctypes.byref(tm),
                                            _ptr(out, "float64"), _ptr(bound_table, "float32"),
                                            float(bound_limit), _stream_ptr(stream),
                                            ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def gl_surrogate_features(ctx, x0, y0, k, f, eta, xi, u1, u2, feat, scale, r_area, bins,
                          stream=None):
    lib = load()
    _check(ctx, lib.gl_surrogate_features(
        ctx, int(len(x0)), *[_ptr(a, "float64") for a in (x0, y0, k, f, eta, xi, u1, u2)],
        _ptr(feat, "float32"), _ptr(scale, "float32"), _ptr(r_area, "float64"),
        _ptr(bins, "int32"), _stream_ptr(stream)))


def gl_surrogate_targets(ctx, f_oblate, f_sphere, scale, t, stream=None):
    lib = load()
    _check(ctx, lib.gl_surrogate_targets(ctx, int(len(t)), _ptr(f_oblate, "float64"),
                                         _ptr(f_sphere, "float64"), _ptr(scale, "float32"),
                                         _ptr(t, "float32"), _stream_ptr(stream)))


def gl_loglike(ctx, flux, data, sigma, loglike, stream=None):
    lib = load()
    n_sets, n_times = int(len(loglike)), int(len(data))
    _check(ctx, lib.gl_loglike(ctx, n_sets, n_times, _ptr(flux, "float64"),
                               _ptr(data, "float64"), _ptr(sigma, "float64"),
                               _ptr(loglike, "float64"), _stream_ptr(stream)))


def gl_q_to_u(q1, q2):
    q1 = np.ascontiguousarray(q1, dtype=np.float64)
    q2 = np.ascontiguousarray(q2, dtype=np.float64)
    u1 = np.empty_like(q1)
    u2 = np.empty_like(q1)
    rc = load().gl_q_to_u(q1.size, q1.ctypes.data, q2.ctypes.data, u1.ctypes.data, u2.ctypes.data)
    if rc != GL_OK:
        raise GLError(rc, "gl_q_to_u")
    return u1, u2


def gl_sync(ctx, stream=None) -> int:
    return load().gl_sync(ctx, _stream_ptr(stream))


def gl_launch_count(ctx) -> int:
    return load().gl_launch_count(ctx)


def gl_counts_enable(ctx, on: bool = True) -> int:
    return load().gl_counts_enable(ctx, int(bool(on)))


def gl_counts_read(ctx) -> dict:
    buf = (ctypes.c_int64 * len(COUNT_NAMES))()
    _check(ctx, load().gl_counts_read(ctx, buf, len(COUNT_NAMES)))
    return dict(zip(COUNT_NAMES, list(buf)))


def gl_graphs_enable(ctx, on: bool = True) -> int:
    return load().gl_graphs_enable(ctx, int(bool(on)))


def gl_graph_launches(ctx) -> int:
    return load().gl_graph_launches(ctx)


def gl_item_pipeline(ctx, on: bool = True, max_items: int = 0) -> None:
    _check(ctx, load().gl_item_pipeline(ctx, int(bool(on)), int(max_items)))


def gl_profile_enable(ctx, on=True) -> int:
    """on: False/0 off, True/1 eager per-kernel events, 2 event nodes inside the
    replayed step graph (PROFILE_GRAPH)."""
    mode = int(on) if not isinstance(on, bool) else int(on)
    return load().gl_profile_enable(ctx, mode)


def gl_profile_read(ctx, kind: int):
    """(total device milliseconds, number of timed launches) of a kernel kind."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(ctx, load().gl_profile_read(ctx, int(kind), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


class Mlp:
    """Owns one gl_mlp (surrogate network); arrays are float32 tensors/arrays."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.gl_mlp_create(ctypes.byref(h), int(device))
        if rc != GL_OK:
            raise GLError(rc, "gl_mlp_create failed")
        self.handle = h
        self.n_params = int(lib.gl_mlp_param_count())

    def close(self):
        if self.handle is not None:
            load().gl_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc, what):
        if rc != GL_OK:
            raise GLError(rc, what)

    def set_params(self, p):
        self._rc(load().gl_mlp_set_params(self.handle, _ptr(p, "float32"), self.n_params),
                 "gl_mlp_set_params")

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._rc(load().gl_mlp_get_params(self.handle, out.ctypes.data, self.n_params),
                 "gl_mlp_get_params")
        return out

    def get_grads(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._rc(load().gl_mlp_get_grads(self.handle, out.ctypes.data, self.n_params),
                 "gl_mlp_get_grads")
        return out

    def forward(self, x, y, stream=None):
        self._rc(load().gl_mlp_forward(self.handle, int(len(y)), _ptr(x, "float32"),
                                       _ptr(y, "float32"), _stream_ptr(stream)), "gl_mlp_forward")

    def loss_grad(self, x, t, stream=None) -> float:
        loss = ctypes.c_double()
        self._rc(load().gl_mlp_loss_grad(self.handle, int(len(t)), _ptr(x, "float32"),
                                         _ptr(t, "float32"), ctypes.byref(loss),
                                         _stream_ptr(stream)), "gl_mlp_loss_grad")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._rc(load().gl_mlp_adam(self.handle, lr, beta1, beta2, eps, _stream_ptr(stream)),
                 "gl_mlp_adam")

    def status(self) -> int:
        return load().gl_mlp_status(self.handle)

    def wait_probe(self, polls: int):
        self._rc(load().gl_mlp_wait_probe(self.handle, int(polls)), "gl_mlp_wait_probe")

    def profile(self, on: bool = True):
        """Time every launch of the network's kernels with CUDA events (resets)."""
        self._rc(load().gl_mlp_profile(self.handle, 1 if on else 0), "gl_mlp_profile")

    def profile_read(self, kind: int):
        """(total device ms, timed launches) of kernel kind GL_MLP_KERNEL_*."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._rc(load().gl_mlp_profile_read(self.handle, int(kind), ctypes.byref(ms),
                                            ctypes.byref(n)), "gl_mlp_profile_read")
        return ms.value, n.value

    def init(self, seed: int = 0):
        self._rc(load().gl_mlp_init(self.handle, int(seed)), "gl_mlp_init")

    def train(self, feat, target, cfg: TrainConfig, first_step: int, n_steps: int,
              stream=None) -> float:
        """Steps [first_step, first_step + n_steps) of the run cfg describes; returns
        their mean mini-batch loss."""
        loss = ctypes.c_double()
        self._rc(load().gl_surrogate_train(self.handle, int(len(target)), _ptr(feat, "float32"),
                                           _ptr(target, "float32"), ctypes.byref(cfg),
                                           int(first_step), int(n_steps), ctypes.byref(loss),
                                           _stream_ptr(stream)), "gl_surrogate_train")
        return loss.value

    def error_table(self, feat, target, bins, err=None, stream=None) -> np.ndarray:
        table = np.empty(SUR_BINS, dtype=np.float32)
        self._rc(load().gl_surrogate_error_table(
            self.handle, int(len(target)), _ptr(feat, "float32"), _ptr(target, "float32"),
            _ptr(bins, "int32"), table.ctypes.data, _ptr(err, "float32"), _stream_ptr(stream)),
            "gl_surrogate_error_table")
        return table

    def save(self, path: str, table, cfg: TrainConfig, train_step: int):
        table = np.ascontiguousarray(table, dtype=np.float32)
        self._rc(load().gl_surrogate_save(self.handle, os.fsencode(path), table.ctypes.data,
                                          ctypes.byref(cfg), int(train_step)), "gl_surrogate_save")

    def load(self, path: str):
        """Restore a checkpoint; returns (table, TrainConfig, train_step)."""
        table = np.empty(SUR_BINS, dtype=np.float32)
        cfg = TrainConfig()
        step = ctypes.c_int64()
        self._rc(load().gl_surrogate_load(self.handle, os.fsencode(path), table.ctypes.data,
                                          ctypes.byref(cfg), ctypes.byref(step)),
                 "gl_surrogate_load")
        return table, cfg, step.value


class Context:
    """Owns one gl_context; convenience wrappers over the C functions."""

    def __init__(self, device: int = 0):
        self.handle = gl_context_create(device)
        self.device = device

    def close(self):
        if self.handle is not None:
            gl_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lightcurve(self, params, t, out, exptime, nsuper=None, nsuper_all=1, offsets=None,
                   precision=GL_FP32C, stream=None, locked=False):
        return gl_lightcurve_batch(self.handle, params, t, out, precision, offsets, exptime,
                                   nsuper, nsuper_all, stream, locked=locked)

    def flux_sky(self, x0, y0, z, k, f, eta, xi, u1, u2, out, precision=GL_FP32C, stream=None):
        return gl_flux_sky(self.handle, x0, y0, z, k, f, eta, xi, u1, u2, out, precision, stream)

    def flux_sky_simpson(self, x0, y0, z, k, f, eta, xi, u1, u2, out, n_intervals,
                         precision=GL_FP32C, stream=None):
        return gl_flux_sky_simpson(self.handle, x0, y0, z, k, f, eta, xi, u1, u2, out,
                                   n_intervals, precision, stream)

    def flux_sphere(self, x0, y0, z, p, u1, u2, out, precision=GL_FP32C, stream=None):
        return gl_flux_sphere(self.handle, x0, y0, z, p, u1, u2, out, precision, stream)

    def sync(self, stream=None) -> int:
        return gl_sync(self.handle, stream)

    def launches(self) -> int:
        return gl_launch_count(self.handle)

    def last_error(self) -> str:
        return gl_last_error(self.handle)

    def configure(self, precision, threads=0, nodes=0, quad_ctas=0, exposure_block=0):
        gl_configure(self.handle, precision, threads, nodes, quad_ctas, exposure_block)

    def autotune(self, params, t, out, exptime, nsuper=None, nsuper_all=1, offsets=None,
                 precision=GL_FP32C, stream=None) -> dict:
        return gl_autotune(self.handle, params, t, out, precision, offsets, exptime, nsuper,
                           nsuper_all, stream)

    def counts(self, on: bool = True):
        gl_counts_enable(self.handle, on)

    def counts_read(self) -> dict:
        return gl_counts_read(self.handle)

    def graphs(self, on: bool = True):
        gl_graphs_enable(self.handle, on)

    def graph_launches(self) -> int:
        return gl_graph_launches(self.handle)

    def item_pipeline(self, on: bool = True, max_items: int = 0):
        gl_item_pipeline(self.handle, on, max_items)

    def alloc_limit(self, nbytes: int):
        _check(self.handle, load().gl_debug_alloc_limit(self.handle, int(nbytes)))

    def profile(self, on=True):
        _check(self.handle, gl_profile_enable(self.handle, on))

    def profile_read(self, kind: int):
        return gl_profile_read(self.handle, kind)


# ------------------------------------------------------------------ pipe throughput
GLP_FFMA, GLP_DFMA, GLP_MUFU = 0, 1, 2
_peaks_lib = None


def _load_peaks():
    global _peaks_lib
    if _peaks_lib is None:
        from . import build as _build
        path = _build.PEAKS_LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2410_05408_b300.build.build()")
        lib = ctypes.CDLL(path)
        lib.glp_measure.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
        lib.glp_measure.restype = ctypes.c_int
        _peaks_lib = lib
    return _peaks_lib


def glp_measure(device: int, kind: int, repeats: int = 5) -> dict:
    """Measured throughput of one pipe (include/gl_peaks.h): flops/s (FMA = 2),
    the best launch's milliseconds and operations per launch."""
    f, ms, ops = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = _load_peaks().glp_measure(int(device), int(kind), int(repeats), ctypes.byref(f),
                                   ctypes.byref(ms), ctypes.byref(ops))
    if rc != 0:
        raise GLError(rc, f"glp_measure(kind={kind}) failed")
    return {"flops_per_s": f.value, "best_ms": ms.value, "ops": ops.value}
