"""FP64 CPU oracle for oblate-planet transit light curves.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2410_05408_b300``) never imports it, and this package imports nothing
from the product path.

The arithmetic lives in ``oracle.c`` (plain C, FP64, optional OpenMP); this
module builds it with gcc into ``liboracle.so`` beside the source and exposes it
through ctypes.  Functions and the passages of the paper they follow:

* ``kepler_E``          - Kepler's equation (orbit generalising Sec. 2, Eq. coord-map)
* ``sky_position``      - planet centre in the sky frame (Sec. 2)
* ``projected_ellipse`` - Eqs. dx, dy1, dy2 for a general triaxial ellipsoid (Sec. 2)
* ``oblate_ellipse``    - the b = c case (Appendix A) with the mean-radius
                          parameterisation of Sec. 3
* ``occulted_moments``  - area, Integral(mu) and Integral(r^2) over the occulted region,
                          by adaptive iterated quadrature (the definition the
                          line integrals of Sec. 2 reach)
* ``flux_sky``          - relative flux for a quadratic limb-darkening law
* ``lightcurve``        - batch of light curves with exposure supersampling
* ``flux_sky_batch``    - ``flux_sky`` over arrays (OpenMP)
* ``q_to_u``            - Kipping (2013) map cited in Sec. 3 (not printed there)

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, textbook special cases, Monte Carlo or the paper's worked
example; see the test module docstring for the pin of each function.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP).  Returns the path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        d = ctypes.c_double
        pd = ctypes.POINTER(ctypes.c_double)
        lib.orc_kepler_E.restype = d
        lib.orc_kepler_E.argtypes = [d, d]
        lib.orc_cos_inclination.restype = d
        lib.orc_cos_inclination.argtypes = [d, d, d, d]
        lib.orc_mean_anomaly_conjunction.restype = d
        lib.orc_mean_anomaly_conjunction.argtypes = [d, d]
        lib.orc_sky_position.restype = None
        lib.orc_sky_position.argtypes = [d, d, d, d, d, d, d, pd, pd, pd]
        lib.orc_projected_ellipse.restype = None
        lib.orc_projected_ellipse.argtypes = [d, d, d, d, d, d, pd, pd, pd]
        lib.orc_oblate_ellipse.restype = None
        lib.orc_oblate_ellipse.argtypes = [d, d, d, d, pd, pd, pd]
        lib.orc_q_to_u.restype = None
        lib.orc_q_to_u.argtypes = [d, d, pd, pd]
        lib.orc_occulted_moments.restype = ctypes.c_int
        lib.orc_occulted_moments.argtypes = [d, d, d, d, d, d, pd]
        lib.orc_flux_sky.restype = d
        lib.orc_flux_sky.argtypes = [d, d, d, d, d, d, d, d, d]
        lib.orc_lightcurve.restype = ctypes.c_int
        lib.orc_lightcurve.argtypes = ([ctypes.c_int64] + [pd] * 14 + [ctypes.c_int, pd]
                                       + [ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                          pd, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, d,
                                          ctypes.c_int, pd])
        lib.orc_flux_sky_batch.restype = None
        lib.orc_flux_sky_batch.argtypes = [ctypes.c_int64] + [pd] * 11 + [d, ctypes.c_int, pd]
        lib.orc_locked_ellipse.restype = None
        lib.orc_locked_ellipse.argtypes = [d, d, d, d, d, d, d, d, pd, pd, pd]
        lib.orc_triaxial_ellipse.restype = None
        lib.orc_triaxial_ellipse.argtypes = [d, d, d, d, d, d, pd, pd, pd]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_failures.restype = ctypes.c_int64
        lib.orc_failures.argtypes = []
        lib.orc_reset_failures.restype = None
        lib.orc_reset_failures.argtypes = []
        _lib = lib
        return lib


DEFAULT_TOL = 1e-15


class OracleQuadratureError(RuntimeError):
    """Some evaluation's adaptive quadrature ran out of panels before reaching
    its tolerance: that value is not the Sec. 2 integral to the stated accuracy."""


def failures() -> int:
    """Evaluations whose quadrature missed its tolerance since the last reset
    (each one's flux is NaN)."""
    return int(_load().orc_failures())


def reset_failures() -> None:
    _load().orc_reset_failures()


def _checked(run, strict: bool):
    """Run one oracle call with the failure counter reset before it; raise if any
    evaluation in it missed its tolerance (strict), else leave the NaNs."""
    with _lock_calls:
        reset_failures()
        out = run()
        nfail = failures()
    if nfail and strict:
        raise OracleQuadratureError(
            f"{nfail} oracle evaluation(s) did not reach the quadrature tolerance")
    return out


_lock_calls = threading.Lock()


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def kepler_E(M: float, e: float) -> float:
    return _load().orc_kepler_E(float(M), float(e))


def cos_inclination(b: float, a_rs: float, e: float, w: float) -> float:
    return _load().orc_cos_inclination(float(b), float(a_rs), float(e), float(w))


def sky_position(t, t0, period, a_rs, cosi, e, w):
    x, y, z = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_sky_position(float(t), float(t0), float(period), float(a_rs), float(cosi),
                             float(e), float(w), ctypes.byref(x), ctypes.byref(y),
                             ctypes.byref(z))
    return x.value, y.value, z.value


def projected_ellipse(a, b, c, zeta, eta, xi):
    o = [ctypes.c_double() for _ in range(3)]
    _load().orc_projected_ellipse(float(a), float(b), float(c), float(zeta), float(eta),
                                  float(xi), *[ctypes.byref(v) for v in o])
    return tuple(v.value for v in o)


def oblate_ellipse(k, f, eta, xi):
    o = [ctypes.c_double() for _ in range(3)]
    _load().orc_oblate_ellipse(float(k), float(f), float(eta), float(xi),
                               *[ctypes.byref(v) for v in o])
    return tuple(v.value for v in o)


def triaxial_ellipse(k, f, g, zeta, eta, xi):
    """(dx, dy1, dy2) of a triaxial ellipsoid: c the largest semi-axis,
    b = c (1 - g), a = c (1 - f), geometric mean k."""
    o = [ctypes.c_double() for _ in range(3)]
    _load().orc_triaxial_ellipse(float(k), float(f), float(g), float(zeta), float(eta),
                                 float(xi), *[ctypes.byref(v) for v in o])
    return tuple(v.value for v in o)


def locked_ellipse(a, b, c, zeta, eta, xi, alpha, beta):
    """(dx, dy1, dy2) of a tidally locked body (Appendix B) at orbital angle
    alpha and elevation beta."""
    o = [ctypes.c_double() for _ in range(3)]
    _load().orc_locked_ellipse(*[float(v) for v in (a, b, c, zeta, eta, xi, alpha, beta)],
                               *[ctypes.byref(v) for v in o])
    return tuple(v.value for v in o)


def _optional(arr, n):
    if arr is None:
        return None, None
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, dtype=np.float64), (n,)).copy())
    return a, _p(a)


def q_to_u(q1, q2):
    u1, u2 = ctypes.c_double(), ctypes.c_double()
    _load().orc_q_to_u(float(q1), float(q2), ctypes.byref(u1), ctypes.byref(u2))
    return u1.value, u2.value


def occulted_moments(x0, y0, dx, dy1, dy2, tol=DEFAULT_TOL):
    """(area, Integral mu dA, Integral r^2 dA) over the ellipse-disk overlap."""
    out = np.zeros(3)
    st = _load().orc_occulted_moments(float(x0), float(y0), float(dx), float(dy1),
                                      float(dy2), float(tol), _p(out))
    if st < 0:
        raise RuntimeError("oracle quadrature did not reach its tolerance")
    return out


def flux_sky(x0, y0, z, dx, dy1, dy2, u1, u2, tol=DEFAULT_TOL, strict: bool = True):
    """Relative flux of one sky configuration.  OracleQuadratureError if the
    quadrature missed `tol` (strict), else NaN for that case."""
    return _checked(lambda: _load().orc_flux_sky(float(x0), float(y0), float(z), float(dx),
                                                 float(dy1), float(dy2), float(u1), float(u2),
                                                 float(tol)), strict)


PARAM_NAMES = ("t0", "period", "a_rs", "b", "ecc", "omega", "k", "f", "eta", "xi",
               "u1", "u2")


def lightcurve(params: dict, t, exptime, nsuper, offsets=None,
               tol: float = DEFAULT_TOL, nthreads: int = 0, locked: bool = False,
               strict: bool = True) -> np.ndarray:
    """Supersampled light curves for a batch of parameter sets.

    ``params`` maps each of PARAM_NAMES to an array of n_sets floats, and may add
    "g" and "zeta" (triaxial shape: c the largest semi-axis, b = c (1 - g),
    a = c (1 - f); rotation zeta about x').  ``locked`` makes the body
    tidally locked (Appendix B): its projection follows the orbital angle.  With
    ``offsets`` None, ``t`` is one grid shared by every set and the result has
    shape (n_sets, len(t)); otherwise set s owns t[offsets[s]:offsets[s+1]] and the
    result is flat in the same layout.  ``nsuper`` is an int or an array of
    n_sets ints.
    """
    lib = _load()
    arrs = [np.ascontiguousarray(np.asarray(params[n], dtype=np.float64).reshape(-1))
            for n in PARAM_NAMES]
    n_sets = arrs[0].size
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))
    exptime = np.ascontiguousarray(np.broadcast_to(np.asarray(exptime, dtype=np.float64),
                                                   (n_sets,)).copy())
    if offsets is None:
        out = np.empty(n_sets * t.size)
        offp = None
        n_times = t.size
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        out = np.empty(int(offsets[-1]))
        offp = offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        n_times = 0
    if np.ndim(nsuper) == 0:
        ns_arr, ns_p, ns_all = None, None, int(nsuper)
    else:
        ns_arr = np.ascontiguousarray(np.asarray(nsuper, dtype=np.int32))
        ns_p, ns_all = ns_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0
    g_arr, g_p = _optional(params.get("g"), n_sets)
    z_arr, z_p = _optional(params.get("zeta"), n_sets)
    st = _checked(lambda: lib.orc_lightcurve(n_sets, *[_p(a) for a in arrs], g_p, z_p,
                                             int(bool(locked)), _p(t), offp, n_times,
                                             _p(exptime), ns_p, ns_all, float(tol),
                                             int(nthreads), _p(out)), strict)
    if st != 0:
        raise ValueError("oracle rejected its inputs")
    if offsets is None:
        return out.reshape(n_sets, t.size)
    return out


def flux_sky_batch(x0, y0, z, k, f, eta, xi, u1, u2, tol: float = DEFAULT_TOL,
                   nthreads: int = 0, g=None, zeta=None, strict: bool = True) -> np.ndarray:
    """Relative flux for arrays of sky positions and shapes (k, f, eta, xi; with
    g and zeta, the triaxial shape of triaxial_ellipse).  An evaluation whose
    quadrature misses ``tol`` raises OracleQuadratureError (``strict``), else is
    NaN."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
            for a in (x0, y0, z, k, f, eta, xi, u1, u2)]
    n = arrs[0].size
    g_arr, g_p = _optional(g, n)
    z_arr, z_p = _optional(zeta, n)
    out = np.empty(n)
    _checked(lambda: _load().orc_flux_sky_batch(n, *[_p(a) for a in arrs], g_p, z_p, float(tol),
                                                int(nthreads), _p(out)), strict)
    return out


def max_threads() -> int:
    return _load().orc_max_threads()


__all__ = ["build", "kepler_E", "cos_inclination", "sky_position", "projected_ellipse",
           "oblate_ellipse", "q_to_u", "occulted_moments", "flux_sky", "lightcurve",
           "flux_sky_batch", "failures", "reset_failures", "OracleQuadratureError",
           "max_threads", "PARAM_NAMES", "DEFAULT_TOL", "math"]
