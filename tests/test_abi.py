"""C-ABI checks that need no GPU: the library builds, loads, and exports every
function include/gl.h declares; host-only entry points behave; calls that need
a GPU fail with an error code, not a crash, when none is present."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2410_05408_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header=None, prefix="gl_"):
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h") and (header is None or fn == header):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(" + prefix +
                                r"[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(binding.LIB_PATH)
    declared = _declared_functions("gl.h")
    assert "gl_lightcurve_batch" in declared and "gl_context_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.EXPORTED) == set(declared)


def test_peaks_library_exports_its_header():
    build.build()
    lib = ctypes.CDLL(build.PEAKS_LIB)
    declared = _declared_functions("gl_peaks.h", prefix="glp_")
    assert declared == ["glp_measure"]
    for name in declared:
        assert hasattr(lib, name), name
    # bad arguments are refused before any CUDA call
    d = ctypes.c_double()
    assert lib.glp_measure(0, 7, 3, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d)) == -1
    assert lib.glp_measure(0, 0, 0, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d)) == -1
    assert lib.glp_measure(0, 0, 3, None, None, None) == -1


def test_q_to_u_host_entry_point():
    q1 = np.linspace(0, 1, 11)
    q2 = np.linspace(1, 0, 11)
    u1, u2 = binding.gl_q_to_u(q1, q2)
    np.testing.assert_allclose((u1 + u2) ** 2, q1, atol=1e-15)
    lib = binding.load()
    assert lib.gl_q_to_u(-1, None, None, None, None) == binding.GL_EINVAL


def test_null_context_is_rejected():
    lib = binding.load()
    assert lib.gl_lightcurve_batch(None, None, None, None, 0, None) == binding.GL_EINVAL
    assert lib.gl_sync(None, None) == binding.GL_EINVAL
    assert lib.gl_context_destroy(None) == binding.GL_OK
    assert lib.gl_context_create(None, 0) == binding.GL_EINVAL
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert lib.gl_mlp_profile(None, 1) == binding.GL_EINVAL
    assert lib.gl_mlp_profile_read(None, 0, ctypes.byref(ms), ctypes.byref(n)) == binding.GL_EINVAL


def test_context_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = binding.load()
    h = ctypes.c_void_p()
    rc = lib.gl_context_create(ctypes.byref(h), 0)
    assert rc in (binding.GL_ECUDA, binding.GL_EINVAL)
    assert not h.value
