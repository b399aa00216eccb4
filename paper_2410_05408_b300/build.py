"""Compile the CUDA library ``libgl.so`` in-tree for sm_103a (B300).

nvcc cross-compiles without a GPU.  The library is built beside this file so it
travels with the source tree; nothing is installed into site-packages.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgl.so")
SOURCES = [os.path.join(HERE, "csrc", "gl_api.cu"), os.path.join(HERE, "csrc", "gl_mlp.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))
                  if f.endswith((".cuh", ".h"))] + [os.path.join(ROOT, "include", "gl.h")]
# the pipe-throughput probes of the roofline denominators (include/gl_peaks.h)
PEAKS_LIB = os.path.join(HERE, "libglpeaks.so")
PEAKS_SOURCES = [os.path.join(HERE, "csrc", "gl_peaks.cu")]
PEAKS_DEPS = PEAKS_SOURCES + [os.path.join(ROOT, "include", "gl_peaks.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date(lib: str = LIB, deps=None) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in (deps or DEPS) if os.path.exists(d))


def _compile(lib: str, sources, verbose: bool) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), *sources, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libgl.so and libglpeaks.so if a source changed; returns libgl.so's path."""
    if force or not up_to_date(PEAKS_LIB, PEAKS_DEPS):
        _compile(PEAKS_LIB, PEAKS_SOURCES, verbose)
    if force or not up_to_date():
        _compile(LIB, SOURCES, verbose)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
