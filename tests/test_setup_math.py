"""Host build of the per-set transcendentals (own FP64 sincos and cube root used
by the constants kernel) against long-double libm: Cody-Waite reduction plus
Taylor series, and an FP32 seed plus one Halley step, must stay within a few
units in the last place."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cmath>
#include <random>
#include "gl_math.cuh"
int main() {
  std::mt19937_64 g(1);
  std::uniform_real_distribution<double> U(-1, 1);
  double ws = 0, wc = 0, wb = 0, wn = 0;
  for (int i = 0; i < 300000; i++) {
    double x = (i % 3 == 0) ? U(g) * 7 : (i % 3 == 1 ? U(g) * 1e3 : U(g) * 1e5);
    double s, c;
    gl::sincos_setup(x, &s, &c);
    ws = fmax(ws, (double)fabsl(s - sinl((long double)x)));
    wc = fmax(wc, (double)fabsl(c - cosl((long double)x)));
    wn = fmax(wn, fabs(s * s + c * c - 1.0));
    double a = 0.1 + 0.9 * fabs(U(g));
    long double r = cbrtl((long double)a);
    wb = fmax(wb, (double)(fabsl(gl::cbrt_setup(a) - r) / r));
  }
  double s, c;
  gl::sincos_setup(0.0, &s, &c);
  int exact0 = (s == 0.0 && c == 1.0);
  printf("%.6e %.6e %.6e %.6e %d\n", ws, wc, wb, wn, exact0);
}
'''


def test_own_sincos_and_cbrt_against_long_double():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        with open(src, "w") as fh:
            fh.write(SRC)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        ws, wc, wb, wn, exact0 = subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()
    eps = 2.220446049250313e-16
    assert float(ws) <= 2 * eps and float(wc) <= 2 * eps
    assert float(wb) <= 4 * eps
    assert float(wn) <= 4 * eps
    assert exact0 == "1"
