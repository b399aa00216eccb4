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


CONV_SRC = r'''
#include <cstdio>
#include <cmath>
#include <cstring>
#include <cfloat>
#include <random>
#include "gl_math.cuh"
static unsigned fb(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static double db(unsigned long long u) { double d; memcpy(&d, &u, 8); return d; }
int main() {
  std::mt19937_64 g(3);
  long bad = 0, n = 0, zeroed = 0;
  auto check = [&](double x) {
    ++n;
    const float got = gl::f64_to_f32_int(x), ref = (float)x;
    if (std::isnan(ref)) { bad += !std::isnan(got); return; }
    if (std::fabs(ref) < FLT_MIN) {   // subnormal range: a signed zero by design
      zeroed += 1;
      bad += !(got == 0.0f && std::signbit(got) == std::signbit(x));
      return;
    }
    bad += fb(got) != fb(ref);
  };
  for (int i = 0; i < 2000000; ++i) check(db(g()));                  // every exponent
  std::uniform_real_distribution<double> U(-1e6, 1e6);
  for (int i = 0; i < 2000000; ++i) check(U(g));                      // times in days
  for (int i = 0; i < 200000; ++i) {                                  // ties and neighbours
    const float f = std::ldexp((float)(g() % 16777215u + 1u), -(int)(g() % 200) + 60);
    const double ulp = std::ldexp(1.0, std::ilogb(f) - 23);
    for (int k = -2; k <= 2; ++k) check((double)f + 0.5 * ulp + k * std::ldexp(ulp, -29));
    check(-((double)f + 0.5 * ulp));
  }
  const double edge[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, DBL_MAX, -DBL_MAX, FLT_MAX,
                         (double)FLT_MAX * (1 + 1e-9), (double)FLT_MAX + std::ldexp(1.0, 103),
                         FLT_MIN, -FLT_MIN, 0.5 * FLT_MIN, DBL_MIN, 1.0, -1.0};
  for (double x : edge) check(x);
  printf("%ld %ld %ld\n", bad, n, zeroed);
}
'''


def test_integer_double_to_float_conversion_matches_the_c_conversion():
    """f64_to_f32_int (the window test's conversion without an FP64 instruction)
    must give the bits of C's round-to-nearest-even conversion for every normal
    result, infinity on overflow, NaN for NaN and a signed zero below FLT_MIN."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "c.cpp")
        exe = os.path.join(d, "c")
        with open(src, "w") as fh:
            fh.write(CONV_SRC)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, src,
                            "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        bad, n, zeroed = map(int, subprocess.run([exe], capture_output=True, text=True,
                                                 check=True).stdout.split())
    assert n > 5_000_000 and zeroed > 0
    assert bad == 0
