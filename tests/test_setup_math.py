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


KEPLER_SRC = r'''
#include <cstdio>
#include <cmath>
#include <cstring>
#include <cfloat>
#include <random>
#include "gl_math.cuh"
typedef long double L;
// independent long-double sky position: E - e sin E = M by Newton from M
static void ref_pos(L tau, L P, L a, L e, L w, L cosi, L* x, L* y) {
  const L pi = 3.14159265358979323846264338327950288L;
  const L sw = sinl(w), cw = cosl(w), se = sqrtl((1 - e) * (1 + e));
  const L cEc = (e + sw) / (1 + e * sw), sEc = se * cw / (1 + e * sw);
  const L Ec = atan2l(sEc, cEc);
  const L M = Ec - e * sinl(Ec) + 2 * pi / P * tau;
  L E = M;
  for (int i = 0; i < 100; ++i) {
    L dE = (E - e * sinl(E) - M) / (1 - e * cosl(E));
    E -= dE;
    if (fabsl(dE) < 1e-19L) break;
  }
  const L X = a * (cosl(E) - e), Y = a * se * sinl(E);
  const L p1 = X * cw - Y * sw, p2 = X * sw + Y * cw;
  *y = -p1;
  *x = p2 * cosi;
}
int main() {
  std::mt19937_64 g(11);
  std::uniform_real_distribution<double> U(0, 1);
  double worst = 0, worst_mid = 0, bad_conv = 0;
  long n = 0;
  for (int i = 0; i < 20000; ++i) {
    const double e = (i % 4 == 0) ? 0.0 : 0.95 * U(g) * U(g);
    const double P = 1 + 500 * U(g), a = 3 + 250 * U(g), w = 6.283185307179586 * U(g);
    const double b = 0.9 * U(g);
    gl::SetConst c;
    if (!gl::set_setup(0.0, P, a, b, e, w, 0.1, 0.2, 0.3, 0.4, 0.4, 0.25, 0.02, 15, &c)) continue;
    for (int k = 0; k < 8; ++k) {
      // times in and around the transit window, and anywhere in the orbit
      double tau = (k < 6) ? c.tau_lo + (c.tau_hi - c.tau_lo) * (1.5 * U(g) - 0.25)
                           : P * (U(g) - 0.5);
      double x, y, z;
      gl::sky_position(c, tau, &x, &y, &z);
      L xr, yr;
      ref_pos(tau, P, a, e, w, c.cosi, &xr, &yr);
      const double err = (double)fmaxl(fabsl(x - xr), fabsl(y - yr)) / a;
      if (err > worst) worst = err;
      if (fabs(xr) < 2 && fabs(yr) < 2) {   // the FP32 midpoint state near the star
        const gl::MidState m = gl::mid_state_at(c, tau, false);
        const double em = (double)fmaxl(fabsl(m.x - xr), fabsl(m.y - yr));
        if (em > worst_mid) worst_mid = em;
      }
      ++n;
    }
  }
  // integer FP32 -> FP64 conversion and the bit-pattern comparison
  for (int i = 0; i < 3000000; ++i) {
    unsigned u = (unsigned)g();
    float f;
    memcpy(&f, &u, 4);
    const double r = gl::f32_to_f64_int(f);
    if (std::isnan(f)) { bad_conv += !std::isnan(r); continue; }
    if (std::fabs(f) < FLT_MIN) { bad_conv += !(r == 0.0 && std::signbit(r) == std::signbit(f)); continue; }
    bad_conv += !(r == (double)f);
    const double m = std::fabs((double)U(g) * 4.0);
    const double x = (double)f;
    bad_conv += gl::abs_le(x, m) != (std::fabs(x) <= m);
  }
  bad_conv += gl::abs_le(NAN, 1.0) || !gl::abs_le(-0.0, 0.0) || gl::abs_le(INFINITY, DBL_MAX);
  printf("%.6e %.6e %ld %.0f\n", worst, worst_mid, n, bad_conv);
}
'''


def test_kepler_newton_step_against_long_double():
    """The FP64 Kepler solve (FP32 Newton, then FP64 Newton steps with a refined
    FP32 reciprocal, accepted below a per-set step bound) against a long-double
    Newton solve of E - e sin E = M on 20 000 random orbits (e up to 0.95):
    sky positions within 2e-14 of a (relative), and the FP32 midpoint state within
    FP32 rounding of the exact position.  Also the integer FP32 -> FP64 conversion
    (exact) and abs_le (|x| <= m by bit patterns)."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cpp")
        exe = os.path.join(d, "k")
        with open(src, "w") as fh:
            fh.write(KEPLER_SRC)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, src,
                            "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        worst, worst_mid, n, bad = subprocess.run([exe], capture_output=True, text=True,
                                                  check=True).stdout.split()
    assert int(n) > 100_000
    assert float(worst) <= 2e-14, worst   # measured 2.0e-15
    assert float(worst_mid) <= 1.2e-7, worst_mid   # FP32 rounding of |x| < 2
    assert float(bad) == 0


KEYS_SRC = r'''
#include <cstdio>
#include <cmath>
#include <cstring>
#include <cfloat>
#include <random>
#include "gl_math.cuh"
static double db(unsigned long long u) { double d; memcpy(&d, &u, 8); return d; }
int main() {
  std::mt19937_64 g(9);
  std::uniform_real_distribution<double> U(-3.0, 3.0);
  long bad = 0, n = 0;
  const double edge[] = {0.0, -0.0, 1.0, -1.0, DBL_MIN, -DBL_MIN, DBL_MAX, -DBL_MAX, INFINITY,
                         -INFINITY, 5e-324, -5e-324, 0.25, 0.02, -0.02};
  auto pick = [&](int i) -> double {
    if (i % 4 == 0) return edge[g() % 15];
    if (i % 4 == 1) return db(g());             // any bit pattern, every exponent
    return U(g);
  };
  for (int i = 0; i < 4000000; ++i) {
    const double a = pick(i), b = pick(i + 1);
    if (std::isnan(a) || std::isnan(b)) continue;
    ++n;
    // order of values (pairs of zeros aside: -0 sorts just below +0, pinned below)
    if (!(a == 0.0 && b == 0.0)) {
      bad += (gl::dkey(a) < gl::dkey(b)) != (a < b);
      bad += (gl::dkey(a) <= gl::dkey(b)) != (a <= b);
    }
    bad += gl::neg_bits(a) != (a < 0.0);
    const double m = std::fabs(b);
    bad += gl::abs_lt(a, m) != (std::fabs(a) < m);
    bad += gl::abs_le(a, m) != (std::fabs(a) <= m);
    bad += gl::finite_bits(a) != (bool)std::isfinite(a);
  }
  // NaN of either sign: ordered by its sign bit, never finite, never below a bound
  const double pnan = db(0x7ff8000000000000ull), nnan = db(0xfff8000000000000ull);
  bad += gl::neg_bits(pnan) || !gl::neg_bits(nnan);
  bad += !(gl::dkey(pnan) > gl::dkey(INFINITY)) || !(gl::dkey(nnan) < gl::dkey(-INFINITY));
  bad += gl::abs_lt(pnan, 1.0) || gl::abs_lt(nnan, 1.0) || gl::abs_le(nnan, DBL_MAX);
  bad += gl::finite_bits(pnan) || gl::finite_bits(nnan);
  bad += gl::dkey(-0.0) != gl::dkey(0.0) - 1 || gl::neg_bits(-0.0) || !gl::abs_le(-0.0, 0.0);
  printf("%ld %ld\n", bad, n);
}
'''


def test_integer_keys_order_doubles_like_their_values():
    """dkey, neg_bits, abs_lt, abs_le and finite_bits (the integer compares that
    replace FP64 compares in the window test, sign tests and series branches)
    against the FP64 comparisons on random bit patterns, ordinary values and
    edge cases (zeros, subnormals, extremes, infinities; -0 sorts just below +0;
    a NaN sorts by its sign bit, beyond the infinity of that sign)."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cpp")
        exe = os.path.join(d, "k")
        with open(src, "w") as fh:
            fh.write(KEYS_SRC)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, src,
                            "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        bad, n = map(int, subprocess.run([exe], capture_output=True, text=True,
                                         check=True).stdout.split())
    assert n > 3_000_000
    assert bad == 0
