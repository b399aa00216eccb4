"""Host build of the quadrature's case analysis (no GPU), checked by other routes:

* maybe_two_maxima: where it says "one maximum", g(th) = |p(th)|^2 - 1 sampled on a
  fine grid has exactly one local maximum, and Newton's method (the whole-ellipse
  path) lands on it;
* crossing-arc classification by parity: the inside/outside flags agree with the
  sign of g at each arc's midpoint, evaluated directly from the ellipse;
* the crossing moments with gathered arcs equal the whole-ellipse moments when the
  ellipse lies inside the disk and approach them as it reaches the limb;
* the FP32 crossings (crossing_roots_f32) against the roots of the FP64 quartic of
  the same centre: the same count, roots within 1e-4 (1 + |t|), the FP64 fallback
  rare on random limb geometries and taken at near-tangency;
* the short path of the FP32 crossing items (partial_short: no crossing or two)
  gives the bits of the general routine (partial_general) on the same items.
"""
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
using namespace gl;
// g(th) of the ellipse x = x0 + dx cos th, y = y0 + dy1 cos th + dy2 sin th
static double gdir(const SetConst& c, double x0, double y0, double th) {
  double x = x0 + c.dx * cos(th), y = y0 + c.dy1 * cos(th) + c.dy2 * sin(th);
  return x * x + y * y - 1.0;
}
int main() {
  std::mt19937_64 gen(12);
  std::uniform_real_distribution<double> U(0, 1);
  long n_one = 0, bad_count = 0, n_two_flag = 0;
  double worst_angle = 0;
  const int M = 4096;
  for (int it = 0; it < 60000; ++it) {
    double k = 0.01 + 0.3 * U(gen), f = 0.95 * U(gen), eta = acos(U(gen)), xi = M_PI * U(gen);
    SetConst c;
    set_setup(0, 10, 20, 0.1, 0, M_PI / 2, k, f, eta, xi, 0.4, 0.25, 0.01, 1, &c);
    double rho = (1 - c.req) * sqrt(U(gen)), ph = 2 * M_PI * U(gen);
    double x0 = rho * cos(ph), y0 = rho * sin(ph);
    if (!maybe_two_maxima(c, (float)x0, (float)y0)) {
      ++n_one;
      // local maxima of g on a fine periodic grid
      int nmax = 0;
      double thmax = 0;
      for (int j = 0; j < M; ++j) {
        double a = gdir(c, x0, y0, 2 * M_PI * (j - 1) / M), b = gdir(c, x0, y0, 2 * M_PI * j / M),
               d = gdir(c, x0, y0, 2 * M_PI * (j + 1) / M);
        if (b > a && b >= d) { ++nmax; thmax = 2 * M_PI * j / M; }
      }
      if (nmax != 1) ++bad_count;
      double omr2 = (1 - x0) * (1 + x0) - y0 * y0;
      Geo<double> g = make_geo<double>(c, x0, y0, omr2);
      Trig2<double> t = limb_poly<double>(c, x0, y0, omr2);
      double cs, ss;
      nearest_limb_angle<double>(g, t, &cs, &ss);
      double d = fabs(remainder(atan2(ss, cs) - thmax, 2 * M_PI));
      if (d > worst_angle) worst_angle = d;
    } else {
      ++n_two_flag;
    }
  }
  // parity classification of crossing arcs vs direct midpoint signs
  long arcs = 0, mismatch = 0;
  for (int it = 0; it < 40000; ++it) {
    double k = 0.01 + 0.3 * U(gen), f = 0.95 * U(gen), eta = acos(U(gen)), xi = M_PI * U(gen);
    SetConst c;
    set_setup(0, 10, 20, 0.1, 0, M_PI / 2, k, f, eta, xi, 0.4, 0.25, 0.01, 1, &c);
    double rho = 1 - c.req + 2 * c.req * U(gen), ph = 2 * M_PI * U(gen);
    double x0 = rho * cos(ph), y0 = rho * sin(ph);
    double omr2 = (1 - x0) * (1 + x0) - y0 * y0;
    Trig2<double> t = limb_poly<double>(c, x0, y0, omr2);
    int kb = frame_choice<double>(t);
    Frame<double> fr = make_frame_k<double>(t, kb);
    double tr[8];
    int nr = frame_roots<double>(fr, tr);
    if (nr < 2 || (nr & 1)) continue;
    bool wrap_in = fr.q[4] < 0.0;
    for (int i = 0; i + 1 < nr; ++i) {
      bool parity_in = wrap_in != (((i + 1) & 1) != 0);
      double ct, st;
      frame_angle<double>(fr, 0.5 * (tr[i] + tr[i + 1]), &ct, &st);
      double gm = gdir(c, x0, y0, atan2(st, ct));
      if (fabs(gm) < 1e-12) continue;
      ++arcs;
      if (parity_in != (gm < 0)) ++mismatch;
    }
  }
  printf("%ld %ld %ld %.3e %ld %ld\n", n_one, bad_count, n_two_flag, worst_angle, arcs, mismatch);
}
'''


SRC_F32 = r'''
#include <cstdio>
#include <cmath>
#include <random>
#include "gl_math.cuh"
using namespace gl;
// FP32 and FP64 frames of the same (FP32) centre, as the FP32 quadrature forms them
static void frames(const SetConst& c, float x0, float y0, Frame<float>* ff, Frame<double>* fd) {
  const double xd = x0, yd = y0, omr2 = fma(-yd, yd, fma(-xd, xd, 1.0));
  const Trig2<float> tf = limb_poly<float>(c, x0, y0, (float)omr2);
  const int kb = frame_choice<float>(tf);
  *ff = make_frame_k<float>(tf, kb);
  *fd = make_frame_k<double>(limb_poly<double>(c, xd, yd, omr2), kb);
}
int main() {
  std::mt19937_64 gen(21);
  std::uniform_real_distribution<double> U(0, 1);
  long n = 0, fallback = 0, count_mismatch = 0, with_roots = 0;
  double worst = 0;
  for (int it = 0; it < 200000; ++it) {
    double k = 0.01 + 0.3 * U(gen), f = 0.95 * U(gen), eta = acos(U(gen)), xi = M_PI * U(gen);
    SetConst c;
    set_setup(0, 10, 20, 0.1, 0, M_PI / 2, k, f, eta, xi, 0.4, 0.25, 0.01, 1, &c);
    double rho = 1 - c.req + 2 * c.req * U(gen), ph = 2 * M_PI * U(gen);
    Frame<float> ff;
    Frame<double> fd;
    frames(c, (float)(rho * cos(ph)), (float)(rho * sin(ph)), &ff, &fd);
    float t32[4];
    double t64[8];
    const int n64 = frame_roots<double>(fd, t64), n32 = crossing_roots_f32(ff, t32);
    ++n;
    if (n32 < 0) { ++fallback; continue; }
    if (n32 != n64) { ++count_mismatch; continue; }
    with_roots += n32 > 0;
    for (int i = 0; i < n32; ++i)
      worst = fmax(worst, fabs(t32[i] - t64[i]) / (1 + fabs(t64[i])));
  }
  // near-tangency: a circle (f = 0) whose edge passes about 1e-9 beyond the limb
  // (the FP32 centre moves it by up to ~1e-7) crosses it twice, very close
  // together: mostly the FP64 fallback or no crossing; a pair that does stand
  // must be the FP64 quartic's pair for the same centre
  long tangent_total = 0, tangent_fb = 0, tangent_zero = 0, tangent_bad = 0;
  for (int it = 0; it < 2000; ++it) {
    double k = 0.05 + 0.2 * U(gen), ph = 2 * M_PI * U(gen);
    SetConst c;
    set_setup(0, 10, 20, 0.1, 0, M_PI / 2, k, 0.0, 0.3, 0.2, 0.4, 0.25, 0.01, 1, &c);
    const double rho = 1 - c.req + 1e-9;
    Frame<float> ff;
    Frame<double> fd;
    frames(c, (float)(rho * cos(ph)), (float)(rho * sin(ph)), &ff, &fd);
    float t32[4];
    double t64[8];
    const int n32 = crossing_roots_f32(ff, t32), n64 = frame_roots<double>(fd, t64);
    ++tangent_total;
    tangent_fb += n32 < 0;
    tangent_zero += n32 == 0;
    if (n32 > 0) {
      bool same = n32 == n64;
      for (int i = 0; same && i < n32; ++i)
        same = fabs(t32[i] - t64[i]) <= 1e-4 * (1 + fabs(t64[i]));
      tangent_bad += !same;
    }
  }
  printf("%ld %ld %ld %ld %.3e %ld %ld %ld %ld\n", n, fallback, count_mismatch, with_roots, worst,
         tangent_total, tangent_fb, tangent_zero, tangent_bad);
}
'''


SRC_SHORT = r'''
#include <cstdio>
#include <cmath>
#include <cstring>
#include <random>
#include "gl_math.cuh"
using namespace gl;
int main() {
  std::mt19937_64 gen(5);
  std::uniform_real_distribution<double> U(0, 1);
  NodeRule<float> rule;
  rule.n = 16;
  for (int j = 0; j < 16; ++j) {   // any rule serves for an equality test
    const double s = -1 + (2 * j + 1) / 16.0;
    rule.sig[j] = (float)sin(M_PI * s / 2);
    rule.wt[j] = (float)(M_PI / 16 * cos(M_PI * s / 2));
    rule.cph[j] = (float)cos(M_PI * rule.sig[j]);
    rule.sph[j] = (float)sin(M_PI * rule.sig[j]);
  }
  long n[3] = {0, 0, 0}, differ = 0, general = 0;
  for (int it = 0; it < 100000; ++it) {
    double k = 0.01 + 0.3 * U(gen), f = 0.9 * U(gen), eta = acos(U(gen)), xi = M_PI * U(gen);
    SetConst c;
    set_setup(0, 10, 20, 0.1, 0, M_PI / 2, k, f, eta, xi, 0.4, 0.25, 0.01, 1, &c);
    double rho = 1 - c.req + 2 * c.req * U(gen), ph = 2 * M_PI * U(gen);
    const float x0 = (float)(rho * cos(ph)), y0 = (float)(rho * sin(ph));
    const double xd = x0, yd = y0;
    const float omr2 = (float)fma(-yd, yd, fma(-xd, xd, 1.0));
    if (maybe_two_maxima(c, x0, y0)) continue;
    float a[3], b[3];
    occulted_r<float>(c, x0, y0, omr2, kPartial, rule, a);   // short path where it applies
    const Geo<float> g = make_geo<float>(c, x0, y0, omr2);
    const Trig2<float> tg = limb_poly<float>(c, x0, y0, omr2);
    const int kb = frame_choice<float>(tg);
    const Frame<float> frr = make_frame_k<float>(tg, kb);
    float r32[4];
    const int nr = crossing_roots_f32(frr, r32);
    const float cmx[2] = {0, 0}, smx[2] = {0, 0};
    partial_general<float>(c, x0, y0, g, tg, frr, kb, 0, cmx, smx, (float)M_PI * g.dx * g.dy2, rule,
                           nr, r32[0], r32[1], r32[2], r32[3], b);
    if (nr == 2) ++n[2];
    else if (nr == 0) ++n[neg_bits((double)frr.q[4]) ? 1 : 0];
    else ++general;
    if (memcmp(a, b, sizeof a) != 0) ++differ;
  }
  printf("%ld %ld %ld %ld %ld\n", n[0], n[1], n[2], general, differ);
}
'''


def _build_run(code):
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        with open(src, "w") as fh:
            fh.write(code)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        return subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()


def _run():
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
        return subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()


def test_single_maximum_hint_and_parity_classification():
    n_one, bad, n_two, worst_angle, arcs, mismatch = _run()
    n_one, bad, n_two, arcs, mismatch = int(n_one), int(bad), int(n_two), int(arcs), int(mismatch)
    # the hint clears most shapes and is never wrong about a single maximum
    assert n_one > 10 * n_two and bad == 0
    # Newton lands on the grid maximum (grid spacing 2 pi / 4096 = 1.5e-3)
    assert float(worst_angle) < 2e-3
    # crossing parity reproduces the direct sign of g on every arc
    assert arcs > 10000 and mismatch == 0


def test_fp32_crossings_against_the_fp64_quartic():
    n, fb, mis, with_roots, worst, t_total, t_fb, t_zero, t_bad = _build_run(SRC_F32)
    n, fb, mis, with_roots = int(n), int(fb), int(mis), int(with_roots)
    t_total, t_fb, t_zero = int(t_total), int(t_fb), int(t_zero)
    # random limb geometries: the FP32 roots stand (fallback rare), with the FP64
    # count, within 1e-4 (1 + |t|) of the FP64 roots (the Newton acceptance bound)
    assert n == 200000 and fb < n // 1000 and mis == 0 and with_roots > n // 2
    assert float(worst) < 1e-4
    # at near-tangency: mostly the FP64 fallback or no crossing (the sliver beyond
    # the limb is then below 1e-10 of the disk); any pair that stands is exact
    assert t_total == 2000 and t_fb + t_zero > 0.99 * t_total and t_fb > 0
    assert int(t_bad) == 0


def test_short_crossing_path_matches_the_general_routine():
    outside, inside, two, general, differ = (int(v) for v in _build_run(SRC_SHORT))
    # every case of the short path is exercised, and it gives the general bits
    assert outside > 100 and inside > 100 and two > 10000
    assert differ == 0
