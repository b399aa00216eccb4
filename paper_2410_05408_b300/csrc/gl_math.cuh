// gl_math.cuh -- device math of the oblate-planet transit path (sm_103a).
//
// Every function is __host__ __device__ so the same arithmetic compiles for the
// GPU kernels; the library only ever runs it on the GPU.
//
// Path per (parameter set, sub-exposure):
//   set_setup      parameter set -> projected ellipse (Sec. 2, Eqs. dx, dy1, dy2 with
//                  b = c, Appendix A), limb-darkening basis, orbit constants and a
//                  conservative transit window                                (FP64)
//   sky_position   Kepler solve E - e sin E = M about the conjunction, sky
//                  coordinates (generalises Sec. 2's circular alpha, beta)     (FP64)
//   occulted       Green's theorem over the ellipse arcs inside the disk and the
//                  limb arcs inside the ellipse (integrands f_flat, f_lin, f_quad
//                  of Sec. 2).  The crossings are the real roots of a quartic
//                  (FP64); f_flat and f_quad have closed forms on every arc;
//                  f_lin is integrated by Gauss-Legendre in s with
//                  theta = m + h sin(pi s / 2), which makes the (1-r^2)^(3/2)
//                  endpoint behaviour smooth (precision R = float or double).
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <limits.h>

#if defined(__CUDACC__)
#define GL_HD __host__ __device__ __forceinline__
#define GL_HD_NOINLINE __host__ __device__ __noinline__
#else
#define GL_HD inline
#define GL_HD_NOINLINE inline
#endif

namespace gl {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxNodes = 48;

enum : int { kSetInvalid = 1, kSetWholeOrbit = 2, kSetTaylor = 4 };

// Per-parameter-set constants, computed once per set in FP64.
struct SetConst {
  // orbit
  double t0, period, nmean;        // days, days, 2 pi / P
  double a_rs, ecc, b_orb;         // a, e, a sqrt(1 - e^2)
  double cosw, sinw, cosi, sini;
  double cosEc, sinEc, rc;         // eccentric anomaly and radius at conjunction
  double tau_lo, tau_hi;           // window of (t - t0) wrapped to [-P/2, P/2) outside
                                   // of which the planet cannot overlap the star
  double elo, ehi;                 // the window widened by half an exposure (exposure test)
  long long elo_key, ehi_key;      // ... as dkey() keys
  double half_p;                   // 0.49 P: |t - t0| below it needs no wrapping
  // sky position from the Kepler offset d = E - E_c (sky_position):
  // r cos(w + nu) = kc1 (cos d - 1) + ks1 sin d, r sin(w + nu) = rc + kc2 (cos d - 1) + ks2 sin d
  double kc1, ks1, kc2, ks2;
  // projected ellipse x = x0 + dx cos th, y = y0 + dy1 cos th + dy2 sin th
  double dx, dy1, dy2, req;
  // limb darkening I = c0 + c1 mu + c2 r^2, F0 = pi (1 - u1/3 - u2/6)
  double c0, c1, c2, invF0;
  double exptime;
  double invP;                     // 1 / P
  double W0;                       // dx dy2
  double sub_step;                 // exptime / nsuper
  // FP32 copies of the shape and LD constants for the FP32C quadrature
  float fdx, fdy1, fdy2, freq, fW0, fc0, fc1, fc2, finvF0, fsub_step;
  // shape terms of g(th) = |p(th)|^2 - 1 (limb_poly): A = A0 - (1 - x0^2 - y0^2),
  // D, E; and their FP32 copies
  double lpA0, lpD, lpE;
  float flpA0, flpD, flpE;
  // conservative FP32 window for the per-exposure test (see window_maybe)
  float t0f, Pf, invPf, wlo_f, whi_f, slack_f;
  int nsuper;
  int flags;
  int rule_min;    // least FP32 quadrature order for this shape (index: 16, 20, 24, 28 nodes)
  // body: semi-axes (a along x', b along y', c along z') and the rows of
  // R(zeta, eta, xi), for projections that change along the orbit (tidal locking)
  double ax[3], rot[9];
  // Kepler solve about the conjunction (set_kepler): e cos E_c, e sin E_c and the
  // largest accepted Newton step; FP32 copies of the orbit for the FP32 stages
  double kep_ec, kep_es, kep_smax;
  float kf_ec, kf_es, kf_ir1;          // e cos E_c, e sin E_c, 1 / (1 - e cos E_c)
  float kf_a, kf_bo, kf_e, kf_nm;      // a, a sqrt(1 - e^2), e, n
  float kf_cEc, kf_sEc, kf_cw, kf_sw, kf_ci, kf_si;
};

// Mapped Gauss-Legendre rule on s in [-1, 1] with theta = m + h sin(pi s / 2):
// sig[j] = sin(pi s_j / 2), wt[j] = w_j (pi / 2) cos(pi s_j / 2); for the
// full-turn rule (h = pi) cph/sph hold cos, sin of pi sig[j].
template <typename R>
struct NodeRule {
  int n;
  R sig[kMaxNodes], wt[kMaxNodes], cph[kMaxNodes], sph[kMaxNodes];
};

// ------------------------------------------------------------------ scalar helpers
GL_HD double dsq(double x) { return x * x; }

template <typename R> GL_HD R rsqrt_(R x);
template <> GL_HD double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }
template <> GL_HD float rsqrt_<float>(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
template <typename R> GL_HD R rcp_(R x);
template <> GL_HD double rcp_<double>(double x) { return 1.0 / x; }
template <> GL_HD float rcp_<float>(float x) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
template <typename R> GL_HD void sincos_(R x, R* s, R* c);
template <> GL_HD void sincos_<double>(double x, double* s, double* c) {
#if defined(__CUDA_ARCH__)
  sincos(x, s, c);
#else
  *s = ::sin(x);
  *c = ::cos(x);
#endif
}
template <> GL_HD void sincos_<float>(float x, float* s, float* c) {
#if defined(__CUDA_ARCH__)
  sincosf(x, s, c);   // |x| <= pi here: the accurate version stays on its fast path
#else
  *s = ::sinf(x);
  *c = ::cosf(x);
#endif
}

// sin(pi x) and cos(pi x).
template <typename R> GL_HD void sincospi_(R x, R* s, R* c);
template <> GL_HD void sincospi_<double>(double x, double* s, double* c) {
#if defined(__CUDA_ARCH__)
  sincospi(x, s, c);
#else
  *s = ::sin(kPi * x);
  *c = ::cos(kPi * x);
#endif
}
template <> GL_HD void sincospi_<float>(float x, float* s, float* c) {
#if defined(__CUDA_ARCH__)
  sincospif(x, s, c);
#else
  *s = ::sinf(3.14159265358979f * x);
  *c = ::cosf(3.14159265358979f * x);
#endif
}

// Neumaier-compensated accumulation.
template <typename R>
struct CSum {
  R s = 0, c = 0;
  GL_HD void add(R x) {
    R t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  GL_HD R value() const { return s + c; }
};

// The double or the float copy of a constant, by quadrature precision.
template <typename R> GL_HD R pick(double d, float f);
template <> GL_HD double pick<double>(double d, float) { return d; }
template <> GL_HD float pick<float>(double, float f) { return f; }

// Reciprocal: hardware approximation refined by Newton steps (full precision
// after two; used where a divide would cost a long FP64 sequence).
// Bit patterns of doubles (host and device).
GL_HD unsigned long long dbits(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
GL_HD double dfrombits(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}
// |x| <= m for a finite m >= 0, by the ordering of the bit patterns of
// non-negative doubles (no FP64 instruction); false for NaN.
GL_HD bool abs_le(double x, double m) { return (dbits(x) & 0x7fffffffffffffffull) <= dbits(m); }
// |x| < m likewise
GL_HD bool abs_lt(double x, double m) { return (dbits(x) & 0x7fffffffffffffffull) < dbits(m); }
// isfinite from the exponent bits
GL_HD bool finite_bits(double x) { return ((dbits(x) >> 52) & 0x7ffu) != 0x7ffu; }
// A key that orders doubles like their values (signed integer compare; -0 sorts
// just below +0; a NaN sorts by its sign bit: above +infinity when the bit is
// clear, below -infinity when it is set)
GL_HD long long dkey(double x) {
  const long long b = (long long)dbits(x);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
// x < 0 (below -0) by its key; for a NaN, whether its sign bit is set
GL_HD bool neg_bits(double x) { return dkey(x) < -1; }

GL_HD double rcp64(double x) {
#if defined(__CUDA_ARCH__)
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
#else
  return 1.0 / x;
#endif
}

// sin(d) and cos(d) - 1 for the Kepler update.  Small |d|: Taylor series in d^2
// (coefficients 1/n!, truncation below 1e-21 for |d| < 1/4); otherwise sincos.
GL_HD void sin_cosm1(double d, double* sd, double* cm1) {
  if (abs_lt(d, 0.02)) {   // (integer compares: no FP64 instruction)
    // truncation below 1e-26 for |d| < 0.02
    double d2 = d * d;
    double s = -1.0 / 5040.0;
    s = s * d2 + 1.0 / 120.0;
    s = s * d2 - 1.0 / 6.0;
    *sd = d + d * d2 * s;
    double c = 1.0 / 40320.0;
    c = c * d2 - 1.0 / 720.0;
    c = c * d2 + 1.0 / 24.0;
    c = c * d2 - 0.5;
    *cm1 = d2 * c;
  } else if (abs_lt(d, 0.25)) {
    double d2 = d * d;
    double s = 1.0 / 6227020800.0;
    s = s * d2 - 1.0 / 39916800.0;
    s = s * d2 + 1.0 / 362880.0;
    s = s * d2 - 1.0 / 5040.0;
    s = s * d2 + 1.0 / 120.0;
    s = s * d2 - 1.0 / 6.0;
    *sd = d + d * d2 * s;
    double c = -1.0 / 87178291200.0;
    c = c * d2 + 1.0 / 479001600.0;
    c = c * d2 - 1.0 / 3628800.0;
    c = c * d2 + 1.0 / 40320.0;
    c = c * d2 - 1.0 / 720.0;
    c = c * d2 + 1.0 / 24.0;
    c = c * d2 - 0.5;
    *cm1 = d2 * c;
  } else {
    double s, c;
    sincos_<double>(d, &s, &c);
    *sd = s;
    *cm1 = c - 1.0;
  }
}

// ------------------------------------------------------------------ set setup
// Eccentric anomaly from true anomaly.
GL_HD double ecc_anomaly_from_true(double nu, double e) {
  return 2.0 * atan2(sqrt(1.0 - e) * sin(0.5 * nu), sqrt(1.0 + e) * cos(0.5 * nu));
}

// sin x and cos x in FP64 for the per-set constants, with a short dependent
// chain: Cody-Waite reduction by pi/2 (x = k pi/2 + r, pi/2 split in a 33-bit
// head, so that k * head is exact for |k| < 2^20, and a tail), then the Taylor
// series of sin r and cos r on |r| <= pi/4 (terms through r^19 and r^18: the
// first omitted term is below 1e-19) and the quadrant of k.  Beyond |x| = 1e5
// the library sincos is used.
// (the library sincos for the rare large argument, compiled once rather than
// inlined at every call site: the constants kernel runs with cold caches)
GL_HD_NOINLINE void sincos_large(double x, double* s, double* c) { sincos_<double>(x, s, c); }

GL_HD void sincos_setup(double x, double* s, double* c) {
  if (!(fabs(x) <= 1e5)) {
    sincos_large(x, s, c);
    return;
  }
  const double two_over_pi = 0.63661977236758134308;
  const double half_pi_hi = 1.5707963267341256142;     // pi/2 to 33 bits
  const double half_pi_lo = 6.0771005065061922e-11;    // pi/2 - half_pi_hi
  const double kq = rint(x * two_over_pi);
  const double r = (x - kq * half_pi_hi) - kq * half_pi_lo;
  const double r2 = r * r;
  // sin r = r (1 - r^2/3! + r^4/5! - ...), cos r = 1 - r^2/2! + r^4/4! - ...
  double ps = -1.0 / 121645100408832000.0;   // -1/19!
  ps = ps * r2 + 1.0 / 355687428096000.0;    // 1/17!
  ps = ps * r2 - 1.0 / 1307674368000.0;      // 1/15!
  ps = ps * r2 + 1.0 / 6227020800.0;         // 1/13!
  ps = ps * r2 - 1.0 / 39916800.0;           // 1/11!
  ps = ps * r2 + 1.0 / 362880.0;             // 1/9!
  ps = ps * r2 - 1.0 / 5040.0;               // 1/7!
  ps = ps * r2 + 1.0 / 120.0;                // 1/5!
  ps = ps * r2 - 1.0 / 6.0;                  // 1/3!
  const double sr = r + r * r2 * ps;
  double pc = 1.0 / 6402373705728000.0;      // 1/18!
  pc = pc * r2 - 1.0 / 20922789888000.0;     // 1/16!
  pc = pc * r2 + 1.0 / 87178291200.0;        // 1/14!
  pc = pc * r2 - 1.0 / 479001600.0;          // 1/12!
  pc = pc * r2 + 1.0 / 3628800.0;            // 1/10!
  pc = pc * r2 - 1.0 / 40320.0;              // 1/8!
  pc = pc * r2 + 1.0 / 720.0;                // 1/6!
  pc = pc * r2 - 1.0 / 24.0;                 // 1/4!
  pc = pc * r2 + 0.5;                        // 1/2!
  const double cr = 1.0 - r2 * pc;
  const int q = (int)((long long)kq & 3);
  *s = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
  *c = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
}

// Cube root of a > 0 in FP64: FP32 estimate and one Halley step
// y <- y (y^3 + 2a) / (2 y^3 + a), which triples the number of correct digits.
GL_HD_NOINLINE double cbrt_large(double a) { return cbrt(a); }

GL_HD double cbrt_setup(double a) {
  if (!(a > 1e-30 && a < 1e30)) return cbrt_large(a);
  const double y = (double)cbrtf((float)a);
  const double y3 = y * y * y;
  return y * (y3 + 2.0 * a) * rcp64(2.0 * y3 + a);
}

// The per-set constants in four parts with no dependence on one another
// beyond the transcendentals (sin w, cos w, cbrt(1 - f), cos eta, sin xi,
// cos xi), so that a caller may compute the parts in parallel.  Each part
// writes its own fields of c; set_setup_trig runs all four.

// Physical validity of a set (the orbit part also checks |cos i| <= 1).
GL_HD bool set_valid(double t0, double period, double a_rs, double b, double ecc, double omega,
                     double k, double f, double eta, double xi, double u1, double u2,
                     double exptime, int nsuper) {
  bool ok = isfinite(t0) && isfinite(period) && isfinite(a_rs) && isfinite(b) &&
            isfinite(ecc) && isfinite(omega) && isfinite(k) && isfinite(f) &&
            isfinite(eta) && isfinite(xi) && isfinite(u1) && isfinite(u2) &&
            isfinite(exptime) && period > 0.0 && a_rs > 0.0 && ecc >= 0.0 && ecc < 1.0 &&
            k > 0.0 && f >= 0.0 && f < 1.0 && exptime >= 0.0 && nsuper >= 1;
  return ok && kPi * (1.0 - u1 * (1.0 / 3.0) - u2 * (1.0 / 6.0)) > 0.0;
}

// Equatorial radius R_eq = k (1 - f)^(-1/3) (k the mean radius, Appendix A).
GL_HD double set_req(double k, double cbrt1mf) { return k * rcp64(cbrt1mf); }

// Quantities that follow from (dx, dy1, dy2): W0 = dx dy2, the shape terms of
// g(th) and the FP32 copies.
GL_HD void finish_shape(SetConst* c) {
  c->W0 = c->dx * c->dy2;
  c->lpA0 = 0.5 * (c->dx * c->dx + c->dy1 * c->dy1 + c->dy2 * c->dy2);
  c->lpD = 0.5 * (c->dx * c->dx + c->dy1 * c->dy1 - c->dy2 * c->dy2);
  c->lpE = c->dy1 * c->dy2;
  c->fdx = (float)c->dx;
  c->fdy1 = (float)c->dy1;
  c->fdy2 = (float)c->dy2;
  c->fW0 = (float)c->W0;
  c->flpA0 = (float)c->lpA0;
  c->flpD = (float)c->lpD;
  c->flpE = (float)c->lpE;
}

// Projected ellipse of the oblate spheroid (b = c = R_eq, a = R_pol along the
// spin axis n = first row of R(zeta, eta, xi) = (cos eta cos xi, -cos eta sin xi,
// sin eta)).  The sky covariance S = R^T diag(a^2,b^2,c^2) R restricted to (x, y)
// is R_eq^2 I - (R_eq^2 - R_pol^2) n_xy n_xy^T, and (dx, dy1, dy2) of Eqs. dx,
// dy1, dy2 are its Cholesky factor.  Also the least FP32 quadrature order.
GL_HD void set_shape(double k, double f, double cbrt1mf, double ce, double sx, double cx,
                     SetConst* c) {
  double req = set_req(k, cbrt1mf);
  // Least FP32 quadrature order for this shape.  Measured per-evaluation errors
  // of the FP32 path against the FP64 one (random positions on and around the
  // disk, random orientations, f < 0.9) stay below 1e-7 with 16 nodes for
  // R_eq < 0.2 at any f and for f < 0.5 at any R_eq below 0.45; R_eq >= 0.2
  // needs 20 nodes for f in [0.5, 0.7) and 28 beyond; R_eq >= 0.45 (outside the
  // measured range) always takes 28.  A raised order (rule_min > 0) also moves
  // the FP64 path from 32 to 48 nodes.
  c->rule_min = req >= 0.45 ? 3 : (req < 0.2 || f < 0.5) ? 0 : (f < 0.7 ? 1 : 3);
  double delta = req * req * f * (2.0 - f) * ce * ce;   // R_eq^2 - R_pol^2 times cos^2 eta
  double sxx = req * req - delta * cx * cx;
  double sxy = delta * cx * sx;
  double dx = sqrt(sxx);
  double idx = rcp64(dx);
  c->dx = dx;
  c->dy1 = sxy * idx;
  c->dy2 = req * sqrt(req * req - delta) * idx;
  c->req = req;
  c->freq = (float)req;
  finish_shape(c);
}

// Projected ellipse of a general triaxial ellipsoid (Sec. 2, Eqs. dx, dy1, dy2
// with R = Rx(zeta) Ry(eta) Rz(xi), all three angles active): semi-axes c (the
// largest), b = c (1 - g), a = c (1 - f), with c = k ((1 - f)(1 - g))^(-1/3) given
// as c = k / cbrt_fg.  R_eq (the classification radius) is c; the least
// quadrature order uses the larger of f and g.
GL_HD void set_shape_triaxial(double k, double f, double g, double cbrt_fg, double sz,
                              double cz, double se, double ce, double sx, double cx,
                              SetConst* c) {
  const double cax = k * rcp64(cbrt_fg);
  const double a = cax * (1.0 - f), b = cax * (1.0 - g);
  // rows of Rx(zeta) Ry(eta) Rz(xi)
  const double r1 = ce * cx, r2 = -ce * sx, r3 = se;
  const double r4 = cz * sx + sz * se * cx, r5 = cz * cx - sz * se * sx, r6 = -sz * ce;
  const double r7 = sz * sx - cz * se * cx, r8 = sz * cx + cz * se * sx, r9 = cz * ce;
  const double a2 = a * a, b2 = b * b, c2 = cax * cax;
  const double dx = sqrt(a2 * r1 * r1 + b2 * r4 * r4 + c2 * r7 * r7);
  const double idx = rcp64(dx);
  c->dx = dx;
  c->dy1 = (a2 * r1 * r2 + b2 * r4 * r5 + c2 * r7 * r8) * idx;
  c->dy2 = sqrt(a2 * b2 * r9 * r9 + a2 * c2 * r6 * r6 + b2 * c2 * r3 * r3) * idx;
  c->req = cax;
  const double fe = f > g ? f : g;
  c->rule_min = cax >= 0.45 ? 3 : (cax < 0.2 || fe < 0.5) ? 0 : (fe < 0.7 ? 1 : 3);
  c->freq = (float)cax;
  finish_shape(c);
}

// Body semi-axes and the rows of R(zeta, eta, xi) = Rx(zeta) Ry(eta) Rz(xi).
GL_HD void set_body(double a, double b, double cax, double sz, double cz, double se, double ce,
                    double sx, double cx, SetConst* c) {
  c->ax[0] = a;
  c->ax[1] = b;
  c->ax[2] = cax;
  c->rot[0] = ce * cx;
  c->rot[1] = -ce * sx;
  c->rot[2] = se;
  c->rot[3] = cz * sx + sz * se * cx;
  c->rot[4] = cz * cx - sz * se * sx;
  c->rot[5] = -sz * ce;
  c->rot[6] = sz * sx - cz * se * cx;
  c->rot[7] = sz * cx + cz * se * sx;
  c->rot[8] = cz * ce;
}

// Projected ellipse of a tidally locked body (Appendix B) at the orbital angle
// alpha from conjunction (cos, sin given) with beta = pi/2 - i: the body frame is
// x' = R (Rx(-alpha) Ry(beta) x + (0, 0, d)), so with M = R Rx(-alpha) Ry(beta)
// and D = diag(a^2, b^2, c^2) the sky covariance is M^T D M restricted to (x, y):
// dx = sqrt(sum_k D_k M_k1^2), dy1 = sum_k D_k M_k1 M_k2 / dx and
// dy2 = sqrt(D_a D_b M_33^2 + D_a D_c M_23^2 + D_b D_c M_13^2) / dx (a rotation's
// cofactors are its elements) -- the paper's Eqs. dx-locked, dy1-locked,
// dy2-locked in matrix form.  `out` gets a copy of c with the new shape.
GL_HD void locked_shape(const SetConst& c, double ca, double sa, SetConst* out) {
  *out = c;
  const double sb = c.cosi, cb = c.sini;   // beta = pi/2 - i
  // Q = Rx(-alpha) Ry(beta)
  const double q[9] = {cb, 0.0, sb, -sa * sb, ca, sa * cb, -ca * sb, -sa, ca * cb};
  double M[9];
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      M[3 * k + j] = c.rot[3 * k] * q[j] + c.rot[3 * k + 1] * q[3 + j] + c.rot[3 * k + 2] * q[6 + j];
  const double D0 = c.ax[0] * c.ax[0], D1 = c.ax[1] * c.ax[1], D2 = c.ax[2] * c.ax[2];
  const double dx = sqrt(D0 * M[0] * M[0] + D1 * M[3] * M[3] + D2 * M[6] * M[6]);
  const double idx = rcp64(dx);
  out->dx = dx;
  out->dy1 = (D0 * M[0] * M[1] + D1 * M[3] * M[4] + D2 * M[6] * M[7]) * idx;
  out->dy2 = sqrt(D0 * D1 * M[8] * M[8] + D0 * D2 * M[5] * M[5] + D1 * D2 * M[2] * M[2]) * idx;
  finish_shape(out);
}

// Limb darkening in the basis (1, mu, r^2): I = c0 + c1 mu + c2 r^2 with
// F0 = pi (1 - u1/3 - u2/6).
GL_HD void set_ld(double u1, double u2, SetConst* c) {
  c->c0 = 1.0 - u1 - 2.0 * u2;
  c->c1 = u1 + 2.0 * u2;
  c->c2 = u2;
  c->invF0 = rcp64(kPi * (1.0 - u1 * (1.0 / 3.0) - u2 * (1.0 / 6.0)));
  c->fc0 = (float)c->c0;
  c->fc1 = (float)c->c1;
  c->fc2 = (float)c->c2;
  c->finvF0 = (float)c->invF0;
}

// Orbit.  At conjunction nu_c = pi/2 - w: cos nu_c = sin w, sin nu_c = cos w,
// and cos E = (e + cos nu)/(1 + e cos nu), sin E = sqrt(1-e^2) sin nu/(1 + e cos nu),
// r = a (1 - e^2)/(1 + e cos nu).  Returns false when |cos i| > 1.
GL_HD bool set_orbit(double t0, double period, double a_rs, double b, double ecc, double sinw,
                     double cosw, SetConst* c) {
  c->t0 = t0;
  c->period = period;
  double cosi = b * (1.0 + ecc * sinw) * rcp64(a_rs * (1.0 - ecc) * (1.0 + ecc));
  c->invP = rcp64(period);
  c->nmean = 2.0 * kPi * c->invP;
  c->a_rs = a_rs;
  c->ecc = ecc;
  double se = sqrt((1.0 - ecc) * (1.0 + ecc));
  c->b_orb = a_rs * se;
  c->cosw = cosw;
  c->sinw = sinw;
  c->cosi = cosi;
  c->sini = sqrt(fmax(0.0, (1.0 - cosi) * (1.0 + cosi)));
  double iden = rcp64(1.0 + ecc * sinw);
  c->cosEc = (ecc + sinw) * iden;
  c->sinEc = se * cosw * iden;
  c->rc = a_rs * (1.0 - ecc) * (1.0 + ecc) * iden;
  // X = a (cos E - e), Y = a sqrt(1 - e^2) sin E rotated by w, with
  // cos E = cos E_c + cosEc (cos d - 1) - sinEc sin d and
  // sin E = sin E_c + sinEc (cos d - 1) + cosEc sin d
  const double a = a_rs, bo = c->b_orb, ce = c->cosEc, sE = c->sinEc;
  c->kc1 = a * cosw * ce - bo * sinw * sE;
  c->ks1 = -(a * cosw * sE + bo * sinw * ce);
  c->kc2 = a * sinw * ce + bo * cosw * sE;
  c->ks2 = bo * cosw * ce - a * sinw * sE;
  c->half_p = 0.49 * period;
  return fabs(cosi) <= 1.0;
}

// Constants of the Kepler solve about the conjunction (from set_orbit's fields).
// kepler_offset takes Newton steps s = F r with r the reciprocal of F' to a
// relative error below rho = 2^-44 (an FP32 reciprocal refined once in FP64).
// With F' >= 1 - e and |F''| <= e, such a step leaves an error below
// rho |s| + C_N s^2, C_N = e / (2 (1 - e)).  A step is accepted when that bound is
// below 1e-15 and |s| <= 1e-5 (the sin/cos update drops terms of order |s|^3/6);
// kep_smax is the largest such |s|, computed in FP32 and lowered by 10 %.
// (An invalid orbit gives meaningless values here; such sets are never used.)
GL_HD void set_kepler(SetConst* c) {
  const double e = c->ecc;
  c->kep_ec = e * c->cosEc;
  c->kep_es = e * c->sinEc;
  {
    const float ef = (float)e, tol = 1e-15f, rho = 5.684342e-14f;   // 2^-44
    const float cn = ef / (2.0f * (1.0f - ef));
    // positive root of cn s^2 + rho s = tol, in the form without cancellation
    const float sq = 2.0f * tol / (rho + sqrtf(rho * rho + 4.0f * cn * tol));
    c->kep_smax = (double)fminf(0.9f * sq, 1e-5f);
  }
  c->kf_ec = (float)c->kep_ec;
  c->kf_es = (float)c->kep_es;
  c->kf_ir1 = 1.0f / (1.0f - c->kf_ec);
  c->kf_a = (float)c->a_rs;
  c->kf_bo = (float)c->b_orb;
  c->kf_e = (float)e;
  c->kf_nm = (float)c->nmean;
  c->kf_cEc = (float)c->cosEc;
  c->kf_sEc = (float)c->sinEc;
  c->kf_cw = (float)c->cosw;
  c->kf_sw = (float)c->sinw;
  c->kf_ci = (float)c->cosi;
  c->kf_si = (float)c->sini;
}

// Transit window (and its exposure-widened forms); returns the flag
// kSetWholeOrbit.
//  The sky separation is at least r |sin phi| >= a (1-e) |sin phi|, phi = angle
//  from conjunction along the orbit; behind the star (|phi| > pi/2) nothing is
//  occulted.  Outside |phi| <= phi_w the flux is exactly 1.  The window only has
//  to contain every overlapping time, so it is computed in FP32 and widened by a
//  relative 1e-4 plus an absolute 1e-4 days, far more than the FP32 rounding of
//  these few operations.
GL_HD int set_window(double t0, double period, double a_rs, double ecc, double omega,
                     double req, double nmean, double invP, double exptime, int nsuper,
                     SetConst* c) {
  int flags = 0;
  double smax = 1.0 + req * (1.0 + 1e-9) + 1e-9;
  double rmin = a_rs * (1.0 - ecc);
  if (smax >= rmin * (1.0 - 1e-4)) {
    flags |= kSetWholeOrbit;
    c->tau_lo = -period;
    c->tau_hi = period;
  } else {
    // The mean anomaly is a continuous increasing function of the unwrapped true
    // anomaly; across the window it may change by more than pi (eccentric orbits
    // with conjunction near apoapsis), so no wrapping is applied.
    float phw = asinf((float)(smax / rmin)) * 1.0001f;
    float ef = (float)ecc;
    double nuc = 0.5 * kPi - omega;   // true anomaly at conjunction, reduced to [-pi, pi]
    float nucf = (float)(nuc - 2.0 * kPi * rint(nuc * (0.5 / kPi)));
    float sq1 = sqrtf(1.0f - ef), sq2 = sqrtf(1.0f + ef);
    auto mean_anomaly = [&](float nu) {
      float turns = rintf(nu * 0.15915494309189535f);
      float nu0 = nu - 6.283185307179586f * turns;
      float E = 2.0f * atan2f(sq1 * sinf(0.5f * nu0), sq2 * cosf(0.5f * nu0)) +
                6.283185307179586f * turns;
      return E - ef * sinf(E);
    };
    // the mean anomaly at the conjunction and at both ends, in one loop (the
    // function's code is fetched once, not three inlined copies)
    float Mk[3];
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
      const float nu = q == 0 ? nucf : nucf + (q == 2 ? phw : -phw);
      const float m = mean_anomaly(nu);
      Mk[0] = q == 0 ? m : Mk[0];
      Mk[1] = q == 1 ? m : Mk[1];
      Mk[2] = q == 2 ? m : Mk[2];
    }
    const float Mcf = Mk[0];
    float taus[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      float dM = (sgn ? Mk[2] : Mk[1]) - Mcf;
      taus[sgn] = dM / (float)nmean;
    }
    double margin = 1e-4 * (fabs((double)taus[0]) + fabs((double)taus[1])) + 1e-4;
    c->tau_lo = fmin((double)taus[0], 0.0) - margin;
    c->tau_hi = fmax((double)taus[1], 0.0) + margin;
  }
  c->elo = c->tau_lo - 0.5 * exptime;
  c->ehi = c->tau_hi + 0.5 * exptime;
  c->elo_key = dkey(c->elo);
  c->ehi_key = dkey(c->ehi);
  // FP32 copy of the window for the per-exposure test (set_exposure holds the
  // rest of it)
  c->wlo_f = (float)(c->tau_lo - 0.5 * exptime);
  c->whi_f = (float)(c->tau_hi + 0.5 * exptime);
  return flags;
}

// Exposure fields, the rest of the FP32 window test's constants and the
// sub-exposure expansion flag (independent of the window, so that another part
// of the constants kernel can form them); returns the flag kSetTaylor.
GL_HD int set_exposure(double t0, double period, double a_rs, double ecc, double nmean,
                       double invP, double exptime, int nsuper, SetConst* c) {
  int flags = 0;
  c->exptime = exptime;
  c->nsuper = nsuper;
  c->sub_step = exptime / nsuper;
  c->fsub_step = (float)c->sub_step;
  // FP32 copy of the window for the per-exposure test, widened for rounding:
  // every FP32 operation of window_maybe errs by at most 2^-24 of its operands.
  c->t0f = (float)t0;
  c->Pf = (float)period;
  c->invPf = (float)invP;
  c->slack_f = (float)(ldexp(fabs(t0) + period, -20) + 1e-6);
  // Sub-exposure positions may come from a cubic Taylor expansion about the
  // exposure midpoint.  For a Kepler orbit |d^4 r/dt^4| <= C n^4 a (2+e)/(1-e)^5
  // (from r'' = -mu r/|r|^3, mu = n^2 a^3, r >= a(1-e)); with C = 60 the
  // truncation over half an exposure must stay below 1e-10 stellar radii.
  // (The bound is only compared with 1e-10, so FP32 serves: its rounding can
  // move the decision only for a set within 1e-6 of the threshold, whose
  // truncation stays within 1e-10 either way.)
  {
    const float n = (float)nmean, h = 0.5f * (float)exptime;
    const float e = (float)ecc, om = 1.0f - e;
    const float n2 = n * n, h2 = h * h, om2 = om * om;
    const float bound = 2.5f * (n2 * n2) * (float)a_rs * (2.0f + e) * (h2 * h2) /
                        (om2 * om2 * om);   // 60 / 24 = 2.5
    if (bound <= 1e-10f) flags |= kSetTaylor;
  }
  return flags;
}

// Parameters of one set -> constants, given the transcendentals of the set
// (so that a caller can compute them in parallel): sin w, cos w, cbrt(1 - f),
// cos eta, sin xi, cos xi.  Returns false (and sets kSetInvalid) when the set
// is physically invalid.
GL_HD bool set_setup_trig(double t0, double period, double a_rs, double b, double ecc,
                          double omega, double k, double f, double eta, double xi, double u1,
                          double u2, double exptime, int nsuper, double sinw, double cosw,
                          double cbrt1mf, double ce, double sx, double cx, SetConst* c) {
  c->flags = 0;
  c->rule_min = 0;
  c->t0 = t0;
  c->period = period;
  c->exptime = exptime;
  c->nsuper = nsuper;
  if (!set_valid(t0, period, a_rs, b, ecc, omega, k, f, eta, xi, u1, u2, exptime, nsuper) ||
      !set_orbit(t0, period, a_rs, b, ecc, sinw, cosw, c)) {
    c->flags = kSetInvalid;
    return false;
  }
  set_kepler(c);
  set_shape(k, f, cbrt1mf, ce, sx, cx, c);
  set_ld(u1, u2, c);
  c->flags = set_window(t0, period, a_rs, ecc, omega, c->req, c->nmean, c->invP, exptime, nsuper,
                        c) |
             set_exposure(t0, period, a_rs, ecc, c->nmean, c->invP, exptime, nsuper, c);
  return true;
}

GL_HD bool set_setup(double t0, double period, double a_rs, double b, double ecc,
                     double omega, double k, double f, double eta, double xi, double u1,
                     double u2, double exptime, int nsuper, SetConst* c) {
  double sw = 0.0, cw = 1.0, sx = 0.0, cx = 1.0, ce = 1.0, cb = 1.0, se = 0.0;
  if (isfinite(omega)) sincos_setup(omega, &sw, &cw);
  if (isfinite(xi)) sincos_setup(xi, &sx, &cx);
  if (isfinite(eta)) sincos_setup(eta, &se, &ce);
  if (isfinite(f) && f < 1.0) cb = cbrt_setup(1.0 - f);
  const bool ok = set_setup_trig(t0, period, a_rs, b, ecc, omega, k, f, eta, xi, u1, u2, exptime,
                                 nsuper, sw, cw, cb, ce, sx, cx, c);
  if (ok) set_body(c->req * (1.0 - f), c->req, c->req, 0.0, 1.0, se, ce, sx, cx, c);
  return ok;
}

// (t - t0) wrapped to one period around the conjunction.
GL_HD double wrap_tau(const SetConst& c, double t) {
  double tau = t - c.t0;
  if (abs_le(tau, c.half_p)) return tau;   // rint(tau / P) = 0: the same value
  return tau - c.period * rint(tau * c.invP);
}

// FP32 window constants of a set for the per-exposure test (window_maybe), in a
// form a thread can keep in registers while its exposures stay in one set.
struct WinTest {
  float t0f, Pf, invPf, wlo_f, whi_f, slack_f;
  int flags;
};
GL_HD WinTest win_test(const SetConst& c) {
  return WinTest{c.t0f, c.Pf, c.invPf, c.wlo_f, c.whi_f, c.slack_f, c.flags};
}

// FP64 -> FP32 rounded to nearest-even with integer operations only (on B300 an
// FP64 conversion instruction holds the FP64 unit like any FP64 operation).
// Normal results equal the hardware conversion; magnitudes below 2^-126 give a
// signed zero instead of a subnormal; infinities and NaN are kept.
GL_HD float f64_to_f32_int(double x) {
  const unsigned long long b = dbits(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int fe = e - 1023 + 127;
  unsigned r;
  if (e == 0x7ff) {
    r = (b << 12) ? 0x7fc00000u : 0x7f800000u;
  } else if (fe >= 255) {
    r = 0x7f800000u;
  } else if (fe <= 0) {
    r = 0u;
  } else {
    r = ((unsigned)fe << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;   // the 29 dropped bits
    r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;
  }
  const unsigned bits = sign | r;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(bits);
#else
  float f;
  memcpy(&f, &bits, sizeof f);
  return f;
#endif
}

// FP32 -> FP64 with integer operations only: exact for normal numbers, zeros,
// infinities and NaN; FP32 subnormals (below 2^-126) give a signed zero.
GL_HD double f32_to_f64_int(float f) {
#if defined(__CUDA_ARCH__)
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, sizeof u);
#endif
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long r;
  if (e == 0) r = 0;
  else if (e == 0xff) r = (0x7ffull << 52) | ((unsigned long long)m << 29);
  else r = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  return dfrombits(sign | r);
}
// Precision changes without FP64 conversion instructions (identity for double).
GL_HD double to_f64(float x) { return f32_to_f64_int(x); }
GL_HD double to_f64(double x) { return x; }
template <typename R> GL_HD R from_f64(double x);
template <> GL_HD float from_f64<float>(double x) { return f64_to_f32_int(x); }
template <> GL_HD double from_f64<double>(double x) { return x; }

// Conservative FP32 window test of an exposure at time t (true whenever any
// sub-exposure may overlap the star; false positives are resolved in FP64).
GL_HD bool window_maybe(const WinTest& w, double t) {
  if (w.flags & kSetWholeOrbit) return true;
  float tf = f64_to_f32_int(t);
  float tau = tf - w.t0f;
  float ep = rintf(tau * w.invPf);
  float tw = fmaf(-ep, w.Pf, tau);
  float m = (fabsf(tf) + fabsf(w.t0f)) * 4.76837158203125e-07f + w.slack_f;   // 2^-21
  return tw >= w.wlo_f - m && tw <= w.whi_f + m;
}
GL_HD bool window_maybe(const SetConst& c, double t) { return window_maybe(win_test(c), t); }

// Window test of a whole exposure centred at tau (any of its sub-exposures may
// overlap the star).
GL_HD bool exposure_in_window(const SetConst& c, double tau) {
  if (c.flags & kSetWholeOrbit) return true;
  const long long k = dkey(tau);   // (integer compares: no FP64 instruction)
  return k >= c.elo_key && k <= c.ehi_key;
}

GL_HD bool in_window(const SetConst& c, double tau, double halfwidth) {
  if (c.flags & kSetWholeOrbit) return true;
  return tau + halfwidth >= c.tau_lo && tau - halfwidth <= c.tau_hi;
}

// ------------------------------------------------------------------ orbit
// sin(d) and cos(d) - 1 in FP32 (Taylor series below |d| = 1/4: truncation
// below 1e-11; sincosf beyond).
GL_HD void sin_cosm1_f(float d, float* sd, float* cm1) {
  if (fabsf(d) < 0.25f) {
    float d2 = d * d;
    *sd = d + d * d2 * (-1.0f / 6.0f + d2 * (1.0f / 120.0f + d2 * (-1.0f / 5040.0f)));
    *cm1 = d2 * (-0.5f + d2 * (1.0f / 24.0f + d2 * (-1.0f / 720.0f + d2 * (1.0f / 40320.0f))));
  } else {
    float s, c;
    sincos_<float>(d, &s, &c);
    *sd = s;
    *cm1 = c - 1.0f;
  }
}

// Kepler's equation for the eccentric anomaly E = E_c + d about the
// conjunction:  d - e [cos E_c sin d + sin E_c (cos d - 1)] = n tau.
// Newton's method in FP32 first (cheap), then Newton's method in FP64 from the
// FP32 iterate: the residual F in FP64, the reciprocal of F' from FP32 refined by
// one FP64 step (set_kepler bounds the error after a step s and accepts the step
// when |s| <= kep_smax -- one step from a converged FP32 iterate, |s| ~ 1e-7 |d|).
// sin d and cos d - 1 of the final iterate follow from those of the last
// evaluated one by the angle-difference formulas to second order in s.  A
// bisection on the bracket |E - M| <= e backs up an iteration that does not
// settle.  The FP32 <-> FP64 conversions are integer operations (on B300 an FP64
// conversion holds the FP64 unit like an FP64 operation).  Returns sin d and
// cos d - 1.
// Bisection on the bracket |E - M| <= e for Kepler's equation about the
// conjunction (the backup of kepler_offset's Newton steps; compiled once).
GL_HD_NOINLINE void kepler_bisect(const SetConst& c, double nt, double* sd_out, double* cm1_out) {
  const double ec = c.kep_ec, es = c.kep_es;
  double sd, cm1;
  double Ec = atan2(c.sinEc, c.cosEc);
  double M = Ec - c.ecc * c.sinEc + nt;
  double lo = M - c.ecc - Ec, hi = M + c.ecc - Ec;
  for (int it = 0; it < 200 && hi - lo > 1e-16 * (1.0 + fabs(lo)); ++it) {
    double mid = 0.5 * (lo + hi);
    sin_cosm1(mid, &sd, &cm1);
    double F = mid - ec * sd - es * cm1 - nt;
    if (F > 0.0) hi = mid; else lo = mid;
  }
  sin_cosm1(0.5 * (lo + hi), sd_out, cm1_out);
}

GL_HD void kepler_offset(const SetConst& c, double tau, double* sd_out, double* cm1_out) {
  const double nt = c.nmean * tau;
  const double ec = c.kep_ec, es = c.kep_es;
  const float ntf = f64_to_f32_int(nt), ecf = c.kf_ec, esf = c.kf_es;
  const float ir1f = c.kf_ir1;
  float df = ntf * ir1f;
  df -= 0.5f * esf * df * df * ir1f;   // second-order start: F ~ d (1 - ec) + es d^2 / 2 - n tau
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    float sdf, cmf;
    sin_cosm1_f(df, &sdf, &cmf);
    const float F = df - ecf * sdf - esf * cmf - ntf;
    const float Fp = 1.0f - ecf * (1.0f + cmf) + esf * sdf;
    df -= F / Fp;
  }
  const double smax = c.kep_smax;
  double d = isfinite(df) ? f32_to_f64_int(df) : nt;   // (FP32 test)
  double sd, cm1;
  for (int it = 0; it < 12; ++it) {
    sin_cosm1(d, &sd, &cm1);
    const double cp = 1.0 + cm1;
    const double F = d - ec * sd - es * cm1 - nt;
    const double Fp = 1.0 - ec * cp + es * sd;
    const double r0 = f32_to_f64_int(rcp_<float>(f64_to_f32_int(Fp)));
    const double er = fma(-Fp, r0, 1.0);       // 1 - F' r0
    const double sr = F * r0;
    const double step = fma(sr, er, sr);       // F / F' to a relative 2^-44
    d -= step;
    if (!abs_le(step, smax)) continue;         // (NaN continues to the bisection)
    if (!finite_bits(d)) break;
    // sin(d - s), cos(d - s) - 1 from sin d, cos d - 1 of the previous iterate
    const double hs2 = 0.5 * step * step;
    *sd_out = sd - step * cp - hs2 * sd;
    *cm1_out = cm1 + step * sd - hs2 * cp;
    return;
  }
  kepler_bisect(c, nt, sd_out, cm1_out);
}

// Sky position at time offset tau from conjunction.  The sky coordinates are
// formed from differences to the conjunction point, where r cos(w + nu) = 0 and
// r sin(w + nu) = r_c, so no large terms cancel.
GL_HD void sky_position(const SetConst& c, double tau, double* x0, double* y0, double* z) {
  double sd, cm1;
  kepler_offset(c, tau, &sd, &cm1);
  const double p1 = fma(cm1, c.kc1, sd * c.ks1);           // r cos(w + nu)  (0 at conjunction)
  const double p2 = fma(sd, c.ks2, fma(cm1, c.kc2, c.rc));  // r sin(w + nu)  (r_c at conjunction)
  *y0 = -p1;
  *x0 = p2 * c.cosi;
  *z = -p2 * c.sini;
}


// ------------------------------------------------------------------ precision helpers
GL_HD double m_sqrt(double x) { return sqrt(x); }
GL_HD float m_sqrt(float x) { return sqrtf(x); }
GL_HD double m_cbrt(double x) { return cbrt(x); }
GL_HD float m_cbrt(float x) { return cbrtf(x); }
GL_HD double m_acos(double x) { return acos(x); }
GL_HD float m_acos(float x) { return acosf(x); }
GL_HD double m_cos(double x) { return cos(x); }
GL_HD float m_cos(float x) { return cosf(x); }
GL_HD double m_atan2(double y, double x) { return atan2(y, x); }
GL_HD float m_atan2(float y, float x) { return atan2f(y, x); }
GL_HD double m_abs(double x) { return fabs(x); }
GL_HD float m_abs(float x) { return fabsf(x); }
GL_HD double m_copysign(double a, double b) { return copysign(a, b); }
GL_HD float m_copysign(float a, float b) { return copysignf(a, b); }
GL_HD bool m_finite(double x) { return isfinite(x); }
GL_HD bool m_finite(float x) { return isfinite(x); }
template <typename T> GL_HD T m_eps();
template <> GL_HD double m_eps<double>() { return 2.220446049250313e-16; }
template <> GL_HD float m_eps<float>() { return 1.1920929e-07f; }

// ------------------------------------------------------------------ sky geometry
enum : int { kOut = 0, kFull = 1, kPartial = 2 };

// Quick classification from the centre distance alone (R_eq is the largest
// semi-axis of the projection).  kPartial means "decide with the roots".
// `slack` widens the undecided band to cover rounding of the centre.
template <typename T>
GL_HD int classify_t(T req, T x0, T y0, T z, T slack) {
  if (z > T(0)) return kOut;
  T rho = m_sqrt(x0 * x0 + y0 * y0);
  if (rho >= T(1) + req + slack) return kOut;
  if (rho + req <= T(1) - slack) return kFull;
  return kPartial;
}
GL_HD int classify(const SetConst& c, double x0, double y0, double z) {
  return classify_t<double>(c.req, x0, y0, z, 0.0);
}

// Geometry of one evaluation in the quadrature precision R.
template <typename R>
struct Geo {
  R x0, y0, omr2;      // centre, 1 - |centre|^2
  R dx, dy1, dy2;
  R W0, Wc, Ws;        // x y' - y x' = W0 + Wc cos th + Ws sin th
};

// omr2 = 1 - x0^2 - y0^2, supplied by the caller in the best precision it has.
template <typename R>
GL_HD Geo<R> make_geo(const SetConst& c, R x0, R y0, R omr2) {
  Geo<R> g;
  g.x0 = x0;
  g.y0 = y0;
  g.omr2 = omr2;
  g.dx = pick<R>(c.dx, c.fdx);
  g.dy1 = pick<R>(c.dy1, c.fdy1);
  g.dy2 = pick<R>(c.dy2, c.fdy2);
  g.W0 = pick<R>(c.W0, c.fW0);
  g.Wc = x0 * g.dy2;
  g.Ws = y0 * g.dx - x0 * g.dy1;
  return g;
}

// (1 - mu^3) / (3 r^2) written without the r -> 0 cancellation:
// (1 + mu + mu^2) / (3 (1 + mu)), mu = sqrt(1 - r^2).  In FP32 on the GPU the
// square root and the reciprocal are the hardware approximations (about one ulp;
// every node of the f_lin quadrature evaluates this, and the correctly rounded
// forms cost a multi-instruction sequence each).
template <typename R>
GL_HD R lin_kernel(R omr2) {
  const R o = omr2 > R(0) ? omr2 : R(0);
#if defined(__CUDA_ARCH__)
  if constexpr (sizeof(R) == 4) {
    float mu, r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(mu) : "f"(o));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(3.0f + 3.0f * mu));
    return (1.0f + mu + mu * mu) * r;
  }
#endif
  R mu = m_sqrt(o);
  return (R(1) + mu + mu * mu) * rcp_<R>(R(3) + R(3) * mu);
}

// f_lin summand at the point (cos th, sin th) of the boundary:
// (1 - mu^3)/(3 r^2) (x y' - y x').
template <typename R>
GL_HD R lin_point(const Geo<R>& g, R ct, R st) {
  R u = g.dx * ct;
  R v = g.dy1 * ct + g.dy2 * st;
  R omr2 = g.omr2 - R(2) * (g.x0 * u + g.y0 * v) - (u * u + v * v);
  R w = g.W0 + g.Wc * ct + g.Ws * st;
  return lin_kernel<R>(omr2) * w;
}

// Integral of f_lin over the ellipse arc centred at angle m (cos, sin given)
// with half-width h.
template <typename R>
GL_HD R lin_arc(const Geo<R>& g, R cm, R sm, R h, const NodeRule<R>& rule) {
  CSum<R> acc;
  for (int j = 0; j < rule.n; ++j) {
    R sa, ca;
#if defined(__CUDA_ARCH__)
    // FP32: the hardware sine and cosine (absolute error below 4e-7 on [-pi, pi],
    // |h sig| <= pi) place the node; FP64: the library's
    if constexpr (sizeof(R) == 4) __sincosf(h * rule.sig[j], &sa, &ca);
    else sincos_<R>(h * rule.sig[j], &sa, &ca);
#else
    sincos_<R>(h * rule.sig[j], &sa, &ca);
#endif
    R ct = cm * ca - sm * sa;
    R st = sm * ca + cm * sa;
    acc.add(rule.wt[j] * lin_point<R>(g, ct, st));
  }
  return h * acc.value();
}

// Integral of f_lin over the whole ellipse, nodes clustered at th* (the point
// nearest the limb) and at th* + 2 pi: m = th* + pi, h = pi.
template <typename R>
GL_HD R lin_full(const Geo<R>& g, R cs, R ss, const NodeRule<R>& rule) {
  CSum<R> acc;
  for (int j = 0; j < rule.n; ++j) {
    R ct = -(cs * rule.cph[j] - ss * rule.sph[j]);
    R st = -(ss * rule.cph[j] + cs * rule.sph[j]);
    acc.add(rule.wt[j] * lin_point<R>(g, ct, st));
  }
  return R(kPi) * acc.value();
}

// g(th) = |p(th)|^2 - 1 = A + B cos th + C sin th + D cos 2th + E sin 2th.
template <typename T>
struct Trig2 {
  T A, B, C, D, E;
};
// omr2 = 1 - x0^2 - y0^2.
// (A0, D, E depend on the shape only: finish_shape.)
template <typename T>
GL_HD Trig2<T> limb_poly(const SetConst& c, T x0, T y0, T omr2) {
  T dx = pick<T>(c.dx, c.fdx), dy1 = pick<T>(c.dy1, c.fdy1), dy2 = pick<T>(c.dy2, c.fdy2);
  Trig2<T> t;
  t.A = pick<T>(c.lpA0, c.flpA0) - omr2;
  t.B = T(2) * (x0 * dx + y0 * dy1);
  t.C = T(2) * y0 * dy2;
  t.D = pick<T>(c.lpD, c.flpD);
  t.E = pick<T>(c.lpE, c.flpE);
  return t;
}
template <typename T>
GL_HD T trig2_eval(const Trig2<T>& t, T ct, T st) {
  return t.A + t.B * ct + t.C * st + t.D * (ct * ct - st * st) + t.E * (T(2) * st * ct);
}

// Angle of the boundary point nearest the limb (maximum of g): start at the
// point whose outward normal is along the centre direction, then Newton on g'.
template <typename R>
GL_HD void nearest_limb_angle(const Geo<R>& g, const Trig2<R>& t, R* cs, R* ss) {
  R bx = g.dx * g.x0 + g.dy1 * g.y0, by = g.dy2 * g.y0;
  R nrm = m_sqrt(bx * bx + by * by);
  R ct = nrm > R(0) ? bx / nrm : R(1), st = nrm > R(0) ? by / nrm : R(0);
#pragma unroll 1
  for (int it = 0; it < 3; ++it) {
    R c2 = ct * ct - st * st, s2 = R(2) * st * ct;
    R g1 = -t.B * st + t.C * ct - R(2) * t.D * s2 + R(2) * t.E * c2;
    R g2 = -t.B * ct - t.C * st - R(4) * t.D * c2 - R(4) * t.E * s2;
    if (!(g2 < R(0))) break;
    R step = g1 / g2;
    if (step > R(0.5)) step = R(0.5);
    if (step < R(-0.5)) step = R(-0.5);
    R sa, ca;
    if constexpr (sizeof(R) == 4) {
      // |step| <= 1/2: Taylor polynomials of sin (to x^7) and cos (to x^8),
      // truncation below 5e-9, under the FP32 rounding
      const R x = -step, x2 = x * x;
      sa = x * (R(1) - x2 * (R(1.0 / 6.0) - x2 * (R(1.0 / 120.0) - x2 * R(1.0 / 5040.0))));
      ca = R(1) - x2 * (R(0.5) - x2 * (R(1.0 / 24.0) - x2 * (R(1.0 / 720.0) - x2 * R(1.0 / 40320.0))));
    } else {
      sincos_<R>(-step, &sa, &ca);
    }
    R nc = ct * ca - st * sa, ns = st * ca + ct * sa;
    ct = nc;
    st = ns;
  }
  if constexpr (sizeof(R) == 4) {   // back onto the unit circle after the rotations
    const R r = rsqrt_<R>(ct * ct + st * st);
    ct *= r;
    st *= r;
  }
  *cs = ct;
  *ss = st;
}

// Moments of a whole ellipse on the disk whose g has a single maximum (the
// classification and maybe_two_maxima decide that): area, the full-turn f_lin
// rule clustered at the maximum (Newton's method), second moment in closed form.
// The same as occulted_r's whole-ellipse branch for such an ellipse, written on
// its own so that the light-curve kernels can call a small function for the
// common case.
template <typename R>
GL_HD void whole_single_moments(const SetConst& c, R x0, R y0, R omr2, const NodeRule<R>& rule,
                                R I[3]);

// ------------------------------------------------------------------ quartics
// Division and cosine for the quartic solver.  FAST (FP32 on the GPU only): the
// hardware's approximate divide and cosine, for estimates that Newton steps
// refine afterwards (crossing_roots_f32); otherwise the correctly rounded
// divide and the library cosine.
template <typename T, bool FAST>
GL_HD T q_div(T a, T b) {
#if defined(__CUDA_ARCH__)
  if constexpr (FAST && sizeof(T) == 4) return __fdividef(a, b);
#endif
  return a / b;
}
template <typename T, bool FAST>
GL_HD T q_cos(T x) {
#if defined(__CUDA_ARCH__)
  if constexpr (FAST && sizeof(T) == 4) return __cosf(x);
#endif
  return m_cos(x);
}

// Largest real root of z^3 + a z^2 + b z + c, refined by Newton.
template <typename T, bool FAST = false>
GL_HD T cubic_largest_root(T a, T b, T c) {
  T Q = (a * a - T(3) * b) * T(1.0 / 9.0);
  T Rr = (T(2) * a * a * a - T(9) * a * b + T(27) * c) * T(1.0 / 54.0);
  T z;
  if (Q > T(0) && Rr * Rr < Q * Q * Q) {
    T arg = q_div<T, FAST>(Rr, m_sqrt(Q * Q * Q));
    arg = arg < T(-1) ? T(-1) : (arg > T(1) ? T(1) : arg);
    T th = m_acos(arg);
    z = -T(2) * m_sqrt(Q) * q_cos<T, FAST>((th + T(2 * kPi)) * T(1.0 / 3.0)) - a * T(1.0 / 3.0);
  } else {
    T disc = Rr * Rr - Q * Q * Q;
    T A = -m_copysign(m_cbrt(m_abs(Rr) + m_sqrt(disc > T(0) ? disc : T(0))), Rr);
    T B = (A != T(0)) ? q_div<T, FAST>(Q, A) : T(0);
    z = A + B - a * T(1.0 / 3.0);
  }
#pragma unroll 1
  for (int it = 0; it < 3; ++it) {
    T f = ((z + a) * z + b) * z + c;
    T fp = (T(3) * z + T(2) * a) * z + b;
    if (fp == T(0)) break;
    T step = q_div<T, FAST>(f, fp);
    z -= step;
    if (m_abs(step) <= m_eps<T>() * m_abs(z)) break;
  }
  return z;
}

// Real roots of the monic quadratic y^2 + p y + q; returns how many (0 or 2).
template <typename T, bool FAST = false>
GL_HD int quad_roots(T p, T q, T* r) {
  T disc = p * p - T(4) * q;
  if (disc < T(0)) return 0;
  T s = m_sqrt(disc);
  T y1 = -T(0.5) * (p + m_copysign(s, p));
  r[0] = y1;
  r[1] = (y1 != T(0)) ? q_div<T, FAST>(q, y1) : T(0);
  return 2;
}

// Real roots of x^4 + a x^3 + b x^2 + c x + d by Ferrari's resolvent, each
// polished by Newton on the quartic.  Returns the count (0..4).
template <typename T, bool FAST = false>
GL_HD int quartic_real_roots(T a, T b, T c, T d, T* x) {
  T a2 = a * a;
  T p = b - T(0.375) * a2;
  T q = c - T(0.5) * a * b + T(0.125) * a2 * a;
  T r = d - T(0.25) * a * c + T(0.0625) * a2 * b - T(0.01171875) * a2 * a2;
  T y[4];
  int n = 0;
  // resolvent: z^3 + 2p z^2 + (p^2 - 4r) z - q^2 = 0, z = s^2 >= 0
  T z = cubic_largest_root<T, FAST>(T(2) * p, p * p - T(4) * r, -q * q);
  if (z > T(64) * m_eps<T>() * (m_abs(p) + m_sqrt(m_abs(r)) + T(1e-30))) {
    T s = m_sqrt(z);
    const T qs = q_div<T, FAST>(q, s);
    T al = T(0.5) * (p + z - qs), be = T(0.5) * (p + z + qs);
    n += quad_roots<T, FAST>(s, al, y + n);
    n += quad_roots<T, FAST>(-s, be, y + n);
  } else {
    // biquadratic: y^2 = w, w^2 + p w + r = 0
    T w[2];
    int nw = quad_roots<T, FAST>(p, r, w);
    for (int i = 0; i < nw; ++i) {
      if (w[i] >= T(0)) {
        T sw = m_sqrt(w[i]);
        y[n++] = sw;
        y[n++] = -sw;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    T t = y[i] - T(0.25) * a;
    for (int it = 0; it < 3; ++it) {
      T f = (((t + a) * t + b) * t + c) * t + d;
      T fp = ((T(4) * t + T(3) * a) * t + T(2) * b) * t + c;
      if (fp == T(0)) break;
      T step = q_div<T, FAST>(f, fp);
      t -= step;
      if (m_abs(step) <= m_eps<T>() * (T(1) + m_abs(t))) break;
    }
    x[i] = t;
  }
  return n;
}

GL_HD void sort_small(double* v, int n) {
  // (FP64 compares: integer keys measured slower, through register spills in the
  // quadrature kernel)
  for (int i = 1; i < n; ++i) {
    double x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
}
GL_HD void sort_small(float* v, int n) {
  for (int i = 1; i < n; ++i) {
    float x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
}

// g in the frame th = delta + phi, t = tan(phi/2): g (1 + t^2)^2 = sum q_k t^k.
// delta is chosen so that t -> infinity falls on the one of eight sampled
// angles where |g| is largest, which keeps q4 away from zero.
template <typename T>
struct Frame {
  T cd, sd;      // cos, sin of delta
  T q[5];        // q0..q4
};

// Index k of the sampled angle k pi/4 where |g| is largest.
template <typename T>
GL_HD int frame_choice(const Trig2<T>& t) {
  const T r2 = T(0.70710678118654752440);
  const T cs8[8] = {T(1), r2, T(0), -r2, T(-1), -r2, T(0), r2};
  const T sn8[8] = {T(0), r2, T(1), r2, T(0), -r2, T(-1), -r2};
  int kbest = 0;
  T gbest = T(-1);
  for (int kk = 0; kk < 8; ++kk) {
    T c1 = cs8[kk], s1 = sn8[kk];
    T c2 = c1 * c1 - s1 * s1, s2 = T(2) * s1 * c1;
    T gv = m_abs(t.A + t.B * c1 + t.C * s1 + t.D * c2 + t.E * s2);
    if (gv > gbest) {
      gbest = gv;
      kbest = kk;
    }
  }
  return kbest;
}

// The frame whose t = infinity falls on the sampled angle k pi/4.
template <typename T>
GL_HD Frame<T> make_frame_k(const Trig2<T>& t, int kbest) {
  const T r2 = T(0.70710678118654752440);
  const T cs8[8] = {T(1), r2, T(0), -r2, T(-1), -r2, T(0), r2};
  const T sn8[8] = {T(0), r2, T(1), r2, T(0), -r2, T(-1), -r2};
  // delta = k pi/4 + pi, so 2 delta is a multiple of pi/2 and the rotated
  // second harmonic (D', E') is (D, E), (E, -D), (-D, -E) or (-E, D): selected,
  // not multiplied
  Frame<T> f;
  f.cd = -cs8[kbest];
  f.sd = -sn8[kbest];
  const int k4 = kbest & 3;
  const T dsel = (k4 & 1) ? t.E : t.D, esel = (k4 & 1) ? t.D : t.E;
  const T Dp = (k4 & 2) ? -dsel : dsel;
  const T Ep = (k4 == 1 || k4 == 2) ? -esel : esel;
  T Bp = t.B * f.cd + t.C * f.sd, Cp = t.C * f.cd - t.B * f.sd;
  const T AD = t.A + Dp, C2 = T(2) * Cp;
  f.q[4] = AD - Bp;
  f.q[3] = C2 - T(4) * Ep;
  f.q[2] = T(2) * t.A - T(6) * Dp;
  f.q[1] = C2 + T(4) * Ep;
  f.q[0] = AD + Bp;
  return f;
}

template <typename T>
GL_HD Frame<T> make_frame(const Trig2<T>& t) {
  return make_frame_k<T>(t, frame_choice<T>(t));
}

template <typename T>
GL_HD T frame_poly(const Frame<T>& f, T t) {
  return (((f.q[4] * t + f.q[3]) * t + f.q[2]) * t + f.q[1]) * t + f.q[0];
}

// Drop coincident neighbours of a sorted list (tangency: no crossing).
template <typename T>
GL_HD int drop_pairs(T* tr, int nr, T tol) {
  T tt[4];
  int m = 0;
  for (int i = 0; i < nr; ++i) {
    if (i + 1 < nr && m_abs(tr[i + 1] - tr[i]) <= tol * (T(1) + m_abs(tr[i]))) {
      ++i;
      continue;
    }
    tt[m++] = tr[i];
  }
  for (int i = 0; i < m; ++i) tr[i] = tt[i];
  return m;
}

// Real roots of the frame's quartic in t, sorted ascending (= counter-clockwise
// order in theta), in the frame's own precision.
template <typename T>
GL_HD int frame_roots(const Frame<T>& f, T* tr) {
  if (!(m_abs(f.q[4]) > T(0))) return 0;
  T inv = T(1) / f.q[4];
  int nr = quartic_real_roots<T>(f.q[3] * inv, f.q[2] * inv, f.q[1] * inv, f.q[0] * inv, tr);
  sort_small(tr, nr);
  return drop_pairs<T>(tr, nr, T(1024) * m_eps<T>());
}

// Crossings of the boundary with the limb for the FP32 quadrature, from the FP32
// frame alone: Ferrari estimates (the steps of quartic_real_roots, fast divide and
// cosine), then Newton steps on the same FP32 quartic, all on the FP32 pipe and
// in registers (four candidate slots, sorted by a fixed network).  FP32 is enough
// here: the quadrature rounds every crossing to FP32 anyway, and each limb arc
// starts at the radial projection of the ellipse point at the crossing, where the
// Green's-theorem integrands of all three moments vanish (they are multiples of
// x dy - y dx), so an error d in a crossing leaves only the sliver between the
// two curves, O(d^2), in the moments.  Returns the number of roots (r[0..n),
// ascending), or -1 when the estimates cannot be trusted: a root whose Newton
// step has not fallen below 1e-4 (1 + |t|) within three steps (it then sits on
// rounding noise: an ill-conditioned, near-tangent root), or two roots within
// 1e-3 (1 + |t|) of each other (near tangency).  The caller then solves the FP64
// quartic.
GL_HD void quad_roots_slot(float p, float q, float* r0, float* r1, bool* ok) {
  // quad_roots<float, true> into two fixed slots
  const float disc = p * p - 4.0f * q;
  *ok = !(disc < 0.0f);
  const float sq = sqrtf(disc);
  const float y1 = -0.5f * (p + copysignf(sq, p));
  *r0 = y1;
  *r1 = (y1 != 0.0f) ? q_div<float, true>(q, y1) : 0.0f;
}

GL_HD int crossing_roots_f32(const Frame<float>& fr, float r[4]) {
  if (!(fabsf(fr.q[4]) > 0.0f)) return -1;
  const float inv = 1.0f / fr.q[4];
  const float a = fr.q[3] * inv, b = fr.q[2] * inv, c = fr.q[1] * inv, d = fr.q[0] * inv;
  const float a2 = a * a;
  const float p = b - 0.375f * a2;
  const float q = c - 0.5f * a * b + 0.125f * a2 * a;
  const float rq = d - 0.25f * a * c + 0.0625f * a2 * b - 0.01171875f * a2 * a2;
  float y[4];
  bool v[4];
  // resolvent: z^3 + 2p z^2 + (p^2 - 4r) z - q^2 = 0, z = s^2 >= 0
  const float z = cubic_largest_root<float, true>(2.0f * p, p * p - 4.0f * rq, -q * q);
  if (z > 64.0f * m_eps<float>() * (fabsf(p) + sqrtf(fabsf(rq)) + 1e-30f)) {
    const float sz = sqrtf(z);
    const float qs = q_div<float, true>(q, sz);
    quad_roots_slot(sz, 0.5f * (p + z - qs), &y[0], &y[1], &v[0]);
    quad_roots_slot(-sz, 0.5f * (p + z + qs), &y[2], &y[3], &v[2]);
  } else {
    // biquadratic: y^2 = w, w^2 + p w + r = 0
    float w0, w1;
    bool vw;
    quad_roots_slot(p, rq, &w0, &w1, &vw);
    v[0] = vw && w0 >= 0.0f;
    v[2] = vw && w1 >= 0.0f;
    y[0] = v[0] ? sqrtf(w0) : 0.0f;
    y[2] = v[2] ? sqrtf(w1) : 0.0f;
    y[1] = -y[0];
    y[3] = -y[2];
  }
  v[1] = v[0];
  v[3] = v[2];
  const float q0 = fr.q[0], q1 = fr.q[1], q2 = fr.q[2], q3 = fr.q[3], q4 = fr.q[4];
  const float d3 = 4.0f * q4, d2 = 3.0f * q3, d1 = 2.0f * q2;
  bool ok = true;
  // Newton on the monic quartic (quartic_real_roots' polish), then on the frame's
  // quartic until the step settles
  auto refine = [&](float y0) -> float {
    float t = y0 - 0.25f * a;   // (a root of the depressed quartic, shifted back)
#pragma unroll 1
    for (int it = 0; it < 3; ++it) {
      const float f = (((t + a) * t + b) * t + c) * t + d;
      const float fp = ((4.0f * t + 3.0f * a) * t + 2.0f * b) * t + c;
      if (fp == 0.0f) break;
      const float step = q_div<float, true>(f, fp);
      t -= step;
      if (fabsf(step) <= m_eps<float>() * (1.0f + fabsf(t))) break;
    }
    bool settled = false;
#pragma unroll 1
    for (int it = 0; it < 3; ++it) {
      if (!settled) {
        const float pv = (((q4 * t + q3) * t + q2) * t + q1) * t + q0;
        const float dp = ((d3 * t + d2) * t + d1) * t + q1;
        const float step = q_div<float, true>(pv, dp);
        if (!(fabsf(step) <= 1e-2f * (1.0f + fabsf(t)))) break;   // (NaN too)
        t -= step;
        settled = fabsf(step) <= 1e-4f * (1.0f + fabsf(t));
      }
    }
    ok = ok && settled;
    return t;
  };
  // roots come in pairs (one quadratic each: v[0] == v[1], v[2] == v[3]); the
  // pairs are refined in a loop (the code of one pair, not four unrolled slots),
  // the slots kept in registers by selects
  const int nr = (v[0] ? 2 : 0) + (v[2] ? 2 : 0);
#pragma unroll 1
  for (int pq = 0; pq < 2; ++pq) {
    if (v[2 * pq]) {
      const float ta = refine(pq == 0 ? y[0] : y[2]);
      const float tb = refine(pq == 0 ? y[1] : y[3]);
      y[0] = pq == 0 ? ta : y[0];
      y[1] = pq == 0 ? tb : y[1];
      y[2] = pq == 1 ? ta : y[2];
      y[3] = pq == 1 ? tb : y[3];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (!v[i]) y[i] = INFINITY;   // empty slots sort last
  if (!ok) return -1;
  // sorting network on four slots
  auto cx = [&](int i, int j) {
    const float lo = fminf(y[i], y[j]), hi = fmaxf(y[i], y[j]);
    y[i] = lo;
    y[j] = hi;
  };
  cx(0, 1);
  cx(2, 3);
  cx(0, 2);
  cx(1, 3);
  cx(1, 2);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i + 1 < nr && !(y[i + 1] - y[i] > 1e-3f * (1.0f + fabsf(y[i])))) return -1;
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] = y[i];
  return nr;
}

// (cos th, sin th) of the point t of frame f.
template <typename T>
GL_HD void frame_angle(const Frame<T>& f, T t, T* ct, T* st) {
  T den = T(1) / (T(1) + t * t);
  T cph = (T(1) - t * t) * den, sph = T(2) * t * den;
  *ct = f.cd * cph - f.sd * sph;
  *st = f.sd * cph + f.cd * sph;
}

// t of frame f for the angle (cos th, sin th); +inf at phi = pi.
template <typename T>
GL_HD T frame_t(const Frame<T>& f, T ct, T st) {
  T cph = ct * f.cd + st * f.sd, sph = st * f.cd - ct * f.sd;
  T den = T(1) + cph;
  if (!(den > T(1e-30))) return T(INFINITY);
  return sph / den;
}

// Arc of the ellipse from t_a to t_b (counter-clockwise; wrap = passes t = inf):
// half-width h and (cos, sin) of its mid-direction, in precision R.
template <typename R>
GL_HD void frame_arc(R N, R D, bool wrap, R cta, R sta, R* h, R* cm, R* sm) {
  R hyp = m_sqrt(N * N + D * D);
  R ch, sh;
  if (!wrap) {
    *h = m_atan2(N, D);
    ch = D / hyp;
    sh = N / hyp;
  } else {
    *h = R(kPi) + m_atan2(N, D);
    ch = -D / hyp;
    sh = -N / hyp;
  }
  *cm = cta * ch - sta * sh;
  *sm = sta * ch + cta * sh;
}

// Local maxima of g that lie inside the disk (g < 0): the points where the
// boundary comes nearest the limb without reaching it.  The quadrature is split
// there so that the near-singular (1 - r^2)^(3/2) sits at an arc end, where the
// mapped rule clusters its nodes.  Returns (cos, sin) of up to 2 maxima.
template <typename T>
GL_HD int inner_maxima(const Trig2<T>& t, T* cm, T* sm) {
  Trig2<T> d;   // g'(th)
  d.A = T(0);
  d.B = t.C;
  d.C = -t.B;
  d.D = T(2) * t.E;
  d.E = T(-2) * t.D;
  if (!(m_abs(d.B) + m_abs(d.C) + m_abs(d.D) + m_abs(d.E) > T(1e-30))) return 0;
  Frame<T> f = make_frame<T>(d);
  T tr[4];
  int nr = frame_roots<T>(f, tr);
  int m = 0;
  for (int i = 0; i < nr; ++i) {
    T ct, st;
    frame_angle<T>(f, tr[i], &ct, &st);
    T c2 = ct * ct - st * st, s2 = T(2) * st * ct;
    T g2 = -t.B * ct - t.C * st - T(4) * t.D * c2 - T(4) * t.E * s2;
    if (g2 < T(0) && trig2_eval<T>(t, ct, st) < T(0) && m < 2) {
      cm[m] = ct;
      sm[m] = st;
      ++m;
    }
  }
  return m;
}

// Closed-form antiderivative of f_quad along the ellipse boundary (a trig
// polynomial of degree 4 plus a linear term; derived from Sec. 2's f_quad with
// x = x0 + a cos th, y = y0 + b1 cos th + b2 sin th).  Divisions by constants
// are written as products with their reciprocals (a divide is a long
// instruction sequence; the product differs by at most one rounding).
template <typename R>
struct QuadPoly {
  R K, S[4], C[4];
};
template <typename R>
GL_HD QuadPoly<R> quad_poly(R x0, R y0, R a, R b1, R b2) {
  QuadPoly<R> q;
  R a2 = a * a, b12 = b1 * b1, b22 = b2 * b2, x02 = x0 * x0, y02 = y0 * y0;
  q.K = a * b2 * (a2 + b12 + b22 + R(4) * x02 + R(4) * y02) / R(8);
  q.S[0] = R(5) * a2 * b2 * x0 / R(8) + R(3) * a * b1 * b2 * y0 / R(4) + b12 * b2 * x0 / R(8) +
           b22 * b2 * x0 / R(8) + b2 * x02 * x0 * R(1.0 / 6.0) + b2 * x0 * y02 / R(2);
  q.C[0] = -a2 * a * y0 / R(8) - a2 * b1 * x0 / R(8) + a * b12 * y0 / R(8) -
           R(5) * a * b22 * y0 / R(8) - a * x02 * y0 / R(2) - a * y02 * y0 * R(1.0 / 6.0) +
           b12 * b1 * x0 / R(8) + b1 * b22 * x0 / R(8) + b1 * x02 * x0 * R(1.0 / 6.0) +
           b1 * x0 * y02 / R(2);
  q.C[1] = -a2 * a * b1 * R(1.0 / 24.0) - a2 * x0 * y0 / R(4) + a * b12 * b1 * R(1.0 / 24.0) -
           a * b1 * b22 / R(8) + b12 * x0 * y0 / R(4) - b22 * x0 * y0 / R(4);
  q.S[1] = a2 * a * b2 * R(1.0 / 24.0) + a * b12 * b2 / R(8) - a * b22 * b2 * R(1.0 / 24.0) +
           b1 * b2 * x0 * y0 / R(2);
  q.C[2] = -a2 * a * y0 * R(1.0 / 24.0) - a2 * b1 * x0 * R(1.0 / 24.0) + a * b12 * y0 * R(1.0 / 24.0) -
           a * b22 * y0 * R(1.0 / 24.0) + b12 * b1 * x0 * R(1.0 / 24.0) - b1 * b22 * x0 / R(8);
  q.S[2] = -a2 * b2 * x0 * R(1.0 / 24.0) + a * b1 * b2 * y0 * R(1.0 / 12.0) + b12 * b2 * x0 / R(8) -
           b22 * b2 * x0 * R(1.0 / 24.0);
  q.C[3] = -a2 * a * b1 * R(1.0 / 96.0) + a * b12 * b1 * R(1.0 / 96.0) - a * b1 * b22 / R(32);
  q.S[3] = -a2 * a * b2 * R(1.0 / 96.0) + a * b12 * b2 / R(32) - a * b22 * b2 * R(1.0 / 96.0);
  return q;
}

// sum_n S_n sin(n th) + C_n cos(n th), n = 1..4, from (cos th, sin th).
template <typename R>
GL_HD R quad_poly_trig(const QuadPoly<R>& q, R ct, R st) {
  R cn = ct, sn = st, cp = R(1), sp = R(0), acc = R(0);
  for (int n = 0; n < 4; ++n) {
    acc += q.S[n] * sn + q.C[n] * cn;
    R cnext = R(2) * ct * cn - cp, snext = R(2) * ct * sn - sp;
    cp = cn;
    sp = sn;
    cn = cnext;
    sn = snext;
  }
  return acc;
}

// ------------------------------------------------------------------ the paper's scheme
// Integrands of the paper's snapped-boundary scheme (Sec. 2) at angle th of the
// projected ellipse.  The boundary point p = (x0 + dx cos th, y0 + dy1 cos th +
// dy2 sin th) and its derivative p' = (-dx sin th, -dy1 sin th + dy2 cos th); a
// point outside the disk is moved along its ray to the limb, (x_d, y_d) =
// p / |p| = (cos lambda, sin lambda), with d lambda / d th = (x y' - y x') / |p|^2
// and the derivative of the moved point lambda' (-y_d, x_d).  On the moved curve
// the three integrands reduce to lambda'/2, lambda'/3 and
// lambda' ((x_d^4 + y_d^4)/3 + 2 x_d^2 y_d^2) / 2.  Their integrals over th in
// [0, 2 pi) are the area, Integral mu dA and Integral r^2 dA of the overlap (the
// paper's f_flat, f_lin, f_quad; f_lin written without the small-r cancellation).
template <typename T>
GL_HD void snapped_integrands(T x0, T y0, T dx, T dy1, T dy2, T ct, T st, T* ff, T* fl, T* fq) {
  const T xe = x0 + dx * ct, ye = y0 + dy1 * ct + dy2 * st;
  const T xp = -dx * st, yp = -dy1 * st + dy2 * ct;
  const T r2 = xe * xe + ye * ye;
  const T cross = xe * yp - ye * xp;
  if (r2 > T(1)) {
    const T lp = cross / r2;
    const T x2 = xe * xe / r2, y2 = ye * ye / r2;
    *ff = T(0.5) * lp;
    *fl = lp / T(3);
    *fq = T(0.5) * lp * ((x2 * x2 + y2 * y2) / T(3) + T(2) * x2 * y2);
  } else {
    const T mu = m_sqrt(T(1) - r2);
    *ff = T(0.5) * cross;
    *fl = (T(2) / T(3)) * (T(1) + mu + mu * mu) / (T(1) + mu) * (*ff);
    *fq = T(0.5) * (xe * (xe * xe / T(3) + ye * ye) * yp - ye * (xe * xe + ye * ye / T(3)) * xp);
  }
}

// The two arcs into which two directions u0, u1 split the turn: the
// counter-clockwise one from u0 to u1 (half-width h = Delta / 2, Delta in
// (0, 2 pi], its middle u0 rotated by h) and the rest (half-width pi - h, middle
// opposite).  Built from the angle alone, so no arc end can sit at a frame's
// t = infinity (two maxima exactly opposite each other are a case of symmetric
// geometry).
template <typename R>
GL_HD void split_turn(R c0, R s0, R c1, R s1, R* acm, R* asn, R* ah) {
  R d = m_atan2(c0 * s1 - s0 * c1, c0 * c1 + s0 * s1);
  if (!(d > R(0))) d += R(2 * kPi);
  const R h = R(0.5) * d;
  R sh, ch;
  sincos_<R>(h, &sh, &ch);
  acm[0] = c0 * ch - s0 * sh;
  asn[0] = s0 * ch + c0 * sh;
  ah[0] = h;
  acm[1] = -acm[0];
  asn[1] = -asn[0];
  ah[1] = R(kPi) - h;
}

// The centre of a single-centre whole-turn rule: the point of the boundary nearest
// the limb (the global maximum of g).  When the quartic of g' found fewer than
// two inner maxima, its one maximum (if any) is compared with Newton's from the
// outward normal along the centre direction and the one with the larger g is
// kept: the FP32 quartic can miss or misplace a shallow second maximum, and a
// turn clustered on a lesser maximum resolves the near-limb part poorly.
template <typename R>
GL_HD void nearest_limb_center(const Geo<R>& g, const Trig2<R>& tg, int nmax, R* cmx, R* smx) {
  R cn, sn;
  nearest_limb_angle<R>(g, tg, &cn, &sn);
  if (nmax == 0 || trig2_eval<R>(tg, cn, sn) > trig2_eval<R>(tg, cmx[0], smx[0])) {
    cmx[0] = cn;
    smx[0] = sn;
  }
}

// The arcs (mid-direction cos/sin, half-width) into which the whole turn of a
// boundary lying inside the disk is split for the f_lin quadrature: at the two
// inner maxima when there are two, otherwise one arc whose two ends meet at the
// single maximum or at the point nearest the limb.
template <typename R>
GL_HD void whole_arcs(const Geo<R>& g, const Trig2<R>& tg, int nmax, const R* cmx, const R* smx,
                      R* acm, R* asn, R* ah, int* na) {
  if (nmax == 2) {
    split_turn<R>(cmx[0], smx[0], cmx[1], smx[1], acm, asn, ah);
    *na = 2;
    return;
  }
  R cs[1] = {nmax >= 1 ? cmx[0] : R(0)}, ss[1] = {nmax >= 1 ? smx[0] : R(0)};
  nearest_limb_center<R>(g, tg, nmax, cs, ss);
  acm[0] = -cs[0];
  asn[0] = -ss[0];
  ah[0] = R(kPi);
  *na = 1;
}

// Whether the boundary of an ellipse centred at (x0, y0) may have two local
// maxima of g (a scheduling hint).  g' is a first harmonic of amplitude
// R1 = |(B, C)| plus a second of amplitude 2 R2, R2 = |(D, E)|; with
// eps = 2 R2 / R1 < 0.447, g' keeps one sign wherever |sin| of the first
// harmonic's phase exceeds eps and is monotone elsewhere, so it has exactly two
// zeros (one maximum).  R1 > 5 R2 leaves margin; below that two maxima may exist.
GL_HD bool maybe_two_maxima(const SetConst& c, float x0, float y0) {
  const float B = 2.0f * (x0 * c.fdx + y0 * c.fdy1), C = 2.0f * y0 * c.fdy2;
  return B * B + C * C <= 25.0f * (c.flpD * c.flpD + c.flpE * c.flpE);
}

template <typename R>
GL_HD void whole_single_moments(const SetConst& c, R x0, R y0, R omr2, const NodeRule<R>& rule,
                                R I[3]) {
  Geo<R> g = make_geo<R>(c, x0, y0, omr2);
  Trig2<R> tg = limb_poly<R>(c, x0, y0, omr2);
  const R area = R(kPi) * g.dx * g.dy2;
  R cs, ss;
  nearest_limb_angle<R>(g, tg, &cs, &ss);
  I[0] = area;
  I[1] = lin_full<R>(g, cs, ss, rule);
  I[2] = area * ((x0 * x0 + y0 * y0) + (g.dx * g.dx + g.dy1 * g.dy1 + g.dy2 * g.dy2) * R(0.25));
}

// Moments of a crossing-class item, every case (Sec. 2): the crossings of the
// boundary with the limb (the FP32 ones, r0.. sorted, the first nr32, when nr32 >= 0;
// else the roots of the FP64 quartic), the inner maxima of g that lie on an
// inside arc as extra breakpoints, the arcs classified by crossing parity (FP64
// tests of g at the arc midpoints for an odd count), the boundary arcs inside
// the disk and the limb arcs inside the ellipse.  Compiled apart (not inlined):
// the FP32 quadrature's common cases take the short path of occulted_r.
template <typename R>
GL_HD_NOINLINE void partial_general(const SetConst& c, R x0, R y0, const Geo<R>& g,
                                    const Trig2<R>& tg, const Frame<R>& frr, int kb, int nmax,
                                    const R* cmx, const R* smx, R area, const NodeRule<R>& rule,
                                    int nr32, float r0, float r1, float r2, float r3, R I[3]) {
  I[0] = I[1] = I[2] = R(0);
  const float r32[4] = {r0, r1, r2, r3};
  double tb[8];
  // the FP32 crossings when they stand (nr32 >= 0), else the FP64 frame and
  // its roots (always for the FP64 quadrature)
  Frame<double> fr;
  bool have64 = false;
  int nr = nr32;
  for (int i = 0; i < 4; ++i)
    if (i < nr) tb[i] = f32_to_f64_int(r32[i]);
  if (nr < 0) {
    const double xd = to_f64(x0), yd = to_f64(y0);
    const Trig2<double> tgd = limb_poly<double>(c, xd, yd, fma(-yd, yd, fma(-xd, xd, 1.0)));
    fr = make_frame_k<double>(tgd, kb);
    have64 = true;
    nr = frame_roots<double>(fr, tb);
  }
  // sign of g at the frame's t = infinity (q4: the largest |g| of eight
  // samples, so its sign is the same in either precision)
  const bool q4_neg = have64 ? neg_bits(fr.q[4]) : neg_bits(to_f64(frr.q[4]));
  // The arcs of the boundary inside the disk are gathered first and integrated
  // by one loop afterwards, so that a warp runs the quadrature once per arc
  // count rather than once per breakpoint index.
  R acm[4], asn[4], ah[4];
  int na = 0;
  CSum<R> sflat, slin, squad;
  if (nr == 0) {
    if (!q4_neg) {
      // boundary entirely outside the disk: disjoint, or the disk inside the ellipse
      R v1 = -g.x0 / g.dx, v2 = (-g.y0 - g.dy1 * v1) / g.dy2;
      if (v1 * v1 + v2 * v2 < R(1)) {
        I[0] = R(kPi);
        I[1] = R(2.0 * kPi / 3.0);
        I[2] = R(0.5 * kPi);
      }
      return;
    }
    // boundary entirely inside the disk: the whole turn, split at the inner
    // maxima as in the whole-ellipse case below
    sflat.add(area);
    squad.add(area * ((x0 * x0 + y0 * y0) + (g.dx * g.dx + g.dy1 * g.dy1 + g.dy2 * g.dy2) / R(4)));
    whole_arcs<R>(g, tg, nmax, cmx, smx, acm, asn, ah, &na);
  } else {
    // g at the frame's t = infinity (q4, the largest |g| of eight samples, so
    // its sign is safe) says whether the arc through it lies inside the disk;
    // g changes sign at each crossing, so the others alternate from there.  An
    // odd count (possible only from the FP64 fallback in degenerate cases)
    // falls back to FP64 tests of g at the arc midpoints.
    const bool wrap_in = q4_neg;
    const bool parity = (nr & 1) == 0 || !have64;   // (FP32 roots come in pairs)
    // breakpoints: the crossings (kind 1) and the inner maxima (kind 0) that
    // lie on an inside arc.  A maximum that rounding placed on an outside arc
    // (between two close crossings) would split that arc and lose the limb arc
    // joining the two crossings, so it is dropped.
    int kind[8];
    for (int i = 0; i < nr; ++i) kind[i] = 1;
    int nb = nr;
    for (int i = 0; i < nmax; ++i) {
      R tvr = frame_t<R>(frr, cmx[i], smx[i]);
      if (!m_finite(tvr)) continue;
      double tv = to_f64(tvr);
      int below = 0;
      const long long kv = dkey(tv);
      for (int k = 0; k < nb; ++k) below += (kind[k] && dkey(tb[k]) < kv) ? 1 : 0;
      const bool on_inside = parity ? (wrap_in != ((below & 1) != 0))
                                    : (frame_poly<double>(fr, tv) < 0.0);
      if (!on_inside) continue;
      int j = nb - 1;
      while (j >= 0 && dkey(tb[j]) > kv) {
        tb[j + 1] = tb[j];
        kind[j + 1] = kind[j];
        --j;
      }
      tb[j + 1] = tv;
      kind[j + 1] = 0;
      ++nb;
    }
    R cth[8], sth[8], px[8], py[8];
    R tr_[8];
    for (int i = 0; i < nb; ++i) {
      tr_[i] = from_f64<R>(tb[i]);
      frame_angle<R>(frr, tr_[i], &cth[i], &sth[i]);
      R qx = g.x0 + g.dx * cth[i];
      R qy = g.y0 + g.dy1 * cth[i] + g.dy2 * sth[i];
      R nrm = rsqrt_<R>(qx * qx + qy * qy);
      px[i] = qx * nrm;
      py[i] = qy * nrm;
    }
    QuadPoly<R> qp = quad_poly<R>(g.x0, g.y0, g.dx, g.dy1, g.dy2);
    int ncross = 0;
    for (int i = 0; i < nb; ++i) {
      int ip = (i + 1 == nb) ? 0 : i + 1;
      bool wrap = (i + 1 == nb);
      ncross += kind[i];
      R h, cm, sm;
      frame_arc<R>(tr_[ip] - tr_[i], R(1) + tr_[i] * tr_[ip], wrap, cth[i], sth[i], &h, &cm,
                   &sm);
      if (nb == 1) {   // a lone breakpoint: the arc is the full turn
        h = R(kPi);
        cm = -cth[i];
        sm = -sth[i];
      }
      bool inside;
      if (wrap) inside = wrap_in;
      else if (parity) inside = wrap_in != ((ncross & 1) != 0);
      else inside = frame_poly<double>(fr, 0.5 * (tb[i] + tb[ip])) < 0.0;
      if (inside) {
        if (na < 4) {
          acm[na] = cm;
          asn[na] = sm;
          ah[na] = h;
          ++na;
        }
        R ca = cth[i], sa = sth[i], cb = cth[ip], sb = sth[ip];
        R dth = R(2) * h;
        sflat.add(R(0.5) * (g.W0 * dth + g.Wc * (sb - sa) - g.Ws * (cb - ca)));
        squad.add(qp.K * dth + (quad_poly_trig<R>(qp, cb, sb) - quad_poly_trig<R>(qp, ca, sa)));
      } else if (kind[i] && kind[ip]) {
        // the limb arc between the same two crossings lies inside the ellipse
        R cr = px[i] * py[ip] - py[i] * px[ip], dt = px[i] * px[ip] + py[i] * py[ip];
        R dl = m_atan2(cr, dt);
        if (dl < R(0)) dl += R(2 * kPi);
        R s4a = R(4) * px[i] * py[i] * (px[i] * px[i] - py[i] * py[i]);
        R s4b = R(4) * px[ip] * py[ip] * (px[ip] * px[ip] - py[ip] * py[ip]);
        sflat.add(R(0.5) * dl);
        slin.add(dl * R(1.0 / 3.0));
        squad.add(R(0.25) * dl - (s4b - s4a) * R(1.0 / 48.0));
      }
    }
  }
  for (int k = 0; k < na; ++k) slin.add(lin_arc<R>(g, acm[k], asn[k], ah[k], rule));
  I[0] = sflat.value();
  I[1] = slin.value();
  I[2] = squad.value();
}

// The common cases of a crossing-class item in the FP32 quadrature, where g has a
// single maximum: no crossing (the boundary wholly outside the disk, or wholly
// inside it: the whole turn centred opposite the maximum of g nearest the limb),
// or two crossings t0 < t1 (one boundary arc inside the disk, the limb arc
// between the crossings inside the ellipse).  The operations and their order are
// partial_general's for these cases, so both give the same bits.
template <typename R>
GL_HD void partial_short(const Geo<R>& g, const Trig2<R>& tg, const Frame<R>& frr, R x0, R y0,
                         R area, const NodeRule<R>& rule, int nr, R t0, R t1, bool q4_neg,
                         R I[3]) {
  CSum<R> sflat, slin, squad;
  R h, cm, sm;
  if (nr == 0) {
    if (!q4_neg) {
      // boundary entirely outside the disk: disjoint, or the disk inside the ellipse
      R v1 = -g.x0 / g.dx, v2 = (-g.y0 - g.dy1 * v1) / g.dy2;
      const bool cover = v1 * v1 + v2 * v2 < R(1);
      I[0] = cover ? R(kPi) : R(0);
      I[1] = cover ? R(2.0 * kPi / 3.0) : R(0);
      I[2] = cover ? R(0.5 * kPi) : R(0);
      return;
    }
    sflat.add(area);
    squad.add(area * ((x0 * x0 + y0 * y0) + (g.dx * g.dx + g.dy1 * g.dy1 + g.dy2 * g.dy2) / R(4)));
    R cs[1] = {R(0)}, ss[1] = {R(0)};
    nearest_limb_center<R>(g, tg, 0, cs, ss);
    cm = -cs[0];
    sm = -ss[0];
    h = R(kPi);
  } else {
    R c0, s0, c1, s1;
    frame_angle<R>(frr, t0, &c0, &s0);
    frame_angle<R>(frr, t1, &c1, &s1);
    // the crossings projected radially onto the limb
    const R qx0 = g.x0 + g.dx * c0, qy0 = g.y0 + g.dy1 * c0 + g.dy2 * s0;
    const R n0 = rsqrt_<R>(qx0 * qx0 + qy0 * qy0);
    const R px0 = qx0 * n0, py0 = qy0 * n0;
    const R qx1 = g.x0 + g.dx * c1, qy1 = g.y0 + g.dy1 * c1 + g.dy2 * s1;
    const R n1 = rsqrt_<R>(qx1 * qx1 + qy1 * qy1);
    const R px1 = qx1 * n1, py1 = qy1 * n1;
    const QuadPoly<R> qp = quad_poly<R>(g.x0, g.y0, g.dx, g.dy1, g.dy2);
    // boundary arc ta -> tb inside the disk
    auto ellipse = [&](R ta, R tb, bool wrap, R ca, R sa, R cb, R sb) {
      frame_arc<R>(tb - ta, R(1) + ta * tb, wrap, ca, sa, &h, &cm, &sm);
      const R dth = R(2) * h;
      sflat.add(R(0.5) * (g.W0 * dth + g.Wc * (sb - sa) - g.Ws * (cb - ca)));
      squad.add(qp.K * dth + (quad_poly_trig<R>(qp, cb, sb) - quad_poly_trig<R>(qp, ca, sa)));
    };
    // limb arc a -> b inside the ellipse
    auto limb = [&](R pxa, R pya, R pxb, R pyb) {
      const R cr = pxa * pyb - pya * pxb, dt = pxa * pxb + pya * pyb;
      R dl = m_atan2(cr, dt);
      if (dl < R(0)) dl += R(2 * kPi);
      const R s4a = R(4) * pxa * pya * (pxa * pxa - pya * pya);
      const R s4b = R(4) * pxb * pyb * (pxb * pxb - pyb * pyb);
      sflat.add(R(0.5) * dl);
      slin.add(dl * R(1.0 / 3.0));
      squad.add(R(0.25) * dl - (s4b - s4a) * R(1.0 / 48.0));
    };
    // g < 0 at t = infinity: the arc through it (t1 -> t0) lies inside the disk
    if (q4_neg) {
      limb(px0, py0, px1, py1);
      ellipse(t1, t0, true, c1, s1, c0, s0);
    } else {
      ellipse(t0, t1, false, c0, s0, c1, s1);
      limb(px1, py1, px0, py0);
    }
  }
  slin.add(lin_arc<R>(g, cm, sm, h, rule));
  I[0] = sflat.value();
  I[1] = slin.value();
  I[2] = squad.value();
}

// ------------------------------------------------------------------ occulted moments
// Moments of the region where the projected ellipse covers the stellar disk:
// I[0] = area, I[1] = Integral mu dA, I[2] = Integral r^2 dA.
// (x0, y0, omr2 = 1 - x0^2 - y0^2) in the quadrature precision R; the
// crossings are found in FP64 from the same (x0, y0) widened to double.
// `cls` comes from the classification (kFull skips the crossings).
template <typename R>
GL_HD void occulted_r(const SetConst& c, R x0, R y0, R omr2, int cls, const NodeRule<R>& rule,
                      R I[3]) {
  I[0] = I[1] = I[2] = R(0);
  if (cls == kOut) return;
  Geo<R> g = make_geo<R>(c, x0, y0, omr2);
  Trig2<R> tg = limb_poly<R>(c, x0, y0, omr2);
  R area = R(kPi) * g.dx * g.dy2;
  R cmx[2], smx[2];
  int nmax;
  const bool one_max = !maybe_two_maxima(c, (float)x0, (float)y0);
  if (cls == kFull && one_max) {
    // a whole ellipse whose g has a single maximum (maybe_two_maxima): find it
    // by Newton's method rather than through the quartic of g'
    nearest_limb_angle<R>(g, tg, &cmx[0], &smx[0]);
    nmax = 1;
  } else if (cls == kPartial && one_max) {
    // a single maximum of g: if the boundary crosses the limb, g > 0 there, so
    // there is no maximum inside the disk; if it does not cross, the whole-turn
    // split below finds the maximum by Newton's method (whole_arcs, nmax = 0)
    nmax = 0;
  } else {
    nmax = inner_maxima<R>(tg, cmx, smx);
  }
  if (cls == kPartial) {
    const int kb = frame_choice<R>(tg);
    const Frame<R> frr = make_frame_k<R>(tg, kb);
    float r32[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int nr32 = -1;
    if constexpr (sizeof(R) == 4) {
      // FP32 quadrature: the crossings from the FP32 frame, in registers; the
      // common cases (g with a single maximum, no crossing or two) stay here
      nr32 = crossing_roots_f32(frr, r32);
      if (nmax == 0 && (nr32 == 0 || nr32 == 2)) {
        const bool q4_neg = neg_bits(to_f64(frr.q[4]));
        partial_short<R>(g, tg, frr, x0, y0, area, rule, nr32, r32[0], r32[1], q4_neg, I);
        return;
      }
    }
    partial_general<R>(c, x0, y0, g, tg, frr, kb, nmax, cmx, smx, area, rule, nr32, r32[0], r32[1],
                       r32[2], r32[3], I);
    return;
  }
  // whole ellipse inside the disk: split the turn at the inner maxima
  I[0] = area;
  I[2] = area * ((x0 * x0 + y0 * y0) + (g.dx * g.dx + g.dy1 * g.dy1 + g.dy2 * g.dy2) / R(4));
  if (nmax <= 1) {
    // (a single maximum from Newton's method is already the nearest point)
    if (!(cls == kFull && one_max)) nearest_limb_center<R>(g, tg, nmax, cmx, smx);
    I[1] = lin_full<R>(g, cmx[0], smx[0], rule);
  } else {
    R acm[2], asn[2], ah[2];
    split_turn<R>(cmx[0], smx[0], cmx[1], smx[1], acm, asn, ah);
    I[1] = lin_arc<R>(g, acm[0], asn[0], ah[0], rule) + lin_arc<R>(g, acm[1], asn[1], ah[1], rule);
  }
}

// Same, from an FP64 centre (omr2 formed in FP64 before rounding to R).
template <typename R>
GL_HD void occulted(const SetConst& c, double x0, double y0, int cls, const NodeRule<R>& rule,
                    R I[3]) {
  occulted_r<R>(c, (R)x0, (R)y0, (R)((1.0 - x0) * (1.0 + x0) - y0 * y0), cls, rule, I);
}

// Relative flux of one sub-exposure.  The subtraction from 1 is in FP64.
template <typename R>
GL_HD double subexposure_flux(const SetConst& c, double tau, const NodeRule<R>& rule) {
  if (!in_window(c, tau, 0.0)) return 1.0;
  double x0, y0, z;
  sky_position(c, tau, &x0, &y0, &z);
  int cls = classify(c, x0, y0, z);
  if (cls == kOut) return 1.0;
  R I[3];
  occulted<R>(c, x0, y0, cls, rule, I);
  R def = (R)c.c0 * I[0] + (R)c.c1 * I[1] + (R)c.c2 * I[2];
  return 1.0 - (double)def * c.invF0;
}

// ------------------------------------------------------------------ spherical planet
// Moments of the region a circle of radius p at distance z from the star's
// centre covers (the planet boundary x = z + p cos phi, y = p sin phi):
// crossings at cos phi_c = (1 - z^2 - p^2)/(2 z p) in closed form; f_flat and
// f_quad (Sec. 2) in closed form on the planet arc and the limb arc; f_lin on the
// planet arc by the mapped Gauss-Legendre rule over the half-arc [phi_c, pi]
// (the arc is symmetric about phi = pi), whose end phi_c carries the
// (1 - r^2)^(3/2) behaviour.  omz2 = 1 - z^2 from the caller's best precision.
template <typename R>
GL_HD void sphere_moments(R z, R p, R omz2, const NodeRule<R>& rule, R I[3]) {
  I[0] = I[1] = I[2] = R(0);
  if (!(p > R(0)) || z >= R(1) + p) return;
  if (z <= p - R(1)) {            // the planet covers the whole star
    I[0] = R(kPi);
    I[1] = R(2.0 * kPi / 3.0);
    I[2] = R(0.5 * kPi);
    return;
  }
  const R p2 = p * p;
  R phc, sphc, cphc;               // planet-arc crossing angle
  R lam = R(0), s4lam = R(0);      // limb-arc half-angle and sin(4 lambda_c)
  bool full = (z + p <= R(1));
  if (full) {
    phc = R(0);
    sphc = R(0);
    cphc = R(1);
  } else {
    // triangle (star centre, planet centre, crossing) with sides 1, z, p: twice
    // its area by Heron's formula, with 1 - z taken from 1 - z^2 (no cancellation
    // near tangency); then the angles at the planet centre and the star centre
    R omz = omz2 / (R(1) + z);
    R h2 = (R(1) + z + p) * (R(1) + z - p) * (p + omz) * (p - omz);
    R twoK = R(0.5) * m_sqrt(h2 > R(0) ? h2 : R(0));             // = z p sin(phi_c)
    R cnum = R(0.5) * (omz2 - p2);                                // = z p cos(phi_c)
    phc = m_atan2(twoK, cnum);
    R zp = z * p;
    sphc = twoK / zp;
    cphc = cnum / zp;
    R lnum = R(0.5) * (R(1) + z * z - p2);                         // = z cos(lambda_c)
    lam = m_atan2(twoK, lnum);                                      // z sin(lambda_c) = 2K
    R nrm = rsqrt_<R>(lnum * lnum + twoK * twoK);
    R cl = lnum * nrm, sl = twoK * nrm;
    s4lam = R(4) * sl * cl * (cl * cl - sl * sl);
  }
  // f_flat: planet arc [phi_c, 2 pi - phi_c] + limb arc [-lambda_c, lambda_c]
  I[0] = p2 * (R(kPi) - phc) - z * p * sphc + lam;   // the lens area when partial
  // f_quad: antiderivative along the planet circle (a = b2 = p, b1 = 0, y0 = 0),
  // symmetric arc: F(2 pi - phi_c) - F(phi_c) = K (2 pi - 2 phi_c) - 2 sum_n S_n sin(n phi_c)
  {
    QuadPoly<R> q = quad_poly<R>(z, R(0), p, R(0), p);
    R cn = cphc, sn = sphc, cp = R(1), sp = R(0), sines = R(0);
    for (int n = 0; n < 4; ++n) {
      sines += q.S[n] * sn;
      R cnext = R(2) * cphc * cn - cp, snext = R(2) * cphc * sn - sp;
      cp = cn;
      sp = sn;
      cn = cnext;
      sn = snext;
    }
    I[2] = q.K * (R(2 * kPi) - R(2) * phc) - R(2) * sines + (R(0.5) * lam - s4lam / R(24));
  }
  // f_lin: 2 x half-arc quadrature + limb arc (1/3)(2 lambda_c)
  {
    R a = phc, b = R(kPi);
    R m = R(0.5) * (a + b), h = R(0.5) * (b - a);
    R sm, cm;
    sincos_<R>(m, &sm, &cm);
    CSum<R> acc;
    for (int j = 0; j < rule.n; ++j) {
      R sa, ca;
      sincos_<R>(h * rule.sig[j], &sa, &ca);
      R cph = cm * ca - sm * sa;
      R omr2 = omz2 - p2 - R(2) * z * p * cph;
      acc.add(rule.wt[j] * lin_kernel<R>(omr2) * (z * p * cph + p2));
    }
    I[1] = R(2) * h * acc.value() + R(2) * lam / R(3);
  }
}

// Exposure midpoint state rounded for FP32 sub-exposure steps: position,
// 1 - x^2 - y^2 (formed in FP64) and the Taylor coefficients of the first three
// derivatives (v, a / 2, j / 6).
struct MidState {
  float x, y, z, omr2;
  float d1[3], d2[3], d3[3];
};

// The midpoint state at time offset tau from conjunction: the FP64 Kepler
// position, and (with derivs) velocity, acceleration and jerk from
// r'' = -mu r / |r|^3, mu = n^2 a^3 (exact for a Kepler orbit).  The
// derivatives only scale time offsets within an exposure (|v dt| < 0.1 stellar
// radii), so FP32 (relative error ~1e-7) is ample for them.
GL_HD MidState mid_state_at(const SetConst& c, double tau, bool derivs) {
  double sd, cm1;
  kepler_offset(c, tau, &sd, &cm1);
  const double p1 = fma(cm1, c.kc1, sd * c.ks1);           // r cos(w + nu)
  const double p2 = fma(sd, c.ks2, fma(cm1, c.kc2, c.rc));  // r sin(w + nu)
  const double x = p2 * c.cosi, y = -p1;
  MidState m;   // (conversions by integer operations, see kepler_offset)
  m.x = f64_to_f32_int(x);
  m.y = f64_to_f32_int(y);
  m.z = -f64_to_f32_int(p2) * c.kf_si;   // (only its sign and size matter: FP32)
  m.omr2 = f64_to_f32_int(fma(-y, y, fma(-x, x, 1.0)));
  if (!derivs) {
    for (int k = 0; k < 3; ++k) m.d1[k] = m.d2[k] = m.d3[k] = 0.0f;
    return m;
  }
  const float a = c.kf_a, bo = c.kf_bo, ef = c.kf_e, nm = c.kf_nm;
  const float cm1f = f64_to_f32_int(cm1), sdf = f64_to_f32_int(sd);
  const float cosE = c.kf_cEc + (c.kf_cEc * cm1f - c.kf_sEc * sdf);   // FP32 suffices here
  const float sinE = c.kf_sEc + (c.kf_sEc * cm1f + c.kf_cEc * sdf);
  const float X = a * (cosE - ef), Y = bo * sinE;
  const float r = a * (1.0f - ef * cosE);
  const float ir = 1.0f / r;
  const float Ed = nm * a * ir;                 // dE/dt
  const float Xd = -a * sinE * Ed, Yd = bo * cosE * Ed;
  const float mu = nm * nm * a * a * a;
  const float ir2 = ir * ir, ir3 = ir2 * ir;
  const float rv = X * Xd + Y * Yd;
  const float Xa = -mu * X * ir3, Ya = -mu * Y * ir3;
  const float Xj = -mu * (Xd * ir3 - 3.0f * X * rv * ir3 * ir2);
  const float Yj = -mu * (Yd * ir3 - 3.0f * Y * rv * ir3 * ir2);
  const float in[3][2] = {{Xd, Yd}, {Xa, Ya}, {Xj, Yj}};
  const float scale[3] = {1.0f, 0.5f, 1.0f / 6.0f};
  float* out[3] = {m.d1, m.d2, m.d3};
  const float cw = c.kf_cw, sw = c.kf_sw, ci = c.kf_ci, si = c.kf_si;
  for (int k = 0; k < 3; ++k) {
    const float q1 = in[k][0] * cw - in[k][1] * sw;
    const float q2 = in[k][0] * sw + in[k][1] * cw;
    out[k][0] = q2 * ci * scale[k];
    out[k][1] = -q1 * scale[k];
    out[k][2] = -q2 * si * scale[k];
  }
  return m;
}

// FP32 operations with fixed rounding (no contraction left to the compiler), so
// that code built from them gives the same bits wherever it is inlined.
GL_HD float f_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
GL_HD float f_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
GL_HD float f_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
GL_HD float f_sqrt(float a) {
#if defined(__CUDA_ARCH__)
  return __fsqrt_rn(a);
#else
  return sqrtf(a);
#endif
}

// Position dt after the midpoint by the cubic Taylor step, in FP32.  The step
// is small (|v dt| < 0.1 stellar radii), so its rounding error is far below
// the FP32 quadrature's.
GL_HD void taylor_position(const MidState& m, float dt, float* x, float* y, float* z,
                           float* omr2) {
  float dd[3];
  for (int k = 0; k < 3; ++k) dd[k] = f_mul(f_fma(f_fma(m.d3[k], dt, m.d2[k]), dt, m.d1[k]), dt);
  *x = f_add(m.x, dd[0]);
  *y = f_add(m.y, dd[1]);
  *z = f_add(m.z, dd[2]);
  const float lin = f_fma(m.x, dd[0], f_mul(m.y, dd[1]));
  const float quad = f_fma(dd[0], dd[0], f_mul(dd[1], dd[1]));
  *omr2 = f_add(f_fma(-2.0f, lin, m.omr2), -quad);
}

// Position and overlap class of the sub-exposure at offset (twice / 2) x the
// sub-exposure step from the midpoint, by the Taylor step (fixed-rounding FP32).
GL_HD int taylor_item(const SetConst& c, const MidState& m, int twice, float* x, float* y,
                      float* omr2) {
  float z;
  taylor_position(m, f_mul(0.5f * (float)twice, c.fsub_step), x, y, &z, omr2);
  if (z > 0.0f) return kOut;
  const float rho = f_sqrt(f_fma(*x, *x, f_mul(*y, *y)));
  if (rho >= f_add(f_add(1.0f, c.freq), 1e-6f)) return kOut;
  if (f_add(rho, c.freq) <= f_add(1.0f, -1e-6f)) return kFull;
  return kPartial;
}

// Deficit (1 - flux) of one sub-exposure at the given FP32 geometry.
GL_HD float deficit_f32(const SetConst& c, float x, float y, float z, float omr2,
                        const NodeRule<float>& rule) {
  int cls = classify_t<float>(c.freq, x, y, z, 1e-6f);
  if (cls == kOut) return 0.0f;
  float I[3];
  occulted_r<float>(c, x, y, omr2, cls, rule, I);
  return (c.fc0 * I[0] + c.fc1 * I[1] + c.fc2 * I[2]) * c.finvF0;
}

// Sub-exposure time offset: ((q + 1/2)/n - 1/2) * exptime.
GL_HD double subexposure_offset(int q, int n, double exptime) {
  return ((q + 0.5) / n - 0.5) * exptime;
}

}  // namespace gl
