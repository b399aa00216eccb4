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

#if defined(__CUDACC__)
#define GL_HD __host__ __device__ __forceinline__
#else
#define GL_HD inline
#endif

namespace gl {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxNodes = 48;

enum : int { kSetInvalid = 1, kSetWholeOrbit = 2 };

// Per-parameter-set constants, computed once per set in FP64.
struct SetConst {
  // orbit
  double t0, period, nmean;        // days, days, 2 pi / P
  double a_rs, ecc, b_orb;         // a, e, a sqrt(1 - e^2)
  double cosw, sinw, cosi, sini;
  double cosEc, sinEc, Mc, rc;     // eccentric anomaly, mean anomaly, radius at conjunction
  double tau_lo, tau_hi;           // window of (t - t0) wrapped to [-P/2, P/2) outside
                                   // of which the planet cannot overlap the star
  // projected ellipse x = x0 + dx cos th, y = y0 + dy1 cos th + dy2 sin th
  double dx, dy1, dy2, req;
  // limb darkening I = c0 + c1 mu + c2 r^2, F0 = pi (1 - u1/3 - u2/6)
  double c0, c1, c2, invF0;
  double exptime;
  int nsuper;
  int flags;
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
  __sincosf(x, s, c);   // |x| <= pi here
#else
  *s = ::sinf(x);
  *c = ::cosf(x);
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

// sin(d) and cos(d) - 1 for the Kepler update.  Small |d|: Taylor series in d^2
// (coefficients 1/n!, truncation below 1e-21 for |d| < 1/4); otherwise sincos.
GL_HD void sin_cosm1(double d, double* sd, double* cm1) {
  if (fabs(d) < 0.25) {
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

// Parameters of one set -> constants.  Returns false (and sets kSetInvalid) when
// the set is physically invalid.
GL_HD bool set_setup(double t0, double period, double a_rs, double b, double ecc,
                     double omega, double k, double f, double eta, double xi, double u1,
                     double u2, double exptime, int nsuper, SetConst* c) {
  c->flags = 0;
  c->t0 = t0;
  c->period = period;
  c->exptime = exptime;
  c->nsuper = nsuper;
  bool ok = isfinite(t0) && isfinite(period) && isfinite(a_rs) && isfinite(b) &&
            isfinite(ecc) && isfinite(omega) && isfinite(k) && isfinite(f) &&
            isfinite(eta) && isfinite(xi) && isfinite(u1) && isfinite(u2) &&
            isfinite(exptime) && period > 0.0 && a_rs > 0.0 && ecc >= 0.0 && ecc < 1.0 &&
            k > 0.0 && f >= 0.0 && f < 1.0 && exptime >= 0.0 && nsuper >= 1;
  double F0 = kPi * (1.0 - u1 / 3.0 - u2 / 6.0);
  ok = ok && F0 > 0.0;
  double sinw = 0.0, cosw = 1.0;
  if (ok) {
    sinw = sin(omega);
    cosw = cos(omega);
  }
  double cosi = ok ? b * (1.0 + ecc * sinw) / (a_rs * (1.0 - ecc * ecc)) : 0.0;
  ok = ok && fabs(cosi) <= 1.0;
  if (!ok) {
    c->flags = kSetInvalid;
    return false;
  }
  // -- projected ellipse of the oblate spheroid (b = c = R_eq, a = R_pol along
  //    the spin axis n = first row of R(zeta, eta, xi) = (cos eta cos xi,
  //    -cos eta sin xi, sin eta)).  The sky covariance S = R^T diag(a^2,b^2,c^2) R
  //    restricted to (x, y) is R_eq^2 I - (R_eq^2 - R_pol^2) n_xy n_xy^T, and
  //    (dx, dy1, dy2) of Eqs. dx, dy1, dy2 are its Cholesky factor.
  double req = k / cbrt(1.0 - f);
  double ce = cos(eta), cx = cos(xi), sx = sin(xi);
  double delta = req * req * f * (2.0 - f) * ce * ce;   // R_eq^2 - R_pol^2 times cos^2 eta
  double sxx = req * req - delta * cx * cx;
  double sxy = delta * cx * sx;
  double dx = sqrt(sxx);
  c->dx = dx;
  c->dy1 = sxy / dx;
  c->dy2 = req * sqrt(req * req - delta) / dx;
  c->req = req;
  // -- limb darkening in the basis (1, mu, r^2)
  c->c0 = 1.0 - u1 - 2.0 * u2;
  c->c1 = u1 + 2.0 * u2;
  c->c2 = u2;
  c->invF0 = 1.0 / F0;
  // -- orbit
  c->nmean = 2.0 * kPi / period;
  c->a_rs = a_rs;
  c->ecc = ecc;
  c->b_orb = a_rs * sqrt(1.0 - ecc * ecc);
  c->cosw = cosw;
  c->sinw = sinw;
  c->cosi = cosi;
  c->sini = sqrt(fmax(0.0, 1.0 - cosi * cosi));
  double nuc = 0.5 * kPi - omega;
  double Ec = ecc_anomaly_from_true(nuc, ecc);
  c->cosEc = cos(Ec);
  c->sinEc = sin(Ec);
  c->Mc = Ec - ecc * c->sinEc;
  c->rc = a_rs * (1.0 - ecc * c->cosEc);
  // -- window: the sky separation is at least r |sin phi| >= a (1-e) |sin phi|,
  //    phi = angle from conjunction along the orbit; behind the star (|phi| > pi/2)
  //    nothing is occulted.  Outside |phi| <= phi_w the flux is exactly 1.
  double smax = 1.0 + req * (1.0 + 1e-9) + 1e-9;
  double rmin = a_rs * (1.0 - ecc);
  if (smax >= rmin * (1.0 - 1e-12)) {
    c->flags |= kSetWholeOrbit;
    c->tau_lo = -period;
    c->tau_hi = period;
  } else {
    double phw = asin(smax / rmin);
    double taus[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      double nu = nuc + (sgn ? phw : -phw);
      double E = ecc_anomaly_from_true(nu, ecc);
      double M = E - ecc * sin(E);
      double dM = remainder(M - c->Mc, 2.0 * kPi);
      taus[sgn] = dM / c->nmean;
    }
    double margin = 1e-9 * period + 1e-12;
    c->tau_lo = fmin(taus[0], 0.0) - margin;
    c->tau_hi = fmax(taus[1], 0.0) + margin;
  }
  return true;
}

// (t - t0) wrapped to one period around the conjunction.
GL_HD double wrap_tau(const SetConst& c, double t) {
  double tau = t - c.t0;
  return tau - c.period * rint(tau / c.period);
}

GL_HD bool in_window(const SetConst& c, double tau, double halfwidth) {
  if (c.flags & kSetWholeOrbit) return true;
  return tau + halfwidth >= c.tau_lo && tau - halfwidth <= c.tau_hi;
}

// ------------------------------------------------------------------ orbit
// Sky position at time offset tau from conjunction.  Kepler's equation is
// solved for the eccentric anomaly E = E_c + d about the conjunction:
//   d - e [cos E_c sin d + sin E_c (cos d - 1)] = n tau,
// by Newton's method (bisection safeguard on the bracket |E - M| <= e).  The sky
// coordinates are formed from differences to the conjunction point, where
// r cos(w + nu) = 0 and r sin(w + nu) = r_c, so no large terms cancel.
GL_HD void sky_position(const SetConst& c, double tau, double* x0, double* y0, double* z) {
  double nt = c.nmean * tau;
  double e = c.ecc;
  double ec = e * c.cosEc, es = e * c.sinEc;
  double d = nt / (1.0 - ec);
  double sd, cm1;
  bool conv = false;
  for (int it = 0; it < 12; ++it) {
    sin_cosm1(d, &sd, &cm1);
    double F = d - ec * sd - es * cm1 - nt;
    double Fp = 1.0 - ec * (1.0 + cm1) + es * sd;
    double step = F / Fp;
    d -= step;
    if (fabs(step) <= 1e-16 * (1.0 + fabs(d))) {
      conv = true;
      break;
    }
  }
  if (!conv) {
    // bisection on E in [M - e, M + e], expressed in d = E - E_c
    double M = c.Mc + nt;
    double Ec = atan2(c.sinEc, c.cosEc);
    double lo = M - e - Ec, hi = M + e - Ec;
    for (int it = 0; it < 200 && hi - lo > 1e-16 * (1.0 + fabs(lo)); ++it) {
      double mid = 0.5 * (lo + hi);
      sin_cosm1(mid, &sd, &cm1);
      double F = mid - ec * sd - es * cm1 - nt;
      if (F > 0.0) hi = mid; else lo = mid;
    }
    d = 0.5 * (lo + hi);
  }
  sin_cosm1(d, &sd, &cm1);
  double dcosE = c.cosEc * cm1 - c.sinEc * sd;    // cos E - cos E_c
  double dsinE = c.sinEc * cm1 + c.cosEc * sd;    // sin E - sin E_c
  double dX = c.a_rs * dcosE, dY = c.b_orb * dsinE;
  double p1 = dX * c.cosw - dY * c.sinw;          // r cos(w + nu)     (0 at conjunction)
  double p2 = c.rc + (dX * c.sinw + dY * c.cosw); // r sin(w + nu)     (r_c at conjunction)
  *y0 = -p1;
  *x0 = p2 * c.cosi;
  *z = -p2 * c.sini;
}

// ------------------------------------------------------------------ sky geometry
enum : int { kOut = 0, kFull = 1, kPartial = 2 };

// Quick classification from the centre distance alone (R_eq is the largest
// semi-axis of the projection).  kPartial means "decide with the roots".
GL_HD int classify(const SetConst& c, double x0, double y0, double z) {
  if (z > 0.0) return kOut;
  double rho = sqrt(x0 * x0 + y0 * y0);
  if (rho >= 1.0 + c.req) return kOut;
  if (rho + c.req <= 1.0) return kFull;
  return kPartial;
}

// Geometry of one evaluation in the quadrature precision R.
template <typename R>
struct Geo {
  R x0, y0, omr2;      // centre, 1 - |centre|^2
  R dx, dy1, dy2;
  R W0, Wc, Ws;        // x y' - y x' = W0 + Wc cos th + Ws sin th
};

template <typename R>
GL_HD Geo<R> make_geo(const SetConst& c, double x0, double y0) {
  Geo<R> g;
  g.x0 = (R)x0;
  g.y0 = (R)y0;
  g.omr2 = (R)((1.0 - x0) * (1.0 + x0) - y0 * y0);
  g.dx = (R)c.dx;
  g.dy1 = (R)c.dy1;
  g.dy2 = (R)c.dy2;
  g.W0 = (R)(c.dx * c.dy2);
  g.Wc = (R)(x0 * c.dy2);
  g.Ws = (R)(y0 * c.dx - x0 * c.dy1);
  return g;
}

// (1 - mu^3) / (3 r^2) written without the r -> 0 cancellation:
// (1 + mu + mu^2) / (3 (1 + mu)), mu = sqrt(1 - r^2).
template <typename R>
GL_HD R lin_kernel(R omr2) {
  R q = omr2 > (R)1e-30 ? omr2 : (R)1e-30;
  R mu = q * rsqrt_<R>(q);
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
    sincos_<R>(h * rule.sig[j], &sa, &ca);
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
    // theta = th* + pi + pi sig_j
    R ct = -(cs * rule.cph[j] - ss * rule.sph[j]);
    R st = -(ss * rule.cph[j] + cs * rule.sph[j]);
    acc.add(rule.wt[j] * lin_point<R>(g, ct, st));
  }
  return R(kPi) * acc.value();
}

// g(th) = |p(th)|^2 - 1 = A + B cos th + C sin th + D cos 2th + E sin 2th.
struct Trig2 {
  double A, B, C, D, E;
};
GL_HD Trig2 limb_poly(const SetConst& c, double x0, double y0) {
  Trig2 t;
  t.A = (1.0 - x0) * (1.0 + x0) - y0 * y0;
  t.A = -t.A + 0.5 * (c.dx * c.dx + c.dy1 * c.dy1 + c.dy2 * c.dy2);
  t.B = 2.0 * (x0 * c.dx + y0 * c.dy1);
  t.C = 2.0 * y0 * c.dy2;
  t.D = 0.5 * (c.dx * c.dx + c.dy1 * c.dy1 - c.dy2 * c.dy2);
  t.E = c.dy1 * c.dy2;
  return t;
}

// Angle of the boundary point nearest the limb (maximum of g): start at the
// point whose outward normal is along the centre direction, then Newton on g'.
template <typename R>
GL_HD void nearest_limb_angle(const SetConst& c, double x0, double y0, R* cs, R* ss) {
  R bx = (R)(c.dx * x0 + c.dy1 * y0), by = (R)(c.dy2 * y0);
  R nrm = sqrt(bx * bx + by * by);
  R ct = nrm > R(0) ? bx / nrm : R(1), st = nrm > R(0) ? by / nrm : R(0);
  Trig2 t = limb_poly(c, x0, y0);
  R B = (R)t.B, C = (R)t.C, D = (R)t.D, E = (R)t.E;
  for (int it = 0; it < 3; ++it) {
    R c2 = ct * ct - st * st, s2 = R(2) * st * ct;
    R g1 = -B * st + C * ct - R(2) * D * s2 + R(2) * E * c2;
    R g2 = -B * ct - C * st - R(4) * D * c2 - R(4) * E * s2;
    if (!(g2 < R(0))) break;
    R step = g1 / g2;
    if (step > R(0.5)) step = R(0.5);
    if (step < R(-0.5)) step = R(-0.5);
    R sa, ca;
    sincos_<R>(-step, &sa, &ca);
    R nc = ct * ca - st * sa, ns = st * ca + ct * sa;
    ct = nc;
    st = ns;
  }
  *cs = ct;
  *ss = st;
}

// ------------------------------------------------------------------ quartic (FP64)
// Largest real root of z^3 + a z^2 + b z + c, refined by Newton.
GL_HD double cubic_largest_root(double a, double b, double c) {
  double Q = (a * a - 3.0 * b) / 9.0;
  double Rr = (2.0 * a * a * a - 9.0 * a * b + 27.0 * c) / 54.0;
  double z;
  if (Q > 0.0 && Rr * Rr < Q * Q * Q) {
    double th = acos(fmax(-1.0, fmin(1.0, Rr / sqrt(Q * Q * Q))));
    z = -2.0 * sqrt(Q) * cos((th + 2.0 * kPi) / 3.0) - a / 3.0;
  } else {
    double A = -copysign(cbrt(fabs(Rr) + sqrt(fmax(0.0, Rr * Rr - Q * Q * Q))), Rr);
    double B = (A != 0.0) ? Q / A : 0.0;
    z = A + B - a / 3.0;
  }
  for (int it = 0; it < 3; ++it) {
    double f = ((z + a) * z + b) * z + c;
    double fp = (3.0 * z + 2.0 * a) * z + b;
    if (fp == 0.0) break;
    double step = f / fp;
    z -= step;
    if (fabs(step) <= 1e-16 * fabs(z)) break;
  }
  return z;
}

// Real roots of the monic quadratic y^2 + p y + q; returns how many (0 or 2).
GL_HD int quad_roots(double p, double q, double* r) {
  double disc = p * p - 4.0 * q;
  if (disc < 0.0) return 0;
  double s = sqrt(disc);
  double y1 = -0.5 * (p + copysign(s, p));
  r[0] = y1;
  r[1] = (y1 != 0.0) ? q / y1 : 0.0;
  return 2;
}

// Real roots of x^4 + a x^3 + b x^2 + c x + d by Ferrari's resolvent, each
// polished by Newton on the quartic.  Returns the count (0..4).
GL_HD int quartic_real_roots(double a, double b, double c, double d, double* x) {
  double a2 = a * a;
  double p = b - 0.375 * a2;
  double q = c - 0.5 * a * b + 0.125 * a2 * a;
  double r = d - 0.25 * a * c + 0.0625 * a2 * b - 0.01171875 * a2 * a2;
  double y[4];
  int n = 0;
  // resolvent: z^3 + 2p z^2 + (p^2 - 4r) z - q^2 = 0, z = s^2 >= 0
  double z = cubic_largest_root(2.0 * p, p * p - 4.0 * r, -q * q);
  if (z > 1e-14 * (fabs(p) + sqrt(fabs(r)) + 1e-300)) {
    double s = sqrt(z);
    double al = 0.5 * (p + z - q / s), be = 0.5 * (p + z + q / s);
    n += quad_roots(s, al, y + n);
    n += quad_roots(-s, be, y + n);
  } else {
    // biquadratic: y^2 = w, w^2 + p w + r = 0
    double w[2];
    int nw = quad_roots(p, r, w);
    for (int i = 0; i < nw; ++i) {
      if (w[i] >= 0.0) {
        double sw = sqrt(w[i]);
        y[n++] = sw;
        y[n++] = -sw;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = y[i] - 0.25 * a;
    for (int it = 0; it < 3; ++it) {
      double f = (((t + a) * t + b) * t + c) * t + d;
      double fp = ((4.0 * t + 3.0 * a) * t + 2.0 * b) * t + c;
      if (fp == 0.0) break;
      double step = f / fp;
      t -= step;
      if (fabs(step) <= 1e-16 * (1.0 + fabs(t))) break;
    }
    x[i] = t;
  }
  return n;
}

// Closed-form antiderivative of f_quad along the ellipse boundary (a trig
// polynomial of degree 4 plus a linear term; derived from Sec. 2's f_quad with
// x = x0 + a cos th, y = y0 + b1 cos th + b2 sin th).
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
           b22 * b2 * x0 / R(8) + b2 * x02 * x0 / R(6) + b2 * x0 * y02 / R(2);
  q.C[0] = -a2 * a * y0 / R(8) - a2 * b1 * x0 / R(8) + a * b12 * y0 / R(8) -
           R(5) * a * b22 * y0 / R(8) - a * x02 * y0 / R(2) - a * y02 * y0 / R(6) +
           b12 * b1 * x0 / R(8) + b1 * b22 * x0 / R(8) + b1 * x02 * x0 / R(6) +
           b1 * x0 * y02 / R(2);
  q.C[1] = -a2 * a * b1 / R(24) - a2 * x0 * y0 / R(4) + a * b12 * b1 / R(24) -
           a * b1 * b22 / R(8) + b12 * x0 * y0 / R(4) - b22 * x0 * y0 / R(4);
  q.S[1] = a2 * a * b2 / R(24) + a * b12 * b2 / R(8) - a * b22 * b2 / R(24) +
           b1 * b2 * x0 * y0 / R(2);
  q.C[2] = -a2 * a * y0 / R(24) - a2 * b1 * x0 / R(24) + a * b12 * y0 / R(24) -
           a * b22 * y0 / R(24) + b12 * b1 * x0 / R(24) - b1 * b22 * x0 / R(8);
  q.S[2] = -a2 * b2 * x0 / R(24) + a * b1 * b2 * y0 / R(12) + b12 * b2 * x0 / R(8) -
           b22 * b2 * x0 / R(24);
  q.C[3] = -a2 * a * b1 / R(96) + a * b12 * b1 / R(96) - a * b1 * b22 / R(32);
  q.S[3] = -a2 * a * b2 / R(96) + a * b12 * b2 / R(32) - a * b22 * b2 / R(96);
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

// ------------------------------------------------------------------ trig quartics
// g(th) in the frame th = delta + phi, t = tan(phi/2): g (1 + t^2)^2 = sum q_k t^k.
// delta is chosen so that t -> infinity falls on the one of eight sampled
// angles where |g| is largest, which keeps q4 away from zero.
struct Frame {
  double cd, sd;      // cos, sin of delta
  double q[5];        // q0..q4
};

GL_HD Frame make_frame(const Trig2& t) {
  const double r2 = 0.70710678118654752440;
  const double cs8[8] = {1.0, r2, 0.0, -r2, -1.0, -r2, 0.0, r2};
  const double sn8[8] = {0.0, r2, 1.0, r2, 0.0, -r2, -1.0, -r2};
  int kbest = 0;
  double gbest = -1.0;
  for (int kk = 0; kk < 8; ++kk) {
    double c1 = cs8[kk], s1 = sn8[kk];
    double c2 = c1 * c1 - s1 * s1, s2 = 2.0 * s1 * c1;
    double gv = fabs(t.A + t.B * c1 + t.C * s1 + t.D * c2 + t.E * s2);
    if (gv > gbest) {
      gbest = gv;
      kbest = kk;
    }
  }
  Frame f;
  f.cd = -cs8[kbest];
  f.sd = -sn8[kbest];
  double c2d = f.cd * f.cd - f.sd * f.sd, s2d = 2.0 * f.sd * f.cd;
  double Bp = t.B * f.cd + t.C * f.sd, Cp = t.C * f.cd - t.B * f.sd;
  double Dp = t.D * c2d + t.E * s2d, Ep = t.E * c2d - t.D * s2d;
  f.q[4] = t.A - Bp + Dp;
  f.q[3] = 2.0 * Cp - 4.0 * Ep;
  f.q[2] = 2.0 * t.A - 6.0 * Dp;
  f.q[1] = 2.0 * Cp + 4.0 * Ep;
  f.q[0] = t.A + Bp + Dp;
  return f;
}

GL_HD double frame_poly(const Frame& f, double t) {
  return (((f.q[4] * t + f.q[3]) * t + f.q[2]) * t + f.q[1]) * t + f.q[0];
}

// Real roots in t, sorted ascending (= counter-clockwise order in theta), with
// coincident pairs (tangency, no crossing) removed.
GL_HD int frame_roots(const Frame& f, double* tr) {
  if (!(fabs(f.q[4]) > 0.0)) return 0;
  double inv = 1.0 / f.q[4];
  int nr = quartic_real_roots(f.q[3] * inv, f.q[2] * inv, f.q[1] * inv, f.q[0] * inv, tr);
  for (int i = 1; i < nr; ++i) {
    double v = tr[i];
    int j = i - 1;
    while (j >= 0 && tr[j] > v) {
      tr[j + 1] = tr[j];
      --j;
    }
    tr[j + 1] = v;
  }
  double tt[4];
  int m = 0;
  for (int i = 0; i < nr; ++i) {
    if (i + 1 < nr && fabs(tr[i + 1] - tr[i]) <= 1e-13 * (1.0 + fabs(tr[i]))) {
      ++i;
      continue;
    }
    tt[m++] = tr[i];
  }
  for (int i = 0; i < m; ++i) tr[i] = tt[i];
  return m;
}

// (cos th, sin th) of the point t of frame f.
GL_HD void frame_angle(const Frame& f, double t, double* ct, double* st) {
  double den = 1.0 / (1.0 + t * t);
  double cph = (1.0 - t * t) * den, sph = 2.0 * t * den;
  *ct = f.cd * cph - f.sd * sph;
  *st = f.sd * cph + f.cd * sph;
}

GL_HD double trig2_eval(const Trig2& t, double ct, double st) {
  return t.A + t.B * ct + t.C * st + t.D * (ct * ct - st * st) + t.E * (2.0 * st * ct);
}

// Local maxima of g that lie inside the disk (g < 0): the points where the
// boundary comes nearest the limb without reaching it.  The quadrature is split
// there so that the near-singular (1 - r^2)^(3/2) sits at an arc end, where the
// mapped rule clusters its nodes.  Returns (cos, sin) of up to 2 maxima.
GL_HD int inner_maxima(const Trig2& t, double* cm, double* sm) {
  Trig2 d;   // g'(th)
  d.A = 0.0;
  d.B = t.C;
  d.C = -t.B;
  d.D = 2.0 * t.E;
  d.E = -2.0 * t.D;
  if (!(fabs(d.B) + fabs(d.C) + fabs(d.D) + fabs(d.E) > 1e-300)) return 0;
  Frame f = make_frame(d);
  double tr[4];
  int nr = frame_roots(f, tr);
  int m = 0;
  for (int i = 0; i < nr; ++i) {
    double ct, st;
    frame_angle(f, tr[i], &ct, &st);
    double c2 = ct * ct - st * st, s2 = 2.0 * st * ct;
    double g2 = -t.B * ct - t.C * st - 4.0 * t.D * c2 - 4.0 * t.E * s2;
    if (g2 < 0.0 && trig2_eval(t, ct, st) < 0.0 && m < 2) {
      cm[m] = ct;
      sm[m] = st;
      ++m;
    }
  }
  return m;
}

// t of frame f for the angle (cos th, sin th); +inf at phi = pi.
GL_HD double frame_t(const Frame& f, double ct, double st) {
  double cph = ct * f.cd + st * f.sd, sph = st * f.cd - ct * f.sd;
  double den = 1.0 + cph;
  if (!(den > 1e-300)) return INFINITY;
  return sph / den;
}

// Arc of the ellipse from t_a to t_b (counter-clockwise; wrap = passes t = inf):
// half-width h and (cos, sin) of its mid-direction in theta.
GL_HD void frame_arc(const Frame& f, double ta, double tb, bool wrap, double cta, double sta,
                     double* h, double* cm, double* sm) {
  double N = tb - ta, D = 1.0 + ta * tb;
  double hyp = sqrt(N * N + D * D);
  double ch, sh;
  if (!wrap) {
    *h = atan2(N, D);
    ch = D / hyp;
    sh = N / hyp;
  } else {
    *h = kPi + atan2(N, D);
    ch = -D / hyp;
    sh = -N / hyp;
  }
  *cm = cta * ch - sta * sh;
  *sm = sta * ch + cta * sh;
}

// ------------------------------------------------------------------ occulted moments
// I[0] = area, I[1] = Integral mu dA, I[2] = Integral r^2 dA of the region where
// the projected ellipse covers the stellar disk.  `cls` comes from classify().
template <typename R>
GL_HD void occulted(const SetConst& c, double x0, double y0, int cls, const NodeRule<R>& rule,
                    R I[3]) {
  I[0] = I[1] = I[2] = R(0);
  if (cls == kOut) return;
  Geo<R> g = make_geo<R>(c, x0, y0);
  Trig2 tg = limb_poly(c, x0, y0);
  R area = R(kPi) * g.dx * g.dy2;
  double cmx[2], smx[2];
  int nmax = inner_maxima(tg, cmx, smx);
  if (cls == kPartial) {
    Frame fr = make_frame(tg);
    double tb[8];
    int nr = frame_roots(fr, tb);
    if (nr == 0) {
      if (!(fr.q[4] < 0.0)) {
        // boundary entirely outside the disk: disjoint, or the disk inside the ellipse
        double v1 = -x0 / c.dx, v2 = (-y0 - c.dy1 * v1) / c.dy2;
        if (v1 * v1 + v2 * v2 < 1.0) {
          I[0] = R(kPi);
          I[1] = R(2.0 * kPi / 3.0);
          I[2] = R(0.5 * kPi);
        }
        return;
      }
      cls = kFull;   // boundary entirely inside the disk
    } else {
      // breakpoints: the crossings (kind 1) and the inner maxima (kind 0)
      int kind[8];
      for (int i = 0; i < nr; ++i) kind[i] = 1;
      int nb = nr;
      for (int i = 0; i < nmax; ++i) {
        double tv = frame_t(fr, cmx[i], smx[i]);
        if (!isfinite(tv)) continue;
        int j = nb - 1;
        while (j >= 0 && tb[j] > tv) {
          tb[j + 1] = tb[j];
          kind[j + 1] = kind[j];
          --j;
        }
        tb[j + 1] = tv;
        kind[j + 1] = 0;
        ++nb;
      }
      double cth[8], sth[8], px[8], py[8];
      for (int i = 0; i < nb; ++i) {
        frame_angle(fr, tb[i], &cth[i], &sth[i]);
        px[i] = x0 + c.dx * cth[i];
        py[i] = y0 + c.dy1 * cth[i] + c.dy2 * sth[i];
        double nrm = 1.0 / sqrt(px[i] * px[i] + py[i] * py[i]);
        px[i] *= nrm;
        py[i] *= nrm;
      }
      QuadPoly<R> qp = quad_poly<R>(g.x0, g.y0, g.dx, g.dy1, g.dy2);
      CSum<R> sflat, slin, squad;
      for (int i = 0; i < nb; ++i) {
        int ip = (i + 1 == nb) ? 0 : i + 1;
        bool wrap = (i + 1 == nb);
        double h, cm, sm;
        frame_arc(fr, tb[i], tb[ip], wrap, cth[i], sth[i], &h, &cm, &sm);
        if (nb == 1) {   // a lone breakpoint: the arc is the full turn
          h = kPi;
          cm = -cth[i];
          sm = -sth[i];
        }
        bool inside = wrap ? (fr.q[4] < 0.0) : (frame_poly(fr, 0.5 * (tb[i] + tb[ip])) < 0.0);
        if (inside) {
          slin.add(lin_arc<R>(g, (R)cm, (R)sm, (R)h, rule));
          R ca = (R)cth[i], sa = (R)sth[i], cb = (R)cth[ip], sb = (R)sth[ip];
          R dth = (R)(2.0 * h);
          sflat.add(R(0.5) * (g.W0 * dth + g.Wc * (sb - sa) - g.Ws * (cb - ca)));
          squad.add(qp.K * dth + (quad_poly_trig<R>(qp, cb, sb) - quad_poly_trig<R>(qp, ca, sa)));
        } else if (kind[i] && kind[ip]) {
          // the limb arc between the same two crossings lies inside the ellipse
          double cr = px[i] * py[ip] - py[i] * px[ip], dt = px[i] * px[ip] + py[i] * py[ip];
          double dl = atan2(cr, dt);
          if (dl < 0.0) dl += 2.0 * kPi;
          double s4a = 4.0 * px[i] * py[i] * (px[i] * px[i] - py[i] * py[i]);
          double s4b = 4.0 * px[ip] * py[ip] * (px[ip] * px[ip] - py[ip] * py[ip]);
          R dlr = (R)dl;
          sflat.add(R(0.5) * dlr);
          slin.add(dlr / R(3));
          squad.add(R(0.25) * dlr - (R)((s4b - s4a) / 48.0));
        }
      }
      I[0] = sflat.value();
      I[1] = slin.value();
      I[2] = squad.value();
      return;
    }
  }
  // whole ellipse inside the disk: split the turn at the inner maxima
  I[0] = area;
  I[2] = area * ((R)(x0 * x0 + y0 * y0) + (g.dx * g.dx + g.dy1 * g.dy1 + g.dy2 * g.dy2) / R(4));
  if (nmax <= 1) {
    R cs, ss;
    if (nmax == 1) {
      cs = (R)cmx[0];
      ss = (R)smx[0];
    } else {
      nearest_limb_angle<R>(c, x0, y0, &cs, &ss);
    }
    I[1] = lin_full<R>(g, cs, ss, rule);
  } else {
    Frame fr = make_frame(tg);
    double ta = frame_t(fr, cmx[0], smx[0]), tb2 = frame_t(fr, cmx[1], smx[1]);
    double ca = cmx[0], sa = smx[0], cb = cmx[1], sb = smx[1];
    if (!isfinite(ta) || !isfinite(tb2)) {
      R cs = (R)cmx[0], ss = (R)smx[0];
      I[1] = lin_full<R>(g, cs, ss, rule);
      return;
    }
    if (ta > tb2) {
      double tmp = ta; ta = tb2; tb2 = tmp;
      tmp = ca; ca = cb; cb = tmp;
      tmp = sa; sa = sb; sb = tmp;
    }
    double h1, cm1, sm1, h2, cm2, sm2;
    frame_arc(fr, ta, tb2, false, ca, sa, &h1, &cm1, &sm1);
    frame_arc(fr, tb2, ta, true, cb, sb, &h2, &cm2, &sm2);
    I[1] = lin_arc<R>(g, (R)cm1, (R)sm1, (R)h1, rule) + lin_arc<R>(g, (R)cm2, (R)sm2, (R)h2, rule);
  }
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

// Sub-exposure time offset: ((q + 1/2)/n - 1/2) * exptime.
GL_HD double subexposure_offset(int q, int n, double exptime) {
  return ((q + 0.5) / n - 0.5) * exptime;
}

}  // namespace gl
