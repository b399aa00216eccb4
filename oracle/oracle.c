/*
 * oracle.c -- plain FP64 CPU oracle for oblate-planet transit light curves.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may link, import or call this file.  It is used by the
 * tests, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.
 *
 * It computes, by the plain definition and slowly, the relative flux
 *
 *     F(t) = 1 - (1/F0) * Integral_{E(t) n D} I(r) dA
 *
 * where D is the unit stellar disk, E(t) the sky-plane projection of the
 * planet (Sec. 2, "Ellipsoid Transit Model", Eqs. dx, dy1, dy2), and
 * I(r) = 1 - u1 (1-mu) - u2 (1-mu)^2, mu = sqrt(1-r^2) the quadratic
 * limb-darkening law named in Sec. 2 and Sec. 3.  F0 = Integral_D I dA.
 *
 * The area integral is an iterated integral, outer over x, inner over y.  The
 * inner integral is done with the textbook antiderivatives of 1, sqrt(R^2-y^2)
 * and x^2+y^2; the outer one by globally adaptive Gauss-Legendre quadrature
 * with breakpoints at every kink of the outer integrand (the x of each
 * ellipse/limb crossing, and x = +-1).  It does NOT use Green's theorem, the
 * intersection quartic or any node table of the GPU path.
 *
 * Orbit: Keplerian, solved by bisection-safeguarded Newton on E - e sin E = M.
 * Sec. 2 uses a circular orbit (x0 = d cos(alpha) sin(beta), y0 = d sin(alpha));
 * the eccentric generalisation follows the usual convention (transit at true
 * anomaly nu = pi/2 - omega, t0 = time of conjunction) and reduces to the
 * paper's formulas when e = 0, omega = pi/2.
 *
 * Every function cites the passage of the paper it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes, computed at start-up by Newton iteration on  */
/* the Legendre polynomial recurrence (textbook; no stored tables).   */
/* ------------------------------------------------------------------ */
#define ORC_GL_N 16
static double gl_x[ORC_GL_N], gl_w[ORC_GL_N];
static int gl_ready = 0;

static void gl_init(void) {
    if (gl_ready) return;
    const int n = ORC_GL_N;
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    gl_ready = 1;
}

/* ------------------------------------------------------------------ */
/* Orbit (Sec. 2, Eq. coord-map with the circular orbit generalised)  */
/* ------------------------------------------------------------------ */

/* Solve Kepler's equation E - e sin E = M for E, |E - M| <= e.
 * Monotone in E for 0 <= e < 1, so bisection on [M-e, M+e] always converges;
 * Newton steps are taken whenever they stay inside the bracket. */
double orc_kepler_E(double M, double e) {
    double Mr = remainder(M, 2.0 * M_PI);
    double shift = M - Mr;
    if (e == 0.0) return M;
    double lo = Mr - e, hi = Mr + e;
    double E = Mr + 0.85 * e * (sin(Mr) >= 0 ? 1.0 : -1.0);
    if (E < lo || E > hi) E = Mr;
    for (int it = 0; it < 200; ++it) {
        double fE = E - e * sin(E) - Mr;
        if (fE == 0.0) break;
        if (fE > 0) hi = E; else lo = E;
        double fp = 1.0 - e * cos(E);
        double En = E - fE / fp;
        if (!(En > lo && En < hi)) En = 0.5 * (lo + hi);
        if (fabs(En - E) <= 1e-16 * (1.0 + fabs(E)) || hi - lo <= 1e-16 * (1.0 + fabs(E))) {
            E = En;
            break;
        }
        E = En;
    }
    return E + shift;
}

/* Orbital inclination from the impact parameter at conjunction:
 * b = (a/R*) cos i (1 - e^2)/(1 + e sin w). */
double orc_cos_inclination(double b, double a_rs, double e, double w) {
    return b * (1.0 + e * sin(w)) / (a_rs * (1.0 - e * e));
}

/* Mean anomaly at conjunction (true anomaly nu_c = pi/2 - w). */
double orc_mean_anomaly_conjunction(double e, double w) {
    double nu = 0.5 * M_PI - w;
    double E = 2.0 * atan2(sqrt(1.0 - e) * sin(0.5 * nu), sqrt(1.0 + e) * cos(0.5 * nu));
    return E - e * sin(E);
}

/* Sky position of the planet centre, in stellar radii.
 * x: perpendicular to the transit chord; y: along the chord; z: along the line
 * of sight from the observer to the star (z < 0: planet in front).
 * With e = 0 and w = pi/2 this is x = d cos(alpha) sin(beta), y = d sin(alpha),
 * z = -d cos(alpha) cos(beta), alpha = mean anomaly from conjunction,
 * beta = 90 deg - i (Sec. 2). */
void orc_sky_position(double t, double t0, double period, double a_rs, double cosi,
                      double e, double w, double *x, double *y, double *z) {
    double Mc = orc_mean_anomaly_conjunction(e, w);
    double M = Mc + 2.0 * M_PI * (t - t0) / period;
    double E = orc_kepler_E(M, e);
    double nu = 2.0 * atan2(sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E));
    double r = a_rs * (1.0 - e * cos(E));
    double sini = sqrt(fmax(0.0, 1.0 - cosi * cosi));
    *y = -r * cos(w + nu);
    *x = r * sin(w + nu) * cosi;
    *z = -r * sin(w + nu) * sini;
}

/* ------------------------------------------------------------------ */
/* Projection of the ellipsoid (Sec. 2, Eqs. dx, dy1, dy2)             */
/* ------------------------------------------------------------------ */

static void rot_x(double t, double R[9]) {
    double c = cos(t), s = sin(t);
    double m[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    memcpy(R, m, sizeof m);
}
static void rot_y(double t, double R[9]) {
    double c = cos(t), s = sin(t);
    double m[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    memcpy(R, m, sizeof m);
}
static void rot_z(double t, double R[9]) {
    double c = cos(t), s = sin(t);
    double m[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    memcpy(R, m, sizeof m);
}
static void matmul3(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

/* Semi-axes a, b, c along x', y', z'; R(zeta, eta, xi) = Rx(zeta) Ry(eta) Rz(xi)
 * with components r1..r9 (Sec. 2); the boundary of the projection is
 * x = x0 + dx cos(th), y = y0 + dy1 cos(th) + dy2 sin(th). */
void orc_projected_ellipse(double a, double b, double c, double zeta, double eta,
                           double xi, double *dx, double *dy1, double *dy2) {
    double Rx[9], Ry[9], Rz[9], T[9], R[9];
    rot_x(zeta, Rx);
    rot_y(eta, Ry);
    rot_z(xi, Rz);
    matmul3(Rx, Ry, T);
    matmul3(T, Rz, R);
    double r1 = R[0], r2 = R[1], r3 = R[2], r4 = R[3], r5 = R[4], r6 = R[5];
    double r7 = R[6], r8 = R[7], r9 = R[8];
    double a2 = a * a, b2 = b * b, c2 = c * c;
    double ddx = sqrt(a2 * r1 * r1 + b2 * r4 * r4 + c2 * r7 * r7);
    *dx = ddx;
    *dy1 = (a2 * r1 * r2 + b2 * r4 * r5 + c2 * r7 * r8) / ddx;
    *dy2 = sqrt(a2 * b2 * r9 * r9 + a2 * c2 * r6 * r6 + b2 * c2 * r3 * r3) / ddx;
}

/* Oblate spheroid b = c (Appendix A): a = polar radius R_pol = R_eq (1 - f)
 * (definition of f, Sec. 1); the fitted radius r is the geometric mean of the
 * three semi-axes (Sec. 3), so R_eq = r (1 - f)^(-1/3). */
void orc_oblate_ellipse(double k, double f, double eta, double xi, double *dx,
                        double *dy1, double *dy2) {
    double req = k / cbrt(1.0 - f);
    double rpol = req * (1.0 - f);
    orc_projected_ellipse(rpol, req, req, 0.0, eta, xi, dx, dy1, dy2);
}

/* General triaxial ellipsoid (Sec. 2: semi-axes a, b, c along x', y', z', all
 * three rotation angles active).  Parameterised like the oblate case: c is the
 * largest semi-axis, b = c (1 - g), a = c (1 - f), and k is the geometric mean of
 * the three (Sec. 3), so c = k ((1 - f)(1 - g))^(-1/3).  g = 0 is the oblate
 * spheroid, for which zeta has no effect. */
void orc_triaxial_ellipse(double k, double f, double g, double zeta, double eta, double xi,
                          double *dx, double *dy1, double *dy2) {
    double c = k / cbrt((1.0 - f) * (1.0 - g));
    orc_projected_ellipse(c * (1.0 - f), c * (1.0 - g), c, zeta, eta, xi, dx, dy1, dy2);
}

/* Tidally locked body (Appendix B): the projection at orbital angle alpha and
 * elevation beta by the printed Eqs. dx-locked, dy1-locked, dy2-locked, with
 * r1..r9 the components of R(zeta, eta, xi) as in Sec. 2. */
void orc_locked_ellipse(double a, double b, double c, double zeta, double eta, double xi,
                        double alpha, double beta, double *dx, double *dy1, double *dy2) {
    double Rx[9], Ry[9], Rz[9], T[9], R[9];
    rot_x(zeta, Rx);
    rot_y(eta, Ry);
    rot_z(xi, Rz);
    matmul3(Rx, Ry, T);
    matmul3(T, Rz, R);
    double r1 = R[0], r2 = R[1], r3 = R[2], r4 = R[3], r5 = R[4], r6 = R[5];
    double r7 = R[6], r8 = R[7], r9 = R[8];
    double sa = sin(alpha), ca = cos(alpha), sb = sin(beta), cb = cos(beta);
    double a2 = a * a, b2 = b * b, c2 = c * c;
    double u1 = sb * (r3 * ca + r2 * sa) - r1 * cb;
    double u2 = sb * (r6 * ca + r5 * sa) - r4 * cb;
    double u3 = sb * (r9 * ca + r8 * sa) - r7 * cb;
    double ddx = sqrt(a2 * u1 * u1 + b2 * u2 * u2 + c2 * u3 * u3);
    *dx = ddx;
    *dy1 = (a2 * u1 * (r3 * sa - r2 * ca) + b2 * u2 * (r6 * sa - r5 * ca) +
            c2 * u3 * (r9 * sa - r8 * ca)) / ddx;
    double w1 = r7 * sb + cb * (r9 * ca + r8 * sa);
    double w2 = r4 * sb + cb * (r6 * ca + r5 * sa);
    double w3 = r1 * sb + cb * (r3 * ca + r2 * sa);
    *dy2 = sqrt(a2 * b2 * w1 * w1 + a2 * c2 * w2 * w2 + b2 * c2 * w3 * w3) / ddx;
}

/* Kipping (2013) map from (q1, q2) to quadratic coefficients (cited in Sec. 3,
 * Table priors, note f; the formula itself is not printed in the paper). */
void orc_q_to_u(double q1, double q2, double *u1, double *u2) {
    double s = sqrt(q1);
    *u1 = 2.0 * s * q2;
    *u2 = s * (1.0 - 2.0 * q2);
}

/* ------------------------------------------------------------------ */
/* Occulted moments by iterated integration                           */
/* ------------------------------------------------------------------ */

typedef struct {
    double x0, y0, dx, dy1, dy2;
} orc_geom;

/* Inner integral over y at the abscissa x = x0 + dx cos(phi), phi in [0, pi],
 * times the Jacobian dx sin(phi) of the outer substitution.  Returns the three
 * moments Integral 1 dy, Integral sqrt(1-x^2-y^2) dy, Integral (x^2+y^2) dy over
 * the part of the vertical chord that lies in both the ellipse and the disk. */
static void inner(const orc_geom *g, double phi, double out[3]) {
    double cp = cos(phi), sp = sin(phi);
    double x = g->x0 + g->dx * cp;
    out[0] = out[1] = out[2] = 0.0;
    if (!(fabs(x) < 1.0)) return;
    double R2 = (1.0 - x) * (1.0 + x);
    double R = sqrt(R2);
    double yc = g->y0 + g->dy1 * cp, hh = g->dy2 * sp;
    double lo = fmax(yc - hh, -R), hi = fmin(yc + hh, R);
    if (!(hi > lo)) return;
    double jac = g->dx * sp;
    /* antiderivative of sqrt(R^2 - y^2): (y w + R^2 atan2(y, w))/2, w = sqrt(R^2-y^2) */
    double wl = sqrt(fmax(0.0, (R - lo) * (R + lo)));
    double wh = sqrt(fmax(0.0, (R - hi) * (R + hi)));
    double G1 = 0.5 * (hi * wh + R2 * atan2(hi, wh)) - 0.5 * (lo * wl + R2 * atan2(lo, wl));
    double I0 = hi - lo;
    double I2 = x * x * I0 + (hi * hi * hi - lo * lo * lo) / 3.0;
    out[0] = jac * I0;
    out[1] = jac * G1;
    out[2] = jac * I2;
}

static void gl_panel(const orc_geom *g, double a, double b, double q[3]) {
    double h = 0.5 * (b - a), m = 0.5 * (a + b);
    q[0] = q[1] = q[2] = 0.0;
    for (int i = 0; i < ORC_GL_N; ++i) {
        double v[3];
        inner(g, m + h * gl_x[i], v);
        q[0] += gl_w[i] * v[0];
        q[1] += gl_w[i] * v[1];
        q[2] += gl_w[i] * v[2];
    }
    q[0] *= h;
    q[1] *= h;
    q[2] *= h;
}

/* |p(th)|^2 - 1 on the projected boundary (Sec. 2; the sign tells inside/outside
 * of the stellar disk as in the snapping rule). */
static double gfun(const orc_geom *g, double th) {
    double c = cos(th), s = sin(th);
    double x = g->x0 + g->dx * c, y = g->y0 + g->dy1 * c + g->dy2 * s;
    return x * x + y * y - 1.0;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

#define ORC_MAX_IV 4096
#define ORC_NSAMP 4096

typedef struct {
    double a, b, q[3], err;
} orc_iv;

/* Moments of the occulted region E n D:
 *   out[0] = area, out[1] = Integral mu dA, out[2] = Integral r^2 dA.
 * tol is an absolute tolerance on each moment.  Returns the number of panels
 * used, or -1 if the panel budget ran out before the tolerance was met. */
int orc_occulted_moments(double x0, double y0, double dx, double dy1, double dy2,
                         double tol, double out[3]) {
    gl_init();
    orc_geom g = {x0, y0, dx, dy1, dy2};
    out[0] = out[1] = out[2] = 0.0;
    double rho = hypot(x0, y0);
    double amax = sqrt(dx * dx + dy1 * dy1 + dy2 * dy2); /* >= largest semi-axis */
    if (rho >= 1.0 + amax) return 0;

    /* Breakpoints in phi: crossings of the boundary with the limb, near-tangent
     * extrema of g, and the abscissae x = +-1. */
    double bp[72];
    int nbp = 0;
    bp[nbp++] = 0.0;
    bp[nbp++] = M_PI;
    const int Ns = ORC_NSAMP;
    double prev_th = 0.0, prev_g = gfun(&g, 0.0);
    double prev_d = gfun(&g, 1e-7) - gfun(&g, -1e-7);
    for (int i = 1; i <= Ns; ++i) {
        double th = 2.0 * M_PI * i / Ns;
        double gv = gfun(&g, th);
        double dv = gfun(&g, th + 1e-7) - gfun(&g, th - 1e-7);
        if ((prev_g < 0) != (gv < 0)) {
            double lo = prev_th, hi = th, glo = prev_g;
            for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
                double m = 0.5 * (lo + hi), gm = gfun(&g, m);
                if ((gm < 0) == (glo < 0)) { lo = m; glo = gm; } else hi = m;
            }
            double r = 0.5 * (lo + hi);
            double phi = r <= M_PI ? r : 2.0 * M_PI - r;
            if (nbp < 60) bp[nbp++] = phi;
        }
        if ((prev_d < 0) != (dv < 0)) {
            /* extremum of g: if it grazes the limb, it is a (near-)kink */
            double lo = prev_th, hi = th;
            double dlo = prev_d;
            for (int it = 0; it < 100 && hi - lo > 1e-15; ++it) {
                double m = 0.5 * (lo + hi);
                double dm = gfun(&g, m + 1e-7) - gfun(&g, m - 1e-7);
                if ((dm < 0) == (dlo < 0)) { lo = m; dlo = dm; } else hi = m;
            }
            double r = 0.5 * (lo + hi);
            double gr = gfun(&g, r);
            if (fabs(gr) < 1e-6) {
                double phi = r <= M_PI ? r : 2.0 * M_PI - r;
                if (nbp < 60) bp[nbp++] = phi;
            }
            /* two crossings inside one sampling step: the samples on both sides
             * of the extremum share a sign that the extremum does not */
            if ((prev_g < 0) == (gv < 0) && (gr < 0) != (gv < 0)) {
                double ends[2][2] = {{prev_th, r}, {r, th}};
                for (int side = 0; side < 2; ++side) {
                    double a = ends[side][0], b = ends[side][1], ga = gfun(&g, a);
                    for (int it = 0; it < 200 && b - a > 1e-17; ++it) {
                        double m = 0.5 * (a + b), gm = gfun(&g, m);
                        if ((gm < 0) == (ga < 0)) { a = m; ga = gm; } else b = m;
                    }
                    double rr = 0.5 * (a + b);
                    double phi = rr <= M_PI ? rr : 2.0 * M_PI - rr;
                    if (nbp < 60) bp[nbp++] = phi;
                }
            }
        }
        prev_th = th;
        prev_g = gv;
        prev_d = dv;
    }
    for (int s = -1; s <= 1; s += 2) {
        double c = (s - x0) / dx;
        if (c > -1.0 && c < 1.0 && nbp < 62) bp[nbp++] = acos(c);
    }
    qsort(bp, nbp, sizeof(double), cmp_double);

    orc_iv *iv = (orc_iv *)malloc(sizeof(orc_iv) * ORC_MAX_IV);
    int niv = 0;
    for (int i = 0; i + 1 < nbp; ++i) {
        if (bp[i + 1] - bp[i] <= 1e-15) continue;
        iv[niv].a = bp[i];
        iv[niv].b = bp[i + 1];
        gl_panel(&g, iv[niv].a, iv[niv].b, iv[niv].q);
        iv[niv].err = INFINITY;
        niv++;
    }
    /* Globally adaptive refinement: split the panel with the largest error
     * estimate, where the estimate is |Q(panel) - Q(left) - Q(right)|. */
    int status = 0;
    for (;;) {
        double tot = 0.0, emax = -1.0;
        int imax = -1;
        for (int i = 0; i < niv; ++i) {
            tot += iv[i].err;
            if (iv[i].err > emax) { emax = iv[i].err; imax = i; }
        }
        if (tot <= tol) break;
        if (niv + 1 >= ORC_MAX_IV) { status = -1; break; }
        orc_iv *p = &iv[imax];
        double m = 0.5 * (p->a + p->b);
        if (!(m > p->a && m < p->b)) { p->err = 0.0; continue; }
        orc_iv L = {p->a, m, {0, 0, 0}, 0}, Rr = {m, p->b, {0, 0, 0}, 0};
        gl_panel(&g, L.a, L.b, L.q);
        gl_panel(&g, Rr.a, Rr.b, Rr.q);
        double e = 0.0;
        for (int k = 0; k < 3; ++k) e = fmax(e, fabs(L.q[k] + Rr.q[k] - p->q[k]));
        L.err = Rr.err = 0.5 * e;
        *p = L;
        iv[niv++] = Rr;
    }
    /* sum small-to-large for a tidy total */
    for (int k = 0; k < 3; ++k) {
        double s = 0.0, cmp = 0.0;
        for (int i = 0; i < niv; ++i) {
            double y = iv[i].q[k] - cmp;
            double t = s + y;
            cmp = (t - s) - y;
            s = t;
        }
        out[k] = s;
    }
    free(iv);
    return status < 0 ? -1 : niv;
}

/* Evaluations whose occulted moments ran out of panels before reaching the
 * tolerance since the last orc_reset_failures().  Such an evaluation is not the
 * Sec. 2 integral to the stated accuracy, so its flux is returned as NaN and
 * counted here; the Python layer refuses results when this is non-zero. */
static int64_t orc_nfail = 0;

int64_t orc_failures(void) {
    int64_t v;
#pragma omp atomic read
    v = orc_nfail;
    return v;
}

void orc_reset_failures(void) {
#pragma omp atomic write
    orc_nfail = 0;
}

/* Relative flux of one sky configuration (Sec. 2, "Ellipsoid Transit Model").
 * I(r) = c0 + c1 mu + c2 r^2 with c0 = 1-u1-2u2, c1 = u1+2u2, c2 = u2 (the
 * quadratic law rewritten in the basis of the three integrands f_flat, f_lin,
 * f_quad), F0 = pi (1 - u1/3 - u2/6).  A planet behind the star (z > 0) does
 * not occult it (secondary eclipse is not modelled).  NaN (and a count in
 * orc_failures) if the quadrature did not reach `tol`. */
double orc_flux_sky(double x0, double y0, double z, double dx, double dy1, double dy2,
                    double u1, double u2, double tol) {
    if (z > 0.0) return 1.0;
    double m[3];
    if (orc_occulted_moments(x0, y0, dx, dy1, dy2, tol, m) < 0) {
#pragma omp atomic update
        orc_nfail += 1;
        return NAN;
    }
    if (m[0] == 0.0 && m[1] == 0.0 && m[2] == 0.0) return 1.0;
    double c0 = 1.0 - u1 - 2.0 * u2, c1 = u1 + 2.0 * u2, c2 = u2;
    double F0 = M_PI * (1.0 - u1 / 3.0 - u2 / 6.0);
    return 1.0 - (c0 * m[0] + c1 * m[1] + c2 * m[2]) / F0;
}

/* ------------------------------------------------------------------ */
/* Light-curve batch with exposure-time supersampling                  */
/* ------------------------------------------------------------------ */

/* Parameter sets in structure-of-arrays form; all arrays have n_sets entries.
 * Times: if offsets == NULL, every set uses the same n_times grid t[0..n_times);
 * otherwise set s owns t[offsets[s] .. offsets[s+1]) and out has the same layout.
 * nsuper_arr (per set) or, if NULL, nsuper_all sub-exposures per exposure.
 * Sub-exposure s of exposure j sits at t_j + ((s + 1/2)/n_s - 1/2) * exptime and
 * the exposure flux is their arithmetic mean (supersampling is not described in
 * the paper; this is the midpoint reading).  Returns 0, or -1 on bad input. */
int orc_lightcurve(int64_t n_sets, const double *t0, const double *period,
                   const double *a_rs, const double *b, const double *ecc,
                   const double *omega, const double *k, const double *f,
                   const double *eta, const double *xi, const double *u1,
                   const double *u2, const double *g, const double *zeta, int locked,
                   const double *t, const int64_t *offsets,
                   int64_t n_times, const double *exptime, const int32_t *nsuper_arr,
                   int nsuper_all, double tol, int nthreads, double *out) {
    if (n_sets < 0 || (!nsuper_arr && nsuper_all <= 0)) return -1;
    int64_t total = offsets ? offsets[n_sets] : n_sets * n_times;
    gl_init();
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < total; ++j) {
        int64_t s;
        double tj;
        if (offsets) {
            /* binary search for the owning set */
            int64_t lo = 0, hi = n_sets;
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (offsets[mid] <= j) lo = mid; else hi = mid;
            }
            s = lo;
            tj = t[j];
        } else {
            s = j / n_times;
            tj = t[j % n_times];
        }
        double dx, dy1, dy2;
        if (g || zeta)
            orc_triaxial_ellipse(k[s], f[s], g ? g[s] : 0.0, zeta ? zeta[s] : 0.0, eta[s],
                                 xi[s], &dx, &dy1, &dy2);
        else
            orc_oblate_ellipse(k[s], f[s], eta[s], xi[s], &dx, &dy1, &dy2);
        double cosi = orc_cos_inclination(b[s], a_rs[s], ecc[s], omega[s]);
        int nsuper = nsuper_arr ? nsuper_arr[s] : nsuper_all;
        if (nsuper <= 0) { out[j] = NAN; continue; }
        double acc = 0.0;
        for (int q = 0; q < nsuper; ++q) {
            double tq = tj + ((q + 0.5) / nsuper - 0.5) * exptime[s];
            double x0, y0, z;
            orc_sky_position(tq, t0[s], period[s], a_rs[s], cosi, ecc[s], omega[s], &x0,
                             &y0, &z);
            if (locked) {
                /* Appendix B with the Keplerian orbit: beta = pi/2 - i and alpha the
                 * orbital angle from conjunction, alpha = w + nu - pi/2, from
                 * r cos(alpha) = r sin(w + nu) = x0 cos i - z sin i, r sin(alpha) = y0 */
                double gg = g ? g[s] : 0.0, zz = zeta ? zeta[s] : 0.0;
                double cax = k[s] / cbrt((1.0 - f[s]) * (1.0 - gg));
                double sini = sqrt(1.0 - cosi * cosi);
                double alpha = atan2(y0, x0 * cosi - z * sini);
                double beta = 0.5 * M_PI - acos(cosi);
                orc_locked_ellipse(cax * (1.0 - f[s]), cax * (1.0 - gg), cax, zz, eta[s], xi[s],
                                   alpha, beta, &dx, &dy1, &dy2);
            }
            acc += orc_flux_sky(x0, y0, z, dx, dy1, dy2, u1[s], u2[s], tol);
        }
        out[j] = acc / nsuper;
    }
    return 0;
}

/* Relative flux for n given sky positions and shapes (OpenMP over items). */
void orc_flux_sky_batch(int64_t n, const double *x0, const double *y0, const double *z,
                        const double *k, const double *f, const double *eta, const double *xi,
                        const double *u1, const double *u2, const double *g,
                        const double *zeta, double tol, int nthreads, double *out) {
    gl_init();
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double dx, dy1, dy2;
        if (g || zeta)
            orc_triaxial_ellipse(k[i], f[i], g ? g[i] : 0.0, zeta ? zeta[i] : 0.0, eta[i],
                                 xi[i], &dx, &dy1, &dy2);
        else
            orc_oblate_ellipse(k[i], f[i], eta[i], xi[i], &dx, &dy1, &dy2);
        out[i] = orc_flux_sky(x0[i], y0[i], z[i], dx, dy1, dy2, u1[i], u2[i], tol);
    }
}

/* Number of OpenMP threads the oracle would use (for reporting). */
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
