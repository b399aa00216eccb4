"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test checks an oracle function against mathematics the paper or the
textbook fixes, computed here by a different route:

* Kepler solve       - residual of Kepler's equation; scipy's brentq; E = M at e = 0
* sky position       - the paper's circular formulas (Sec. 2); vis-viva energy and
                       Kepler's second law (areal velocity) along an eccentric orbit;
                       (x, y) = (b, 0) at conjunction
* projection         - brute-force support function of the rotated ellipsoid surface
                       (Sec. 2, Eqs. dx, dy1, dy2); oblate invariance in zeta and the
                       projected semi-axes (Appendix A)
* occulted moments   - Green's theorem with the integrands f_flat, f_lin, f_quad of
                       Sec. 2 integrated in 30-digit arithmetic (mpmath) on the
                       ellipse and limb arcs; circle-circle lens area; quasi-Monte
                       Carlo; full-inside area and second moment
* flux               - spherical planet (f = 0, or spin along the line of sight) vs a
                       radial 1-D integral; total eclipse gives zero; out of transit
                       is exactly one; mirror symmetry; monotone in k
* degeneracy         - the worked example of Appendix A (tests/golden)
* supersampling      - midpoint rule converges to the exposure average at O(n^-2)
* Kipping map        - inverse relations and physical validity over [0,1]^2
"""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, optimize
from scipy.stats import qmc

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Kepler
@pytest.mark.parametrize("e", [0.0, 0.01, 0.3, 0.7, 0.95])
def test_kepler_residual_and_brentq(e):
    for M in np.linspace(-7.0, 7.0, 57):
        E = oracle.kepler_E(M, e)
        assert abs(E - e * math.sin(E) - M) < 4e-15 * (1 + abs(M))
        Mr = math.remainder(M, 2 * math.pi)
        Eb = optimize.brentq(lambda x: x - e * math.sin(x) - Mr, Mr - e - 1e-9,
                             Mr + e + 1e-9, xtol=1e-16, rtol=9e-16)
        assert abs((E - (M - Mr)) - Eb) < 1e-13


def test_kepler_special_values():
    for M in (0.0, math.pi, -math.pi, 2.5):
        assert oracle.kepler_E(M, 0.0) == M
    assert abs(oracle.kepler_E(math.pi, 0.6) - math.pi) < 1e-15
    assert oracle.kepler_E(0.0, 0.6) == 0.0


# ---------------------------------------------------------------- orbit
def _rotmat(axis, t):
    c, s = math.cos(t), math.sin(t)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def test_circular_orbit_matches_paper_formulas():
    """Sec. 2, Eq. coord-map: the planet centre sits at -Ry(-beta) Rx(alpha) (0,0,d),
    i.e. x0 = d cos(alpha) sin(beta), y0 = d sin(alpha)."""
    P, a, b, t0 = 10.0, 12.0, 0.4, 1.25
    cosi = oracle.cos_inclination(b, a, 0.0, math.pi / 2)
    beta = math.pi / 2 - math.acos(cosi)
    for t in np.linspace(t0 - 3.0, t0 + 3.0, 31):
        alpha = 2 * math.pi * (t - t0) / P
        ref = -_rotmat("y", -beta) @ _rotmat("x", alpha) @ np.array([0.0, 0.0, a])
        x, y, z = oracle.sky_position(t, t0, P, a, cosi, 0.0, math.pi / 2)
        assert abs(x - a * math.cos(alpha) * math.sin(beta)) < 1e-13
        assert abs(y - a * math.sin(alpha)) < 1e-13
        np.testing.assert_allclose([x, y, z], ref, atol=1e-12)


@pytest.mark.parametrize("e,w", [(0.3, 0.7), (0.6, 4.0), (0.1, -1.2)])
def test_eccentric_orbit_invariants(e, w):
    P, a, b, t0 = 7.0, 20.0, 0.3, 0.5
    cosi = oracle.cos_inclination(b, a, e, w)
    x, y, z = oracle.sky_position(t0, t0, P, a, cosi, e, w)
    assert abs(x - b) < 1e-12 and abs(y) < 1e-12 and z < 0   # conjunction, in front
    n = 2 * math.pi / P
    mu = n * n * a ** 3
    h = 1e-5
    for t in np.linspace(0.0, P, 23):
        r0 = np.array(oracle.sky_position(t, t0, P, a, cosi, e, w))
        rp = np.array(oracle.sky_position(t + h, t0, P, a, cosi, e, w))
        rm = np.array(oracle.sky_position(t - h, t0, P, a, cosi, e, w))
        v = (rp - rm) / (2 * h)
        r = np.linalg.norm(r0)
        assert abs(0.5 * v @ v - mu / r + mu / (2 * a)) < 1e-6 * mu / a      # vis-viva
        assert abs(np.linalg.norm(np.cross(r0, v)) - n * a * a * math.sqrt(1 - e * e)) \
            < 1e-6 * n * a * a                                                # areal velocity
        r1 = np.array(oracle.sky_position(t + P, t0, P, a, cosi, e, w))
        np.testing.assert_allclose(r1, r0, atol=1e-9)


# ---------------------------------------------------------------- projection
def _ellipsoid_support(a, b, c, zeta, eta, xi, u, n=400):
    """max over the ellipsoid surface of u . (x, y), brute force."""
    R = _rotmat("x", zeta) @ _rotmat("y", eta) @ _rotmat("z", xi)
    th, ph = np.meshgrid(np.linspace(0, np.pi, n), np.linspace(0, 2 * np.pi, 2 * n))
    pts = np.stack([a * np.sin(th) * np.cos(ph), b * np.sin(th) * np.sin(ph),
                    c * np.cos(th)], -1).reshape(-1, 3)
    sky = pts @ R          # x = R^T x'  (rows: R^T applied to each point)
    return np.max(sky[:, :2] @ u)


@pytest.mark.parametrize("abc,angles", [((0.05, 0.08, 0.11), (0.3, 1.1, -0.7)),
                                        ((0.1, 0.1, 0.06), (1.2, 0.4, 2.0)),
                                        ((0.03, 0.07, 0.07), (0.0, 0.9, 0.3))])
def test_projection_support_function(abc, angles):
    dx, dy1, dy2 = oracle.projected_ellipse(*abc, *angles)
    thg = np.linspace(0, 2 * np.pi, 20001)
    for phi in np.linspace(0, np.pi, 13):
        u = np.array([math.cos(phi), math.sin(phi)])
        ell = np.max(u[0] * dx * np.cos(thg) + u[1] * (dy1 * np.cos(thg) + dy2 * np.sin(thg)))
        brute = _ellipsoid_support(*abc, *angles, u)
        assert abs(ell - brute) < 2e-4 * max(abc)


def _locked_support(a, b, c, zeta, eta, xi, alpha, beta, u, n=400):
    """Support function for the tidally locked mapping of Appendix B, brute force:
    body coordinates x' = R(zeta, eta, xi) (Rx(-alpha) Ry(beta) x + (0, 0, d)), so a
    surface point x' sits at x = (R Rx(-alpha) Ry(beta))^T x' from the centre."""
    M = (_rotmat("x", zeta) @ _rotmat("y", eta) @ _rotmat("z", xi)
         @ _rotmat("x", -alpha) @ _rotmat("y", beta))
    th, ph = np.meshgrid(np.linspace(0, np.pi, n), np.linspace(0, 2 * np.pi, 2 * n))
    pts = np.stack([a * np.sin(th) * np.cos(ph), b * np.sin(th) * np.sin(ph),
                    c * np.cos(th)], -1).reshape(-1, 3)
    sky = pts @ M
    return np.max(sky[:, :2] @ u)


@pytest.mark.parametrize("abc,angles,orbit", [((0.05, 0.08, 0.11), (0.3, 1.1, -0.7), (0.4, 0.1)),
                                              ((0.12, 0.09, 0.06), (1.2, 0.4, 2.0), (-0.9, 0.3)),
                                              ((0.07, 0.07, 0.03), (0.0, 0.9, 0.3), (2.5, -0.2))])
def test_locked_projection_support_function(abc, angles, orbit):
    """The printed Eqs. dx-locked, dy1-locked, dy2-locked against a brute-force
    support function of the body in the locked orientation (Appendix B)."""
    dx, dy1, dy2 = oracle.locked_ellipse(*abc, *angles, *orbit)
    thg = np.linspace(0, 2 * np.pi, 20001)
    for phi in np.linspace(0, np.pi, 13):
        u = np.array([math.cos(phi), math.sin(phi)])
        ell = np.max(u[0] * dx * np.cos(thg) + u[1] * (dy1 * np.cos(thg) + dy2 * np.sin(thg)))
        assert abs(ell - _locked_support(*abc, *angles, *orbit, u)) < 2e-4 * max(abc)


def test_locked_projection_special_cases():
    """alpha = beta = 0 is the unlocked projection; a sphere projects to a circle
    of its radius at every orbital angle."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        abc = rng.uniform(0.02, 0.2, 3)
        ang = rng.uniform(-3, 3, 3)
        np.testing.assert_allclose(oracle.locked_ellipse(*abc, *ang, 0.0, 0.0),
                                   oracle.projected_ellipse(*abc, *ang), rtol=1e-12, atol=1e-16)
        r = abc[0]
        dx, dy1, dy2 = oracle.locked_ellipse(r, r, r, *ang, *rng.uniform(-3, 3, 2))
        np.testing.assert_allclose([dx, dy1, dy2], [r, 0.0, r], rtol=1e-12, atol=1e-15)


def test_oblate_projection_axes_and_zeta_invariance():
    rng = np.random.default_rng(0)
    for _ in range(40):
        req, f = rng.uniform(0.01, 0.4), rng.uniform(0, 0.95)
        eta, xi, zeta = rng.uniform(-2, 2, 3)
        rpol = req * (1 - f)
        base = oracle.projected_ellipse(rpol, req, req, 0.0, eta, xi)
        other = oracle.projected_ellipse(rpol, req, req, zeta, eta, xi)
        np.testing.assert_allclose(other, base, rtol=1e-13, atol=1e-16)
        dx, dy1, dy2 = base
        L = np.array([[dx, 0.0], [dy1, dy2]])
        ev = np.sort(np.linalg.eigvalsh(L @ L.T))
        minor2 = req * req * (1 - (2 * f - f * f) * math.cos(eta) ** 2)
        np.testing.assert_allclose(ev, [minor2, req * req], rtol=1e-12)


def test_triaxial_ellipse_closed_forms():
    """Triaxial shape (c largest, b = c (1-g), a = c (1-f), abc = k^3): with every
    angle zero the sky axes are a along x and b along y; with eta = 90 deg the x'
    axis points along the line of sight and the projected area is pi b c for any
    zeta, xi; g = 0 is the oblate spheroid whatever zeta."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        k, f, g = rng.uniform(0.02, 0.3), rng.uniform(0, 0.9), rng.uniform(0, 0.9)
        c = k / ((1 - f) * (1 - g)) ** (1.0 / 3.0)
        a, b = c * (1 - f), c * (1 - g)
        np.testing.assert_allclose(a * b * c, k ** 3, rtol=1e-13)
        dx, dy1, dy2 = oracle.triaxial_ellipse(k, f, g, 0.0, 0.0, 0.0)
        np.testing.assert_allclose([dx, dy1, dy2], [a, 0.0, b], rtol=1e-13, atol=1e-17)
        zeta, xi = rng.uniform(-3, 3, 2)
        dx, dy1, dy2 = oracle.triaxial_ellipse(k, f, g, zeta, 0.5 * math.pi, xi)
        np.testing.assert_allclose(dx * dy2, b * c, rtol=1e-12)
        eta = rng.uniform(-3, 3)
        base = oracle.oblate_ellipse(k, f, eta, xi)
        np.testing.assert_allclose(oracle.triaxial_ellipse(k, f, 0.0, zeta, eta, xi), base,
                                   rtol=1e-12, atol=1e-16)


def test_oblate_ellipse_uses_mean_radius():
    k, f = 0.066, 0.5
    dx, dy1, dy2 = oracle.oblate_ellipse(k, f, 0.0, 0.0)   # spin axis along x
    req = k / (1 - f) ** (1 / 3)
    assert abs(dx - req * (1 - f)) < 1e-15 and abs(dy1) < 1e-16 and abs(dy2 - req) < 1e-15
    assert abs((dx * dy2 * dy2) ** (1 / 3) - k) < 1e-15   # geometric mean of (Rpol, Req, Req)


# ---------------------------------------------------------------- moments (Green's theorem pin)
mp.mp.dps = 30


def _green_moments(x0, y0, dx, dy1, dy2):
    """Moments by Green's theorem: the line integrals of f_flat, f_lin, f_quad
    (Sec. 2) along the ellipse arcs inside the disk and the limb arcs inside
    the ellipse, each integrated by mpmath tanh-sinh in 30 digits."""
    x0, y0, dx, dy1, dy2 = (mp.mpf(v) for v in (x0, y0, dx, dy1, dy2))

    def ell(th):
        c, s = mp.cos(th), mp.sin(th)
        return x0 + dx * c, y0 + dy1 * c + dy2 * s, -dx * s, -dy1 * s + dy2 * c

    def limb(la):
        return mp.cos(la), mp.sin(la), -mp.sin(la), mp.cos(la)

    def integrands(x, y, xp, yp):
        r2 = x * x + y * y
        ff = (x * yp - y * xp) / 2
        fl = mp.mpf(2) / 3 * (1 - mp.power(mp.fabs(1 - r2), mp.mpf(3) / 2)) * ff / r2
        fq = (x * (x * x / 3 + y * y) * yp - y * (x * x + y * y / 3) * xp) / 2
        return ff, fl, fq

    def g(th):
        x, y, _, _ = ell(th)
        return x * x + y * y - 1

    ths = np.linspace(0, 2 * np.pi, 20001)
    gv = np.array([float(g(t)) for t in ths[::10]])
    ths = ths[::10]
    roots = []
    for i in range(len(ths) - 1):
        if (gv[i] < 0) != (gv[i + 1] < 0):
            roots.append(mp.findroot(g, (mp.mpf(ths[i]), mp.mpf(ths[i + 1])), solver="anderson"))
    out = [mp.mpf(0)] * 3
    if not roots:
        if gv[0] < 0:
            pieces = [(ell, mp.mpf(0), 2 * mp.pi)]
        else:
            return np.zeros(3)
    else:
        pieces = []
        m = len(roots)
        for i in range(m):
            a, b = roots[i], roots[(i + 1) % m] + (2 * mp.pi if i + 1 == m else 0)
            if g((a + b) / 2) < 0:
                pieces.append((ell, a, b))
        lam = sorted(mp.atan2(ell(r)[1], ell(r)[0]) for r in roots)
        for i in range(m):
            a, b = lam[i], lam[(i + 1) % m] + (2 * mp.pi if i + 1 == m else 0)
            cm, sm = mp.cos((a + b) / 2), mp.sin((a + b) / 2)
            v1 = (cm - x0) / dx
            v2 = (sm - y0 - dy1 * v1) / dy2
            if v1 * v1 + v2 * v2 < 1:
                pieces.append((limb, a, b))
    for curve, a, b in pieces:
        for k in range(3):
            out[k] += mp.quad(lambda s: integrands(*curve(s))[k], [a, b])
    return np.array([float(v) for v in out])


def _cases():
    rng = np.random.default_rng(42)
    cases = []
    while len(cases) < 10:
        k, f = rng.uniform(0.02, 0.2), rng.uniform(0, 0.9)
        eta, xi = rng.uniform(0, np.pi / 2), rng.uniform(0, np.pi)
        dx, dy1, dy2 = oracle.oblate_ellipse(k, f, eta, xi)
        req = k / (1 - f) ** (1 / 3)
        rho = 1 + req * rng.uniform(-0.9, 0.9)
        ang = rng.uniform(0, 2 * np.pi)
        cases.append((rho * math.cos(ang), rho * math.sin(ang), dx, dy1, dy2))
    # full inside, four crossings, and centre outside the disk
    cases.append((0.3, -0.2, *oracle.oblate_ellipse(0.1, 0.6, 0.5, 1.0)))
    cases.append((0.0, 0.975, 0.42, 0.0, 0.02))
    cases.append((1.05, 0.1, *oracle.oblate_ellipse(0.15, 0.3, 1.0, 0.2)))
    return cases


@pytest.mark.parametrize("case", _cases())
def test_moments_vs_green_theorem(case):
    ref = _green_moments(*case)
    got = oracle.occulted_moments(*case)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-14)


def test_four_crossings_case_really_has_four():
    x0, y0, dx, dy1, dy2 = 0.0, 0.975, 0.42, 0.0, 0.02
    th = np.linspace(0, 2 * np.pi, 100001)
    g = (x0 + dx * np.cos(th)) ** 2 + (y0 + dy1 * np.cos(th) + dy2 * np.sin(th)) ** 2 - 1
    assert np.count_nonzero(np.diff(np.sign(g))) == 4


def _lens_area(p, rho):
    """Circle (radius p, centre distance rho) overlap with the unit disk."""
    if rho >= 1 + p:
        return 0.0
    if rho <= 1 - p:
        return math.pi * p * p
    k0 = math.acos((p * p + rho * rho - 1) / (2 * p * rho))
    k1 = math.acos((1 - p * p + rho * rho) / (2 * rho))
    return p * p * k0 + k1 - 0.5 * math.sqrt(4 * rho * rho - (1 + rho * rho - p * p) ** 2)


@pytest.mark.parametrize("p", [0.01, 0.07, 0.2, 0.4])
def test_circle_area_is_lens_area(p):
    for rho in np.linspace(0.0, 1 + p * 1.01, 29):
        m = oracle.occulted_moments(rho * 0.6, rho * 0.8, p, 0.0, p)
        assert abs(m[0] - _lens_area(p, rho)) < 2e-14


def test_near_tangent_crossing_pair_in_any_orientation():
    """A circle overlapping the limb by a sliver of depth ~5e-8: its two crossings
    are closer than the oracle's sampling step, in every orientation."""
    mp.mp.dps = 40
    for p, depth in [(0.41376514184929669, 4.8e-8), (0.2, 1e-9), (0.05, 3e-7)]:
        z = 1.0 - p + depth
        Z, P = mp.mpf(z), mp.mpf(p)
        k0 = mp.acos((P * P + Z * Z - 1) / (2 * P * Z))
        k1 = mp.acos((1 - P * P + Z * Z) / (2 * Z))
        exact = float(P * P * k0 + k1 - mp.sqrt(4 * Z * Z - (1 + Z * Z - P * P) ** 2) / 2)
        for ang in np.linspace(0.1, 6.2, 7):
            m = oracle.occulted_moments(z * math.cos(ang), z * math.sin(ang), p, 0.0, p)
            assert abs(m[0] - exact) < 1e-14
    mp.mp.dps = 30


def test_full_inside_closed_forms():
    rng = np.random.default_rng(3)
    for _ in range(30):
        k, f = rng.uniform(0.01, 0.2), rng.uniform(0, 0.9)
        eta, xi = rng.uniform(0, np.pi / 2), rng.uniform(0, np.pi)
        dx, dy1, dy2 = oracle.oblate_ellipse(k, f, eta, xi)
        req = k / (1 - f) ** (1 / 3)
        x0, y0 = rng.uniform(-0.4, 0.4, 2)
        m = oracle.occulted_moments(x0, y0, dx, dy1, dy2)
        area = math.pi * req * req * math.sqrt(1 - (2 * f - f * f) * math.cos(eta) ** 2)
        assert abs(m[0] - area) < 1e-15
        # second moment of an ellipse about the origin: area (|c|^2 + (a^2 + b^2)/4)
        minor2 = req * req * (1 - (2 * f - f * f) * math.cos(eta) ** 2)
        assert abs(m[2] - area * (x0 * x0 + y0 * y0 + (req * req + minor2) / 4)) < 1e-15


def test_moments_quasi_monte_carlo():
    rng = np.random.default_rng(11)
    sob = qmc.Sobol(2, scramble=True, seed=5)
    pts = sob.random_base2(21)
    for _ in range(3):
        k, f = rng.uniform(0.1, 0.2), rng.uniform(0.2, 0.8)
        dx, dy1, dy2 = oracle.oblate_ellipse(k, f, rng.uniform(0, 1.5), rng.uniform(0, 3))
        x0, y0 = 0.9, 0.3
        hy = math.hypot(dy1, dy2)
        X = x0 - dx + 2 * dx * pts[:, 0]
        Y = y0 - hy + 2 * hy * pts[:, 1]
        v1 = (X - x0) / dx
        v2 = (Y - y0 - dy1 * v1) / dy2
        r2 = X * X + Y * Y
        inside = (v1 * v1 + v2 * v2 < 1) & (r2 < 1)
        box = 4 * dx * hy
        est = box * np.array([inside.mean(), (np.sqrt(np.clip(1 - r2, 0, None)) * inside).mean(),
                              (r2 * inside).mean()])
        got = oracle.occulted_moments(x0, y0, dx, dy1, dy2)
        np.testing.assert_allclose(got, est, rtol=3e-4, atol=1e-7)


# ---------------------------------------------------------------- flux
def _sphere_flux_radial(p, rho, u1, u2):
    """Spherical planet: the occulted flux as a 1-D integral over stellar radius
    r of I(r) times the length of the circle of radius r inside the planet."""
    def arc(r):
        if r <= 0:
            return 0.0
        if r <= p - rho:
            return 2 * math.pi * r
        if r <= rho - p or r >= rho + p:
            return 0.0
        return 2 * r * math.acos(min(1, max(-1, (r * r + rho * rho - p * p) / (2 * r * rho))))

    def intens(r):
        mu = math.sqrt(max(0.0, 1 - r * r))
        return 1 - u1 * (1 - mu) - u2 * (1 - mu) ** 2

    pts = sorted({abs(rho - p), min(1.0, rho + p)})
    val, _ = integrate.quad(lambda r: intens(r) * arc(r), 0.0, min(1.0, rho + p),
                            points=pts, epsabs=1e-15, epsrel=1e-13, limit=400)
    F0, _ = integrate.quad(lambda r: 2 * math.pi * r * intens(r), 0, 1, epsabs=1e-15)
    return 1 - val / F0


@pytest.mark.parametrize("p,u1,u2", [(0.066, 0.4, 0.25), (0.15, 0.1, 0.6), (0.01, 0.8, -0.1)])
def test_sphere_matches_radial_integral(p, u1, u2):
    for rho in list(np.linspace(0, 1 + 0.99 * p, 17)) + [1 - p + 1e-4, 1 + p - 1e-4]:
        # f = 0: circle of radius k
        dx, dy1, dy2 = oracle.oblate_ellipse(p, 0.0, 0.7, 1.1)
        got = oracle.flux_sky(rho, 0.0, -1.0, dx, dy1, dy2, u1, u2)
        assert abs(got - _sphere_flux_radial(p, rho, u1, u2)) < 1e-12
        # spin along the line of sight: circle of radius R_eq
        f = 0.4
        dx, dy1, dy2 = oracle.oblate_ellipse(p, f, math.pi / 2, 0.3)
        req = p / (1 - f) ** (1 / 3)
        got = oracle.flux_sky(0.0, rho, -1.0, dx, dy1, dy2, u1, u2)
        assert abs(got - _sphere_flux_radial(req, rho, u1, u2)) < 1e-12


def test_total_eclipse_gives_zero_and_uniform_disk():
    # a circle of radius 2 centred on the star covers it: flux must be 0 for any LD
    for u1, u2 in [(0.0, 0.0), (0.4, 0.25), (1.0, -0.3)]:
        assert abs(oracle.flux_sky(0.0, 0.0, -1.0, 2.0, 0.0, 2.0, u1, u2)) < 1e-14
    # uniform disk: flux = 1 - area/pi
    dx, dy1, dy2 = oracle.oblate_ellipse(0.1, 0.5, 0.3, 0.9)
    m = oracle.occulted_moments(0.97, 0.1, dx, dy1, dy2)
    assert abs(oracle.flux_sky(0.97, 0.1, -1.0, dx, dy1, dy2, 0.0, 0.0) - (1 - m[0] / math.pi)) < 1e-15


def test_out_of_transit_is_exactly_one():
    dx, dy1, dy2 = oracle.oblate_ellipse(0.1, 0.5, 0.3, 0.9)
    req = 0.1 / 0.5 ** (1 / 3)
    for ang in np.linspace(0, 2 * np.pi, 9):
        r = 1 + req + 1e-9
        assert oracle.flux_sky(r * math.cos(ang), r * math.sin(ang), -1, dx, dy1, dy2, .4, .2) == 1.0
    assert oracle.flux_sky(0.1, 0.1, +5.0, dx, dy1, dy2, 0.4, 0.2) == 1.0   # behind the star
    p = dict(t0=[0.0], period=[542.0], a_rs=[230.0], b=[0.2], ecc=[0.0], omega=[math.pi / 2],
             k=[0.066], f=[0.5], eta=[0.5], xi=[0.8], u1=[0.4], u2=[0.25])
    t = np.array([-3.0, -1.5, 1.5, 3.0, 271.0])     # days: far from the transit, and the occultation
    out = oracle.lightcurve(p, t, 29.4 / 1440, 15)
    assert np.all(out == 1.0)


def test_mirror_symmetry():
    base = dict(t0=[0.0], period=[542.0], a_rs=[230.0], b=[0.3], ecc=[0.0],
                omega=[math.pi / 2], k=[0.08], f=[0.4], eta=[0.6], u1=[0.4], u2=[0.25])
    tau = np.linspace(0.05, 0.45, 9)
    t = np.concatenate([-tau, tau])
    for xi in (0.0, math.pi / 2):
        out = oracle.lightcurve({**base, "xi": [xi]}, t, 0.02, 3)[0]
        np.testing.assert_allclose(out[:9], out[9:], atol=2e-15)
    xi = 0.7
    plus = oracle.lightcurve({**base, "xi": [xi]}, t, 0.02, 3)[0]
    minus = oracle.lightcurve({**base, "xi": [-xi]}, t, 0.02, 3)[0]
    np.testing.assert_allclose(plus[9:], minus[:9], atol=2e-15)
    assert np.max(np.abs(plus[9:] - plus[:9])) > 1e-6    # asymmetric when misaligned


def test_deficit_monotone_in_k():
    for rho in (0.2, 0.9, 1.02):
        prev = -1.0
        for k in np.linspace(0.01, 0.2, 20):
            dx, dy1, dy2 = oracle.oblate_ellipse(k, 0.3, 0.4, 0.5)
            d = 1 - oracle.flux_sky(rho, 0.05, -1, dx, dy1, dy2, 0.4, 0.25)
            assert d >= prev
            prev = d


# ---------------------------------------------------------------- degeneracy (Appendix A)
def _mu_paper(f, eta):
    return (f - 1) ** 2 + f * (f - 2) * math.cos(2 * eta)


def test_degeneracy_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "degeneracy_example.json")))
    c1, c2 = g["cases"]
    f1, eta1 = c1["f"], c1["eta"]
    f2 = c2["f_num"] / c2["f_den"]
    eta2 = 0.5 * math.acos(c2["cos_2eta_num"] / c2["cos_2eta_den"])
    assert abs(math.degrees(eta2) - 23.28) < 0.01
    assert abs(_mu_paper(f1, eta1) - g["mu"]) < 1e-15
    assert abs(_mu_paper(f2, eta2) - g["mu"]) < 1e-15
    req = g["equatorial_radius_in_figure"] * 0.1
    e1 = oracle.projected_ellipse(req * (1 - f1), req, req, 0.0, eta1, 0.4)
    e2 = oracle.projected_ellipse(req * (1 - f2), req, req, 0.0, eta2, 0.4)
    np.testing.assert_allclose(e1, e2, atol=1e-16)
    L = np.array([[e1[0], 0], [e1[1], e1[2]]])
    sv = np.linalg.svd(L, compute_uv=False)
    assert abs(sv[1] / sv[0] - g["projected_minor_over_major_in_figure"]) < 1e-14
    # identical light curves at equal equatorial radius (mean radius differs)
    base = dict(t0=[0.0], period=[542.0], a_rs=[230.0], b=[0.2], ecc=[0.0],
                omega=[math.pi / 2], xi=[0.4], u1=[0.4], u2=[0.25])
    t = np.linspace(-0.5, 0.5, 41)
    lc1 = oracle.lightcurve({**base, "k": [req * (1 - f1) ** (1 / 3)], "f": [f1],
                             "eta": [eta1]}, t, 0.02, 5)
    lc2 = oracle.lightcurve({**base, "k": [req * (1 - f2) ** (1 / 3)], "f": [f2],
                             "eta": [eta2]}, t, 0.02, 5)
    assert np.max(np.abs(lc1 - 1)) > 1e-3
    np.testing.assert_allclose(lc1, lc2, atol=1e-14)


# ---------------------------------------------------------------- supersampling
def test_supersampling_converges_to_exposure_average():
    p = dict(t0=[0.0], period=[542.0], a_rs=[230.0], b=[0.2], ecc=[0.0],
             omega=[math.pi / 2], k=[0.066], f=[0.5], eta=[0.52], xi=[0.79],
             u1=[0.4], u2=[0.25])
    cosi = oracle.cos_inclination(0.2, 230.0, 0.0, math.pi / 2)
    dx, dy1, dy2 = oracle.oblate_ellipse(0.066, 0.5, 0.52, 0.79)
    texp = 29.4 / 1440
    tc = -0.385     # an exposure across ingress

    def flux(t):
        x, y, z = oracle.sky_position(t, 0.0, 542.0, 230.0, cosi, 0.0, math.pi / 2)
        return oracle.flux_sky(x, y, z, dx, dy1, dy2, 0.4, 0.25)

    exact, _ = integrate.quad(flux, tc - texp / 2, tc + texp / 2, epsabs=1e-14, limit=200)
    exact /= texp
    e1 = abs(oracle.lightcurve(p, [tc], texp, 15)[0, 0] - exact)
    e3 = abs(oracle.lightcurve(p, [tc], texp, 45)[0, 0] - exact)
    assert e1 > 0 and e3 < e1 / 5          # O(n^-2): a factor 9 for 3x more samples
    assert abs(oracle.lightcurve(p, [tc], texp, 1)[0, 0] - flux(tc)) < 1e-15


# ---------------------------------------------------------------- Kipping map
def test_kipping_inverse_and_validity():
    for q1 in np.linspace(0.01, 1, 12):
        for q2 in np.linspace(0, 1, 12):
            u1, u2 = oracle.q_to_u(q1, q2)
            assert abs((u1 + u2) ** 2 - q1) < 1e-14
            if u1 + u2 > 0:
                assert abs(u1 / (2 * (u1 + u2)) - q2) < 1e-14
            mu = np.linspace(0, 1, 101)
            inten = 1 - u1 * (1 - mu) - u2 * (1 - mu) ** 2
            assert inten.min() >= -1e-14 and np.all(np.diff(inten) >= -1e-14)


# ---------------------------------------------------------------- failure reporting
def test_quadrature_failure_is_loud():
    """An evaluation whose adaptive quadrature cannot reach its tolerance (here an
    impossible tolerance of 0) is not the Sec. 2 integral: the flux is NaN, it is
    counted, and the default (strict) wrappers raise instead of returning it."""
    dx, dy1, dy2 = oracle.oblate_ellipse(0.1, 0.3, 0.4, 0.7)
    geo = (0.95, 0.2, -1.0, dx, dy1, dy2, 0.4, 0.25)
    with pytest.raises(oracle.OracleQuadratureError):
        oracle.flux_sky(*geo, tol=0.0)
    v = oracle.flux_sky(*geo, tol=0.0, strict=False)
    assert math.isnan(v) and oracle.failures() == 1
    # the same geometry at the default tolerance is fine and resets the counter
    assert 0.0 < oracle.flux_sky(*geo) < 1.0 and oracle.failures() == 0
    arr = dict(x0=[0.95, 3.0], y0=[0.2, 0.0], z=[-1.0, -1.0], k=[0.1, 0.1], f=[0.3, 0.3],
               eta=[0.4, 0.4], xi=[0.7, 0.7], u1=[0.4, 0.4], u2=[0.25, 0.25])
    with pytest.raises(oracle.OracleQuadratureError):
        oracle.flux_sky_batch(**arr, tol=0.0)
    out = oracle.flux_sky_batch(**arr, tol=0.0, strict=False)
    assert math.isnan(out[0]) and out[1] == 1.0 and oracle.failures() == 1
    p = {n: np.array([v]) for n, v in dict(t0=0.0, period=10.0, a_rs=20.0, b=0.3, ecc=0.0,
                                            omega=math.pi / 2, k=0.1, f=0.3, eta=0.4, xi=0.7,
                                            u1=0.4, u2=0.25).items()}
    t = np.array([-0.04, 0.0, 3.0])
    with pytest.raises(oracle.OracleQuadratureError):
        oracle.lightcurve(p, t, 0.01, 3, tol=0.0)
    lc = oracle.lightcurve(p, t, 0.01, 3, tol=0.0, strict=False)[0]
    assert np.isnan(lc[:2]).all() and lc[2] == 1.0
