"""Pins of the (mu, nu) oracle (Appendix A) and of its stretch-move sweep, against
mathematics computed by other routes (no GPU): the round trip of the map; the
printed Jacobian determinant against finite differences; p(mu, nu) |det J| equal
to cos(eta) (the target prior); the printed marginal and conditional CDFs and
their inverses against numerical integration; inverse-transform draws that are
uniform in f and cos-distributed in eta (KS tests); equal mu giving the same
projected ellipse at equal R_eq; the acceptance rule of the stretch move."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from oracle import munu as M


def _box(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.01, 0.99, n), rng.uniform(0.01, 0.5 * math.pi - 0.01, n)


def test_round_trip():
    f, eta = _box(5000, 1)
    mu, nu = M.mu_of(f, eta), M.nu_of(f, eta)
    assert np.all((mu >= -1) & (mu <= 1) & (nu >= 0) & (nu <= 1))
    f2, eta2 = M.f_eta_of(mu, nu)
    np.testing.assert_allclose(f2, f, atol=1e-13)
    np.testing.assert_allclose(eta2, eta, atol=1e-9)
    assert np.all(f >= M.f_min(mu) - 1e-15)


def test_jacobian_determinant_against_finite_differences():
    f, eta = _box(500, 2)
    h = 1e-6

    def mn(a, b):
        return np.array([M.mu_of(a, b), M.nu_of(a, b)])

    J = np.empty((f.size, 2, 2))
    J[:, :, 0] = ((mn(f + h, eta) - mn(f - h, eta)) / (2 * h)).T
    J[:, :, 1] = ((mn(f, eta + h) - mn(f, eta - h)) / (2 * h)).T
    np.testing.assert_allclose(np.abs(np.linalg.det(J)), np.abs(M.det_jacobian(f, eta)),
                               rtol=1e-6)


def test_joint_density_gives_the_cosine_prior():
    f, eta = _box(2000, 3)
    dens = M.p_munu(M.mu_of(f, eta), M.nu_of(f, eta)) * np.abs(M.det_jacobian(f, eta))
    np.testing.assert_allclose(dens, np.cos(eta), rtol=1e-10)


@pytest.mark.parametrize("nu", [0.05, 0.3, 0.6, 0.95])
def test_marginal_and_conditional_cdfs(nu):
    val, _ = integrate.quad(lambda m: M.p_munu(m, nu), -1.0, 1.0, limit=200)
    assert abs(val - M.p_nu(nu)) < 1e-9 * M.p_nu(nu)
    cum, _ = integrate.quad(M.p_nu, 0.0, nu)
    assert abs(cum - M.cdf_nu(nu)) < 1e-9
    for mu in (-0.8, -0.2, 0.3, 0.9):
        c, _ = integrate.quad(lambda m: M.p_munu(m, nu) / M.p_nu(nu), -1.0, mu, limit=200)
        assert abs(c - M.cdf_mu_given_nu(mu, nu)) < 1e-9
    u = np.linspace(0.001, 0.999, 41)
    np.testing.assert_allclose(M.cdf_nu(M.nu_of_u(u)), u, atol=1e-12)
    np.testing.assert_allclose(M.cdf_mu_given_nu(M.mu_of_w(u, nu), nu), u, atol=1e-12)


def test_inverse_transform_draws_have_the_target_prior():
    rng = np.random.default_rng(4)
    mu, nu = M.prior_draw(rng.uniform(size=200_000), rng.uniform(size=200_000))
    f, eta = M.f_eta_of(mu, nu)
    assert stats.kstest(f, "uniform").pvalue > 1e-3
    assert stats.kstest(eta, lambda x: np.sin(np.clip(x, 0, math.pi / 2))).pvalue > 1e-3


def test_equal_mu_gives_the_same_projection_at_equal_r_eq():
    """mu is what the projected ellipse sees: (f1, eta1) and (f2, eta2) with the
    same mu and any nu project identically when R_eq is the same (Appendix A)."""
    f, eta = _box(60, 5)
    rng = np.random.default_rng(6)
    for f1, e1 in zip(f, eta):
        mu = M.mu_of(f1, e1)
        f2, e2 = M.f_eta_of(mu, rng.uniform(0.02, 0.98))
        xi = rng.uniform(0, math.pi)
        a = oracle.projected_ellipse(0.1 * (1 - f1), 0.1, 0.1, 0.0, e1, xi)
        b = oracle.projected_ellipse(0.1 * (1 - f2), 0.1, 0.1, 0.0, e2, xi)
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)


def test_stretch_half_acceptance_rule():
    """With a flat posterior the move is accepted iff u < z^(D-1); proposals lie on
    the line through the walker and its partner."""
    rng = np.random.default_rng(7)
    w = rng.normal(size=(64, 5))
    lp = np.zeros(64)
    act, oth = np.arange(0, 64, 2), np.arange(1, 64, 2)
    rz, rj, ru = (rng.uniform(size=32) for _ in range(3))
    nw, nlp, ok, _ = M.stretch_half(w, lp, act, oth, rz, rj, ru, lambda y: np.zeros(len(y)))
    z = ((2.0 - 1.0) * rz + 1.0) ** 2 / 2.0
    np.testing.assert_array_equal(ok, ru < z ** 4)
    partner = oth[(rj * 32).astype(int)]
    for i, k in enumerate(act):
        if ok[i]:
            expect = w[partner[i]] + z[i] * (w[k] - w[partner[i]])
            np.testing.assert_allclose(nw[k], expect, rtol=1e-15)
        else:
            np.testing.assert_array_equal(nw[k], w[k])
    np.testing.assert_array_equal(nw[oth], w[oth])


def test_stretch_half_zero_density_cases():
    """min(1, z^(D-1) p(Y)/p(X)) with zero densities: a proposal outside the prior
    is never taken, a walker outside the prior takes any proposal inside it, and
    neither case goes through a NaN (warnings are errors here)."""
    rng = np.random.default_rng(8)
    w = rng.normal(size=(8, 3))
    lp = np.array([-np.inf, 0.0, -np.inf, 0.0, 0.0, 0.0, -np.inf, 0.0])
    act, oth = np.arange(0, 8, 2), np.arange(1, 8, 2)
    rz = np.full(4, 0.5)
    rj = np.array([0.1, 0.3, 0.6, 0.9])
    ru = np.full(4, 0.999999)   # only a forced acceptance passes the log test
    inside = np.array([1.0, -np.inf, -np.inf, 5.0])   # lp(Y) per active walker
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        nw, nlp, ok, lp_new = M.stretch_half(w, lp, act, oth, rz, rj, ru,
                                             lambda y: inside.copy())
    # walker 0: outside -> finite proposal: taken; walker 2: both outside: kept;
    # walker 4: inside -> proposal outside: kept; walker 6: outside -> finite: taken
    np.testing.assert_array_equal(ok, [True, False, False, True])
    np.testing.assert_array_equal(nlp[act], [1.0, -np.inf, 0.0, 5.0])
