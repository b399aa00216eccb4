"""The (mu, nu) reparameterisation of Appendix A and the stretch-move sweep, in
plain FP64 numpy: the oracle of the library's gl_munu_* and gl_ensemble_* kernels.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

Appendix A: for an oblate spheroid, flux depends on (f, eta) only through
mu = (f - 1)^2 + f (f - 2) cos(2 eta).  A second coordinate nu in [0, 1] places f
between its least value for that mu, f_min = 1 - sqrt((mu + 1)/2), and 1:
f = f_min + (1 - f_min) nu.  The joint density p(mu, nu) printed there makes the
implied prior on (f, eta) uniform in f and proportional to cos(eta), and is
drawn by inverse transform from two uniforms (u, w).

The stretch move is Goodman and Weare (2010): each half of an ensemble proposes
along the line through a walker and a random member of the other half,
Y = X_j + z (X_k - X_j), z from g(z) ~ 1/sqrt(z) on [1/a, a], and accepts with
probability min(1, z^(D-1) p(Y) / p(X_k)).
"""
from __future__ import annotations

import numpy as np


def mu_of(f, eta):
    """mu(f, eta) (Appendix A, Eq. mu)."""
    return (f - 1.0) ** 2 + f * (f - 2.0) * np.cos(2.0 * eta)


def f_min(mu):
    return 1.0 - np.sqrt((mu + 1.0) / 2.0)


def nu_of(f, eta):
    """nu(f, eta) as printed in Appendix A."""
    c2 = np.cos(2.0 * eta)
    q = f * (f - 2.0)
    num = 2.0 + 2.0 * q * np.cos(eta) ** 2 + (f - 1.0) * np.sqrt(4.0 + 2.0 * q * (1.0 + c2))
    return num / (2.0 + q * (1.0 + c2))


def f_eta_of(mu, nu):
    """Inverse map: f = f_min + (1 - f_min) nu, then eta in [0, pi/2] from mu."""
    fm = f_min(mu)
    f = fm + (1.0 - fm) * nu
    q = f * (f - 2.0)
    c2 = np.where(q != 0.0, (mu - (f - 1.0) ** 2) / np.where(q != 0.0, q, 1.0), 1.0)
    eta = 0.5 * np.arccos(np.clip(c2, -1.0, 1.0))
    return f, eta


def det_jacobian(f, eta):
    """det d(mu, nu)/d(f, eta) as printed in Appendix A."""
    q = f * (f - 2.0)
    return 2.0 ** 1.5 * q * np.sin(2.0 * eta) / np.sqrt(2.0 + q * (1.0 + np.cos(2.0 * eta)))


def p_munu(mu, nu):
    """Joint density p(mu, nu) (Appendix A, Eq. mu-nu-joint-density)."""
    return 2.0 ** -1.5 * (nu * (nu - 2.0) * (mu * (nu - 1.0) ** 2 + nu * (nu - 2.0) - 1.0)) ** -0.5


def p_nu(nu):
    """Marginal of nu."""
    s = nu * (2.0 - nu)
    return 1.0 / (s + np.sqrt(s))


def cdf_nu(nu):
    return (nu - np.sqrt(nu * (2.0 - nu))) / (nu - 1.0)


def nu_of_u(u):
    """Inverse of cdf_nu."""
    return u * u / (u * u - 2.0 * u + 2.0)


def cdf_mu_given_nu(mu, nu):
    s = np.sqrt(nu * (2.0 - nu))
    return (1.0 + s) * (2.0 - np.sqrt(2.0 - 2.0 * mu * (nu - 1.0) ** 2 - 2.0 * nu * (nu - 2.0))) \
        / (2.0 * (nu - 1.0) ** 2)


def mu_of_w(w, nu):
    """Inverse of cdf_mu_given_nu in mu."""
    s = np.sqrt(nu * (2.0 - nu))
    return (4.0 * w + 4.0 * (w * w - w) * s + 2.0 * (nu * (nu - 2.0) - 1.0) * w * w
            - (nu - 1.0) ** 2) / (nu - 1.0) ** 2


def prior_draw(u, w):
    """(mu, nu) from two uniforms by inverse transform (nu first, then mu | nu)."""
    nu = nu_of_u(u)
    return mu_of_w(w, nu), nu


# ---------------------------------------------------------------- ensemble sweep
def stretch_half(walkers, logpost, active, other, r_z, r_j, r_u, lnpost_fn, a=2.0):
    """One half-step: the walkers `active` propose along lines through members of
    `other` (partner = other[floor(r_j * len(other))]), z = ((a - 1) r_z + 1)^2 / a,
    accept if log(r_u) < (D - 1) log z + lnpost(Y) - lnpost(X), never if
    lnpost(Y) = -inf, always (for a finite lnpost(Y)) if lnpost(X) = -inf.  Returns the new
    walkers, log posteriors, accepted mask and the proposals' log posteriors."""
    walkers = np.array(walkers, dtype=np.float64, copy=True)
    logpost = np.array(logpost, dtype=np.float64, copy=True)
    d = walkers.shape[1]
    z = ((a - 1.0) * r_z + 1.0) ** 2 / a
    partner = np.asarray(other)[np.minimum((r_j * len(other)).astype(np.int64), len(other) - 1)]
    prop = walkers[partner] + z[:, None] * (walkers[active] - walkers[partner])
    lp_new = lnpost_fn(prop)
    lp_old = logpost[active]
    # Acceptance probability min(1, z^(D-1) p(Y)/p(X)) (Goodman and Weare 2010)
    # with the cases of zero density written out, so that no NaN decides a move:
    # a proposal outside the prior (p(Y) = 0) is never taken; a walker outside
    # the prior (p(X) = 0) takes any proposal inside it; otherwise the log test.
    new_in = lp_new > -np.inf
    old_in = lp_old > -np.inf
    with np.errstate(invalid="ignore"):
        log_r = (d - 1) * np.log(z) + np.where(new_in & old_in, lp_new - lp_old, 0.0)
    ok = new_in & (~old_in | (np.log(r_u) < log_r))
    walkers[np.asarray(active)[ok]] = prop[ok]
    logpost[np.asarray(active)[ok]] = lp_new[ok]
    return walkers, logpost, ok, lp_new
