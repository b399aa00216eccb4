"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module only draws numbers (NumPy PCG64): it holds none of the method's
arithmetic.  Limb darkening is drawn as Kipping's (q1, q2) wherever the workload
says so; each consumer converts them to (u1, u2) with its own code.  Angles are
radians, times days, radii in stellar radii.

Workloads (sizes and value distributions follow the paper's K2 setting: long
cadence near 30 min, short cadence 1 min, Sec. 3; and the fitted values of
Table fit-results):

* ``single_transit``   - one long-period transit, 1000 times over +-15 h,
                         29.4-min exposures x 15 sub-samples (15,000 evaluations)
* ``mcmc_batch``       - 256 parameter sets x 2000 shared times, 29.4-min
                         cadence, x 15 sub-samples (7.68e6 evaluations)
* ``uneven_batch``     - 4096 curves, log-uniform lengths 100..50,000, half at
                         60 s (no supersampling), half at 1764 s x 15
* ``surrogate_samples``- uniform samples of the surrogate's input box
* ``injected_curve``   - the single-transit parameters on a 3000-point grid with
                         100 ppm white noise, plus walker start positions
* ``geometry_sample``  - sky positions spread over and around the stellar limb
                         for geometry-level parity tests
"""
from __future__ import annotations

import numpy as np

MINUTE = 1.0 / 1440.0
HOUR = 1.0 / 24.0
DEG = np.pi / 180.0

#: orbital period assumed wherever a workload does not state one (HIP 41378 f, Sec. 3)
PERIOD_DAYS = 542.08
#: long-cadence exposure of 29.4 min (Kepler/K2 long cadence)
LONG_CADENCE = 29.4 * MINUTE
SHORT_CADENCE = 60.0 / 86400.0
UNEVEN_LONG_CADENCE = 1764.0 / 86400.0

PARAM_NAMES = ("t0", "period", "a_rs", "b", "ecc", "omega", "k", "f", "eta", "xi",
               "u1", "u2")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def single_transit(n_times: int = 1000, seed: int = 0) -> dict:
    """One transit with fixed parameters (no randomness; ``seed`` is unused).

    k = 0.066, f = 0.5, obliquity (eta) 30 deg, sky azimuth (xi) 45 deg,
    a/R* = 230, b = 0.2, circular orbit, P = 542 d, u1 = 0.40, u2 = 0.25;
    times uniform over +-15 h of mid-transit inclusive; 29.4-min exposures
    supersampled 15 times.
    """
    p = dict(t0=0.0, period=542.0, a_rs=230.0, b=0.2, ecc=0.0, omega=90.0 * DEG,
             k=0.066, f=0.5, eta=30.0 * DEG, xi=45.0 * DEG, u1=0.40, u2=0.25)
    params = {n: np.array([v], dtype=np.float64) for n, v in p.items()}
    t = np.linspace(-15.0 * HOUR, 15.0 * HOUR, n_times)
    return dict(params=params, t=t, offsets=None, exptime=np.array([LONG_CADENCE]),
                nsuper=15)


def _draw_sets(rng: np.random.Generator, n: int, k_range=(0.05, 0.08)) -> dict:
    """Parameter sets drawn uniformly over the MCMC box; LD as (q1, q2)."""
    return dict(
        t0=np.zeros(n),
        period=np.full(n, PERIOD_DAYS),
        a_rs=rng.uniform(150.0, 300.0, n),
        b=rng.uniform(0.0, 0.9, n),
        ecc=rng.uniform(0.0, 0.3, n),
        omega=rng.uniform(0.0, 2.0 * np.pi, n),
        k=rng.uniform(k_range[0], k_range[1], n),
        f=rng.uniform(0.0, 0.9, n),
        eta=rng.uniform(0.0, 90.0 * DEG, n),
        xi=rng.uniform(0.0, 180.0 * DEG, n),
        q1=rng.uniform(0.0, 1.0, n),
        q2=rng.uniform(0.0, 1.0, n),
    )


def mcmc_batch(n_sets: int = 256, n_times: int = 2000, seed: int = 1) -> dict:
    """Parameter sets x one shared time grid centred on the conjunction.

    t_j = t0 + (j - (n_times - 1)/2) * 29.4 min; each exposure supersampled 15x.
    Returns q1, q2 in ``params`` (no u1, u2).
    """
    rng = _rng(seed)
    params = _draw_sets(rng, n_sets)
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * LONG_CADENCE
    return dict(params=params, t=t, offsets=None,
                exptime=np.full(n_sets, LONG_CADENCE), nsuper=15)


def triaxial_batch(n_sets: int = 12, n_times: int = 400, seed: int = 51) -> dict:
    """The MCMC box with a general triaxial shape: equatorial flattening g
    U[0, 0.6] and rotation zeta U[0, pi) added to each set; k U[0.05, 0.15];
    times every 5 min over +-17 h around the conjunction (the transit), x 7."""
    rng = _rng(seed)
    params = _draw_sets(rng, n_sets, k_range=(0.05, 0.15))
    params["g"] = rng.uniform(0.0, 0.6, n_sets)
    params["zeta"] = rng.uniform(0.0, np.pi, n_sets)
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * (5.0 / 1440.0)
    return dict(params=params, t=t, offsets=None, exptime=np.full(n_sets, 5.0 / 1440.0),
                nsuper=7)


def locked_batch(n_sets: int = 12, n_times: int = 300, seed: int = 61) -> dict:
    """Close-in planets for the tidally locked mapping: P U[1, 4] d, a/R* U[3, 8],
    e U[0, 0.1], b U[0, 0.6], k U[0.08, 0.2], f U[0, 0.5], g U[0, 0.4], all three
    orientation angles uniform; 300 times every 2 min around the conjunction, x 5."""
    rng = _rng(seed)
    p = dict(t0=np.zeros(n_sets), period=rng.uniform(1.0, 4.0, n_sets),
             a_rs=rng.uniform(3.0, 8.0, n_sets), b=rng.uniform(0.0, 0.6, n_sets),
             ecc=rng.uniform(0.0, 0.1, n_sets), omega=rng.uniform(0.0, 2.0 * np.pi, n_sets),
             k=rng.uniform(0.08, 0.2, n_sets), f=rng.uniform(0.0, 0.5, n_sets),
             eta=rng.uniform(0.0, np.pi, n_sets), xi=rng.uniform(0.0, np.pi, n_sets),
             q1=rng.uniform(0.0, 1.0, n_sets), q2=rng.uniform(0.0, 1.0, n_sets),
             g=rng.uniform(0.0, 0.4, n_sets), zeta=rng.uniform(0.0, np.pi, n_sets))
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * (2.0 / 1440.0)
    return dict(params=p, t=t, offsets=None, exptime=np.full(n_sets, 2.0 / 1440.0), nsuper=5)


def uneven_batch(n_curves: int = 4096, seed: int = 2, min_len: int = 100,
                 max_len: int = 50000) -> dict:
    """Curves of log-uniform length; even curves 60-s cadence (nsuper 1), odd
    curves 1764-s cadence (nsuper 15).  Each curve's grid is centred on
    t0 + U(-0.5, 0.5) d.  Times are laid out back to back (CSR ``offsets``)."""
    rng = _rng(seed)
    params = _draw_sets(rng, n_curves, k_range=(0.01, 0.2))
    lengths = np.rint(np.exp(rng.uniform(np.log(min_len), np.log(max_len), n_curves)))
    lengths = lengths.astype(np.int64)
    cadence = np.where(np.arange(n_curves) % 2 == 0, SHORT_CADENCE, UNEVEN_LONG_CADENCE)
    nsuper = np.where(np.arange(n_curves) % 2 == 0, 1, 15).astype(np.int32)
    centre = rng.uniform(-0.5, 0.5, n_curves)
    offsets = np.zeros(n_curves + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    t = np.empty(int(offsets[-1]))
    for s in range(n_curves):
        n = lengths[s]
        t[offsets[s]:offsets[s + 1]] = centre[s] + (np.arange(n) - 0.5 * (n - 1)) * cadence[s]
    return dict(params=params, t=t, offsets=offsets, exptime=cadence.copy(),
                nsuper=nsuper)


def surrogate_samples(n: int, seed: int = 3) -> dict:
    """Uniform samples of the surrogate's input box: sky x, y in [-1.2, 1.2],
    k in [0.01, 0.2], f in [0, 0.9], projected-ellipse angle psi in [0, pi),
    cos(axis tilt) in [0, 1], q1, q2 in [0, 1]; eta = arccos(cos(axis tilt)) is
    the tilt angle itself (the box is uniform in its cosine)."""
    rng = _rng(seed)
    d = dict(
        x=rng.uniform(-1.2, 1.2, n), y=rng.uniform(-1.2, 1.2, n),
        k=rng.uniform(0.01, 0.2, n), f=rng.uniform(0.0, 0.9, n),
        psi=rng.uniform(0.0, np.pi, n), cos_tilt=rng.uniform(0.0, 1.0, n),
        q1=rng.uniform(0.0, 1.0, n), q2=rng.uniform(0.0, 1.0, n),
    )
    d["eta"] = np.arccos(d["cos_tilt"])
    return d


def injected_curve(n_times: int = 3000, n_walkers: int = 1024, noise_ppm: float = 100.0,
                   seed: int = 4) -> dict:
    """Truth = the single-transit parameters; 3000 exposures of 29.4 min centred
    on the transit, supersampled 15x; white Gaussian noise of ``noise_ppm`` drawn
    here (to be added to a model flux by the caller); walker starts scattered
    around the truth."""
    rng = _rng(seed)
    truth = single_transit()["params"]
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * LONG_CADENCE
    noise = rng.normal(0.0, noise_ppm * 1e-6, n_times)
    walkers = {}
    scale = dict(t0=1e-3, period=0.0, a_rs=1.0, b=0.01, ecc=0.0, omega=0.0, k=1e-4,
                 f=0.02, eta=0.02, xi=0.02, u1=0.01, u2=0.01)
    for name in PARAM_NAMES:
        walkers[name] = truth[name][0] + scale[name] * rng.standard_normal(n_walkers)
    walkers["f"] = np.clip(walkers["f"], 0.0, 0.9)
    walkers["b"] = np.abs(walkers["b"])
    return dict(truth=truth, t=t, exptime=LONG_CADENCE, nsuper=15, noise=noise,
                walkers=walkers)


def geometry_sample(n: int, seed: int = 10, k_range=(0.01, 0.2), f_max: float = 0.9,
                    band: float = 1.3) -> dict:
    """Sky geometries for geometry-level parity: shape (k, f, eta, xi) uniform,
    LD (q1, q2) uniform, centre distance rho in [0, 1 + band*2.2*k] (2.2 k
    bounds the planet's largest radius for f <= 0.9), position angle uniform.  A
    third of the samples crowd the limb: rho = 1 + 2.2 k U(-band, band)."""
    rng = _rng(seed)
    k = rng.uniform(k_range[0], k_range[1], n)
    f = rng.uniform(0.0, f_max, n)
    reach = 2.2 * k
    rho = rng.uniform(0.0, 1.0 + band * reach)
    limb = rng.uniform(0.0, 1.0, n) < 1.0 / 3.0
    rho[limb] = np.abs(1.0 + reach[limb] * rng.uniform(-band, band, limb.sum()))
    ang = rng.uniform(0.0, 2.0 * np.pi, n)
    return dict(x0=rho * np.cos(ang), y0=rho * np.sin(ang), z=-np.ones(n) * 100.0,
                k=k, f=f, eta=rng.uniform(0.0, 90.0 * DEG, n),
                xi=rng.uniform(0.0, 180.0 * DEG, n), q1=rng.uniform(0, 1, n),
                q2=rng.uniform(0, 1, n))


def tangency_sample(n: int, seed: int = 21, k_range=(0.01, 0.25), f_max: float = 0.9) -> dict:
    """Shapes and LD as in geometry_sample, a direction angle, a side (inner:
    the planet's outline reaches just past the limb from inside; outer: from
    outside) and a log-uniform offset delta in [1e-8, 1e-3] stellar radii."""
    rng = _rng(seed)
    return dict(k=rng.uniform(k_range[0], k_range[1], n), f=rng.uniform(0.0, f_max, n),
                eta=rng.uniform(0.0, 90.0 * DEG, n), xi=rng.uniform(0.0, 180.0 * DEG, n),
                q1=rng.uniform(0, 1, n), q2=rng.uniform(0, 1, n),
                ang=rng.uniform(0.0, 2.0 * np.pi, n), inner=rng.uniform(0, 1, n) < 0.5,
                delta=10.0 ** rng.uniform(-8.0, -3.0, n))


def extreme_orbits(n_sets: int = 48, n_times: int = 3000, seed: int = 11) -> dict:
    """Short-period, eccentric, close-in orbits with long exposures: P U[0.5, 3.5] d,
    a/R* U[2.5, 10.5], e U[0, 0.8], b U[0, 0.45], k U[0.02, 0.22], exposure
    U[0.01, 0.11] d x 7; 3000 shared times every 0.0021 d around t0.  They exercise
    transit windows that cover the whole orbit, several transits per curve and
    exposures too long for a low-order time expansion of the orbit."""
    rng = _rng(seed)
    p = dict(
        t0=rng.uniform(-0.2, 0.2, n_sets), period=rng.uniform(0.5, 3.5, n_sets),
        a_rs=rng.uniform(2.5, 10.5, n_sets), b=rng.uniform(0.0, 0.45, n_sets),
        ecc=rng.uniform(0.0, 0.8, n_sets), omega=rng.uniform(0.0, 2.0 * np.pi, n_sets),
        k=rng.uniform(0.02, 0.22, n_sets), f=rng.uniform(0.0, 0.9, n_sets),
        eta=rng.uniform(0.0, 90.0 * DEG, n_sets), xi=rng.uniform(0.0, 180.0 * DEG, n_sets),
        q1=rng.uniform(0.0, 1.0, n_sets), q2=rng.uniform(0.0, 1.0, n_sets))
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * 0.0021
    return dict(params=p, t=t, offsets=None, exptime=rng.uniform(0.01, 0.11, n_sets),
                nsuper=7)
