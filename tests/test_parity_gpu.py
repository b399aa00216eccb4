"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (max |delta flux| over every compared exposure): FP64 path 1e-10,
FP32-compensated path 1e-7.  Out-of-transit exposures must be exactly 1.0 on
both paths.  The full-size workloads run on the GPU exactly as the benchmark
launches them; the oracle checks a seeded sample of their parameter sets.
"""
import math

import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

from _common import PARAM_NAMES, nsuper_array, oracle_params, product_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {binding.GL_FP64: 1e-10, binding.GL_FP32C: 1e-7}
PRECS = [binding.GL_FP64, binding.GL_FP32C]


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.array(a, copy=True)).to(device="cuda", dtype=dtype).contiguous()


def _run(ctx, wl, prec, device=True):
    p = product_params(wl)
    n_sets = len(p["t0"])
    exptime = np.ascontiguousarray(np.broadcast_to(wl["exptime"], (n_sets,)), dtype=np.float64)
    ns = nsuper_array(wl, n_sets)
    t = np.ascontiguousarray(wl["t"], dtype=np.float64)
    offsets = wl.get("offsets")
    n_total = n_sets * len(t) if offsets is None else int(offsets[-1])
    if device:
        dp = {k: _dev(v) for k, v in p.items()}
        out = torch.empty(n_total, dtype=torch.float64, device="cuda")
        ctx.lightcurve(dp, _dev(t), out, _dev(exptime), nsuper=_dev(ns, torch.int32),
                       offsets=None if offsets is None else _dev(offsets, torch.int64),
                       precision=prec)
        torch.cuda.synchronize()
        assert ctx.sync() == binding.GL_OK
        return out.cpu().numpy()
    out = np.empty(n_total)
    ctx.lightcurve(p, t, out, exptime, nsuper=ns,
                   offsets=None if offsets is None else np.ascontiguousarray(offsets, np.int64),
                   precision=prec)
    return out


def _compare(got, ref, prec):
    err = np.max(np.abs(got - ref)) if got.size else 0.0
    assert err <= TOL[prec], f"max |dflux| {err:.3e} > {TOL[prec]:.0e}"
    out = ref == 1.0
    assert np.all(got[out] == 1.0), "out-of-transit exposures must be exactly 1"
    return err


# ---------------------------------------------------------------- single transit
@pytest.fixture(scope="module")
def single_ref():
    import oracle
    wl = inputs.single_transit()
    return wl, oracle.lightcurve(oracle_params(wl), wl["t"], wl["exptime"], wl["nsuper"])[0]


@pytest.mark.parametrize("prec", PRECS)
def test_single_transit(ctx, single_ref, prec):
    wl, ref = single_ref
    got = _run(ctx, wl, prec)
    assert np.mean(ref < 1.0) > 0.5     # most of the window is in transit
    _compare(got, ref, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_host_and_device_buffers_agree(ctx, prec):
    wl = inputs.single_transit()
    a = _run(ctx, wl, prec, device=True)
    b = _run(ctx, wl, prec, device=False)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_central_chords_of_strongly_flattened_planets(ctx, prec):
    """Chords through the middle of the disk with f up to 0.9 and the spin axis near
    the sky plane: whole-ellipse items near the centre, where g(th) may have two
    maxima (the separate queue, two mapped arcs), and the single-maximum items
    around them (Newton's maximum); both precisions against the oracle."""
    import oracle
    n = 6
    params = dict(t0=np.zeros(n), period=np.full(n, 542.0), a_rs=np.full(n, 230.0),
                  b=np.array([0.0, 0.02, 0.05, 0.0, 0.1, 0.03]), ecc=np.zeros(n),
                  omega=np.full(n, 0.5 * math.pi),
                  k=np.array([0.1, 0.15, 0.2, 0.12, 0.18, 0.2]),
                  f=np.array([0.6, 0.8, 0.7, 0.85, 0.5, 0.9]),
                  eta=np.array([0.0, 0.1, 0.2, 0.05, 0.0, 0.3]),
                  xi=np.array([0.0, 0.5, 1.0, 1.5, 2.0, 2.5]),
                  u1=np.full(n, 0.4), u2=np.full(n, 0.25))
    t = np.linspace(-0.25, 0.25, 80)   # +- 6 h about mid-transit
    wl = dict(params=params, t=t, offsets=None, exptime=np.full(n, 10.0 / 1440.0), nsuper=5)
    ref = oracle.lightcurve(oracle_params(wl), t, wl["exptime"], 5)
    got = _run(ctx, wl, prec).reshape(n, -1)
    assert np.mean(ref < 1.0) > 0.5
    _compare(got.ravel(), np.asarray(ref).ravel(), prec)


# ---------------------------------------------------------------- MCMC batch
@pytest.fixture(scope="module")
def mcmc():
    import oracle
    wl = inputs.mcmc_batch()
    rng = np.random.default_rng(101)
    idx = np.sort(rng.choice(256, 12, replace=False))
    ref = oracle.lightcurve(oracle_params(wl, idx), wl["t"], wl["exptime"][idx], wl["nsuper"])
    return wl, idx, ref


@pytest.mark.parametrize("prec", PRECS)
def test_mcmc_batch_full_size_sampled(ctx, mcmc, prec):
    wl, idx, ref = mcmc
    got = _run(ctx, wl, prec).reshape(256, -1)
    _compare(got[idx].ravel(), ref.ravel(), prec)
    assert np.all(np.isfinite(got))


# ---------------------------------------------------------------- uneven CSR batch
@pytest.fixture(scope="module")
def uneven():
    import oracle
    wl = inputs.uneven_batch()
    off = wl["offsets"]
    lengths = np.diff(off)
    rng = np.random.default_rng(202)
    short = np.flatnonzero(lengths < 3000)
    longer = np.flatnonzero((lengths >= 3000) & (lengths < 20000))
    idx = np.sort(np.concatenate([rng.choice(short, 16, replace=False),
                                  rng.choice(longer, 4, replace=False)]))
    sub_off = np.zeros(idx.size + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum(lengths[idx])
    t_sub = np.concatenate([wl["t"][off[s]:off[s + 1]] for s in idx])
    ref = oracle.lightcurve(oracle_params(wl, idx), t_sub, wl["exptime"][idx],
                            wl["nsuper"][idx], offsets=sub_off)
    return wl, idx, ref


@pytest.mark.parametrize("prec", PRECS)
def test_uneven_batch_full_size_sampled(ctx, uneven, prec):
    wl, idx, ref = uneven
    got = _run(ctx, wl, prec)
    off = wl["offsets"]
    got_sub = np.concatenate([got[off[s]:off[s + 1]] for s in idx])
    _compare(got_sub, ref, prec)
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("prec", PRECS)
def test_uneven_batch_every_kernel_variant(ctx, uneven, prec):
    """The full CSR batch under each exposure-kernel block and quadrature variant
    (the autotuner's axes): the sampled curves stay within tolerance of the
    oracle and every variant gives the same bits."""
    wl, idx, ref = uneven
    off = wl["offsets"]
    first = None
    try:
        for eb, q in ((256, 4), (64, 8), (64, 4), (256, 8)):
            ctx.configure(prec, quad_ctas=q, exposure_block=eb)
            got = _run(ctx, wl, prec)
            _compare(np.concatenate([got[off[s]:off[s + 1]] for s in idx]), ref, prec)
            if first is None:
                first = got
            else:
                assert np.array_equal(got, first)
    finally:
        ctx.configure(prec)


# ---------------------------------------------------------------- extreme orbits
@pytest.fixture(scope="module")
def extreme():
    import oracle
    wl = inputs.extreme_orbits()
    ref = oracle.lightcurve(oracle_params(wl), wl["t"], wl["exptime"], wl["nsuper"])
    return wl, ref


@pytest.mark.parametrize("prec", PRECS)
def test_extreme_orbits(ctx, extreme, prec):
    wl, ref = extreme
    got = _run(ctx, wl, prec).reshape(ref.shape)
    assert np.mean(ref < 1.0) > 0.05      # several transits per curve
    _compare(got.ravel(), ref.ravel(), prec)


# ---------------------------------------------------------------- geometry level
@pytest.fixture(scope="module")
def geometry():
    import oracle
    g = inputs.geometry_sample(30000)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(g["q1"], g["q2"])])
    g["u1"], g["u2"] = u[:, 0].copy(), u[:, 1].copy()
    ref = oracle.flux_sky_batch(g["x0"], g["y0"], g["z"], g["k"], g["f"], g["eta"], g["xi"],
                                g["u1"], g["u2"])
    return g, ref


@pytest.mark.parametrize("prec", PRECS)
def test_geometry_parity(ctx, geometry, prec):
    g, ref = geometry
    u1, u2 = binding.gl_q_to_u(g["q1"], g["q2"])
    args = [_dev(g[n]) for n in ("x0", "y0", "z", "k", "f", "eta", "xi")] + [_dev(u1), _dev(u2)]
    out = torch.empty(len(ref), dtype=torch.float64, device="cuda")
    ctx.flux_sky(*args, out, precision=prec)
    got = out.cpu().numpy()
    assert np.mean((ref < 1) & (ref > 0)) > 0.5
    _compare(got, ref, prec)


def _extreme_distance(x0, y0, dx, dy1, dy2, largest):
    """Largest (or smallest) distance from the disk centre over the outline
    x0 + dx cos th, y0 + dy1 cos th + dy2 sin th: a 2048-angle grid, then golden-
    section refinement around the best grid angle (vectorised over cases)."""
    th = np.linspace(0.0, 2.0 * np.pi, 2048, endpoint=False)[None, :]
    def dist(t):
        return np.hypot(x0[:, None] + dx[:, None] * np.cos(t),
                        y0[:, None] + dy1[:, None] * np.cos(t) + dy2[:, None] * np.sin(t))
    d = dist(th)
    i = np.argmax(d, axis=1) if largest else np.argmin(d, axis=1)
    lo = (th[0, i] - 2.0 * np.pi / 2048)[:, None]
    hi = (th[0, i] + 2.0 * np.pi / 2048)[:, None]
    r = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(45):
        a = hi - r * (hi - lo)
        b = lo + r * (hi - lo)
        fa, fb = dist(a), dist(b)
        better_a = fa > fb if largest else fa < fb
        hi = np.where(better_a, b, hi)
        lo = np.where(better_a, lo, a)
    return dist(0.5 * (lo + hi))[:, 0]


@pytest.fixture(scope="module")
def tangency():
    """Centres where the outline reaches delta past the limb: from inside
    (largest distance 1 + delta) or from outside (smallest distance 1 - delta),
    found by bisection on the centre distance along the sampled direction.  Two
    close crossings bound a thin sliver there; rounding decides the details."""
    import oracle
    g = inputs.tangency_sample(3000)
    n = len(g["k"])
    ell = np.array([oracle.oblate_ellipse(*a) for a in zip(g["k"], g["f"], g["eta"], g["xi"])])
    dx, dy1, dy2 = ell[:, 0], ell[:, 1], ell[:, 2]
    c, s_ = np.cos(g["ang"]), np.sin(g["ang"])
    target = np.where(g["inner"], 1.0 + g["delta"], 1.0 - g["delta"])
    req = np.maximum(np.abs(dx), np.hypot(dy1, dy2)) * 1.5
    lo = np.where(g["inner"], 1.0 - 2.0 * req, 1.0 - 0.5 * req)
    hi = np.where(g["inner"], 1.0 + 0.5 * req, 1.0 + 2.0 * req)
    inner = g["inner"]
    for _ in range(52):
        mid = 0.5 * (lo + hi)
        val = np.empty(n)
        val[inner] = _extreme_distance(mid[inner] * c[inner], mid[inner] * s_[inner], dx[inner],
                                       dy1[inner], dy2[inner], largest=True)
        val[~inner] = _extreme_distance(mid[~inner] * c[~inner], mid[~inner] * s_[~inner],
                                        dx[~inner], dy1[~inner], dy2[~inner], largest=False)
        up = val < target   # the extreme distance grows with the centre distance
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    rho = 0.5 * (lo + hi)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(g["q1"], g["q2"])])
    geo = dict(x0=rho * c, y0=rho * s_, z=-np.ones(n), k=g["k"], f=g["f"], eta=g["eta"],
               xi=g["xi"], u1=u[:, 0].copy(), u2=u[:, 1].copy())
    ref = oracle.flux_sky_batch(*[geo[q] for q in ("x0", "y0", "z", "k", "f", "eta", "xi",
                                                    "u1", "u2")])
    return geo, ref


@pytest.mark.parametrize("prec", PRECS)
def test_near_tangency_parity(ctx, tangency, prec):
    g, ref = tangency
    args = [_dev(g[n]) for n in ("x0", "y0", "z", "k", "f", "eta", "xi", "u1", "u2")]
    out = torch.empty(len(ref), dtype=torch.float64, device="cuda")
    ctx.flux_sky(*args, out, precision=prec)
    got = out.cpu().numpy()
    assert np.mean((ref < 1) & (ref > 0)) > 0.95
    _compare(got, ref, prec)


@pytest.fixture(scope="module")
def large_flat():
    """Large, strongly flattened planets (R_eq up to ~0.5), the shapes that need
    more FP32 quadrature nodes."""
    import oracle
    g = inputs.geometry_sample(20000, seed=23, k_range=(0.15, 0.25), f_max=0.9)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(g["q1"], g["q2"])])
    g["u1"], g["u2"] = u[:, 0].copy(), u[:, 1].copy()
    ref = oracle.flux_sky_batch(g["x0"], g["y0"], g["z"], g["k"], g["f"], g["eta"], g["xi"],
                                g["u1"], g["u2"])
    return g, ref


@pytest.mark.parametrize("prec", PRECS)
def test_large_flattened_planets_parity(ctx, large_flat, prec):
    g, ref = large_flat
    args = [_dev(g[n]) for n in ("x0", "y0", "z", "k", "f", "eta", "xi", "u1", "u2")]
    out = torch.empty(len(ref), dtype=torch.float64, device="cuda")
    ctx.flux_sky(*args, out, precision=prec)
    _compare(out.cpu().numpy(), ref, prec)


# ---------------------------------------------------------------- spherical planet
# the FP32C spherical base meets the same 1e-7 as the oblate path (worst case on
# this sample, large planets p ~ 0.4 near the limb: 6.3e-8)
SPHERE_TOL = {binding.GL_FP64: 1e-10, binding.GL_FP32C: 1e-7}


@pytest.fixture(scope="module")
def sphere_geometry():
    import oracle
    g = inputs.geometry_sample(20000, seed=12, k_range=(0.005, 0.45), f_max=0.0)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(g["q1"], g["q2"])])
    g["u1"], g["u2"] = u[:, 0].copy(), u[:, 1].copy()
    zeros = np.zeros_like(g["k"])
    ref = oracle.flux_sky_batch(g["x0"], g["y0"], g["z"], g["k"], zeros, zeros, zeros,
                                g["u1"], g["u2"])
    return g, ref


@pytest.mark.parametrize("prec", PRECS)
def test_sphere_parity(ctx, sphere_geometry, prec):
    g, ref = sphere_geometry
    u1, u2 = binding.gl_q_to_u(g["q1"], g["q2"])
    out = torch.empty(len(ref), dtype=torch.float64, device="cuda")
    ctx.flux_sphere(*[_dev(g[n]) for n in ("x0", "y0", "z", "k")], _dev(u1), _dev(u2), out,
                    precision=prec)
    got = out.cpu().numpy()
    assert np.mean((ref < 1) & (ref > 0)) > 0.5
    err = np.max(np.abs(got - ref))
    assert err <= SPHERE_TOL[prec], f"{err:.3e}"
    assert np.all(got[ref == 1.0] == 1.0)


# ---------------------------------------------------------------- worked example
def test_degeneracy_example_on_gpu(ctx):
    """Appendix A: f = 1/2, eta = 0 and f = 2/3, eta = arccos(11/16)/2 at equal R_eq."""
    req = 0.1
    eta2 = 0.5 * math.acos(11 / 16)
    base = dict(t0=0.0, period=542.0, a_rs=230.0, b=0.2, ecc=0.0, omega=math.pi / 2, xi=0.4,
                u1=0.4, u2=0.25)
    p = {n: np.array([base[n]] * 2) for n in base}
    p["k"] = np.array([req * 0.5 ** (1 / 3), req * (1 / 3) ** (1 / 3)])
    p["f"] = np.array([0.5, 2 / 3])
    p["eta"] = np.array([0.0, eta2])
    p = {n: p[n] for n in PARAM_NAMES}
    t = np.linspace(-0.5, 0.5, 401)
    out = np.empty(2 * t.size)
    ctx.lightcurve(p, t, out, np.full(2, 0.02), nsuper_all=5, precision=binding.GL_FP64)
    a, b = out[:t.size], out[t.size:]
    assert np.max(1 - a) > 1e-3
    assert np.max(np.abs(a - b)) < 1e-13


# ---------------------------------------------------------------- edge cases
def test_empty_batches(ctx):
    p = {n: np.zeros(0) for n in PARAM_NAMES}
    ctx.lightcurve(p, np.zeros(0), np.zeros(0), np.zeros(0), nsuper_all=3)
    wl = inputs.single_transit()
    pp = product_params(wl)
    ctx.lightcurve(pp, np.zeros(0), np.zeros(0), np.array([0.02]), nsuper_all=3)
    assert ctx.sync() == binding.GL_OK


def test_ragged_csr_with_empty_curves(ctx):
    import oracle
    wl = inputs.uneven_batch(n_curves=6, max_len=400)
    lengths = np.diff(wl["offsets"])
    lengths[[1, 4]] = 0
    off = np.zeros(7, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    t = np.concatenate([wl["t"][wl["offsets"][s]:wl["offsets"][s] + lengths[s]] for s in range(6)])
    wl2 = dict(wl, t=t, offsets=off)
    ref = oracle.lightcurve(oracle_params(wl2), t, wl["exptime"], wl["nsuper"], offsets=off)
    for prec in PRECS:
        _compare(_run(ctx, wl2, prec), ref, prec)


def test_invalid_set_gives_nan_and_status(ctx):
    wl = inputs.mcmc_batch(n_sets=4, n_times=50)
    p = product_params(wl)
    p["ecc"] = p["ecc"].copy()
    p["ecc"][2] = 1.5          # unbound orbit: invalid
    out = np.empty(4 * 50)
    ctx.lightcurve(p, wl["t"], out, wl["exptime"], nsuper_all=15)
    out = out.reshape(4, 50)
    assert np.all(np.isnan(out[2]))
    assert np.all(np.isfinite(out[[0, 1, 3]]))
    assert ctx.sync() == binding.GL_ENUMERIC
    assert ctx.sync() == binding.GL_OK     # sticky until read


def test_bad_arguments_are_rejected(ctx):
    wl = inputs.single_transit()
    p = product_params(wl)
    out = np.empty(1000)
    with pytest.raises(binding.GLError) as e:
        ctx.lightcurve(p, wl["t"], out, np.array([0.02]), nsuper_all=0)
    assert e.value.code == binding.GL_EINVAL
    bad = dict(p)
    bad["k"] = None
    with pytest.raises((binding.GLError, TypeError)):
        ctx.lightcurve(bad, wl["t"], out, np.array([0.02]), nsuper_all=3)
    with pytest.raises(binding.GLError):
        ctx.lightcurve(p, wl["t"], np.empty(999), np.array([0.02]), nsuper_all=3)


def test_graph_replay_matches_eager_and_follows_in_place_updates(ctx):
    wl = inputs.mcmc_batch(n_sets=32, n_times=400, seed=21)
    p = product_params(wl)
    dp = {k: _dev(v) for k, v in p.items()}
    t, exp = _dev(wl["t"]), _dev(wl["exptime"][:32])
    outs = [torch.empty(32 * 400, dtype=torch.float64, device="cuda") for _ in range(4)]
    g0 = ctx.graph_launches()
    for o in outs[:3]:                      # first eager, then captured and replayed
        ctx.lightcurve(dp, t, o, exp, nsuper_all=15, precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    assert ctx.graph_launches() > g0
    assert torch.equal(outs[0], outs[2])
    dp["k"].mul_(1.1)                       # update a parameter in place
    ctx.lightcurve(dp, t, outs[3], exp, nsuper_all=15, precision=binding.GL_FP32C)
    ctx.graphs(False)
    eager = torch.empty_like(outs[3])
    ctx.lightcurve(dp, t, eager, exp, nsuper_all=15, precision=binding.GL_FP32C)
    ctx.graphs(True)
    torch.cuda.synchronize()
    assert not torch.equal(outs[3], outs[0])
    assert torch.equal(outs[3], eager)


def test_workload_counts(ctx):
    wl = inputs.single_transit()
    ctx.counts(True)
    _run(ctx, wl, binding.GL_FP32C)
    c = ctx.counts_read()
    ctx.counts(False)
    assert c["exposures"] == 1000
    assert c["kept"] >= c["in_window"] > 0
    assert c["items"] == 15 * c["kept"]
    assert c["full"] + c["partial"] <= c["items"]
    assert c["partial"] > 0 and c["full"] > c["partial"]


def test_autotuner_keeps_only_tolerance_passing_configurations(ctx, mcmc):
    import oracle  # noqa: F401  (reference values come from the mcmc fixture)
    wl, idx, ref = mcmc
    p = {k: _dev(v) for k, v in product_params(wl).items()}
    t, exp = _dev(wl["t"]), _dev(wl["exptime"])
    out = torch.empty(256 * len(wl["t"]), dtype=torch.float64, device="cuda")
    rep = ctx.autotune(p, t, out, exp, nsuper_all=15, precision=binding.GL_FP32C)
    assert rep["candidates"] == 16 and rep["admissible"] >= 1
    assert rep["max_abs_err"] <= 0.9e-7 and rep["threads"] in (128, 256)
    assert rep["nodes"] in (16, 20, 24, 28)
    # with the item pipeline (the default) the second axis is the quadrature kernel variant
    assert rep["quad_ctas_per_sm"] >= 4 and rep["exposure_block"] in (64, 256)
    # later calls use the chosen configuration and stay within tolerance of the oracle
    out2 = torch.empty_like(out)
    ctx.lightcurve(p, t, out2, exp, nsuper_all=15, precision=binding.GL_FP32C)
    got = out2.cpu().numpy().reshape(256, -1)
    _compare(got[idx].ravel(), ref.ravel(), binding.GL_FP32C)


def test_configure_pins_a_configuration(ctx, mcmc):
    """gl_configure sets what gl_autotune would choose; every pinned FP32C
    configuration stays within tolerance of the oracle, and bad values are refused."""
    wl, idx, ref = mcmc
    p = {k: _dev(v) for k, v in product_params(wl).items()}
    t, exp = _dev(wl["t"]), _dev(wl["exptime"])
    out = torch.empty(256 * len(wl["t"]), dtype=torch.float64, device="cuda")
    for nodes, quad, eb in ((16, 4, 256), (16, 8, 64), (28, 8, 256), (20, 4, 64)):
        ctx.configure(binding.GL_FP32C, nodes=nodes, quad_ctas=quad, exposure_block=eb)
        ctx.lightcurve(p, t, out, exp, nsuper_all=15, precision=binding.GL_FP32C)
        got = out.cpu().numpy().reshape(256, -1)
        _compare(got[idx].ravel(), ref.ravel(), binding.GL_FP32C)
    for bad in (dict(nodes=17), dict(quad_ctas=5), dict(threads=64), dict(exposure_block=128)):
        with pytest.raises(binding.GLError):
            ctx.configure(binding.GL_FP32C, **bad)
    with pytest.raises(binding.GLError):
        ctx.configure(binding.GL_FP64, nodes=16)
    ctx.configure(binding.GL_FP32C)   # back to the defaults


def test_launches_are_counted(ctx):
    n0 = ctx.launches()
    _run(ctx, inputs.single_transit(n_times=10), binding.GL_FP32C)
    assert ctx.launches() > n0
