"""The surrogate path: training data against the oracle, a trained network's
light curves against the oracle (with the exact fallback on), and what the
network gains over the exact path on the surrogate-in-the-loop workload."""
import time

import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs, surrogate

from _common import PARAM_NAMES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = binding.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def trained(ctx):
    m = binding.Mlp(0)
    rng = np.random.default_rng(0)
    from oracle import mlp as omlp          # initial weights only
    p0 = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in omlp.init_params(rng)])
    m.set_params(p0.astype(np.float32))
    train = surrogate.make_dataset(ctx, 300_000, seed=31)
    held = surrogate.make_dataset(ctx, 100_000, seed=32)
    hist = surrogate.train(m, train, epochs=4, batch=8192)
    table = surrogate.error_table(m, held)
    yield m, table, hist, held
    m.close()


def test_targets_match_oracle(ctx):
    import oracle
    d = surrogate.make_dataset(ctx, 3000, seed=33)
    s = inputs.surrogate_samples(3000, 33)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(s["q1"], s["q2"])])
    eta = np.arccos(s["cos_tilt"])
    zeros = np.zeros(3000)
    f_obl = oracle.flux_sky_batch(s["x"], s["y"], -np.ones(3000), s["k"], s["f"], eta, s["psi"],
                                  u[:, 0], u[:, 1])
    r_area = np.array([np.sqrt(a * c) for a, _, c in
                       (oracle.oblate_ellipse(k, f, e, x) for k, f, e, x in
                        zip(s["k"], s["f"], eta, s["psi"]))])
    f_sph = oracle.flux_sky_batch(s["x"], s["y"], -np.ones(3000), r_area, zeros, zeros, zeros,
                                  u[:, 0], u[:, 1])
    scale = d["scale"].cpu().numpy().astype(np.float64)
    got = d["t"].cpu().numpy().astype(np.float64) * scale
    assert np.max(np.abs(got - (f_obl - f_sph))) < 1e-9
    assert np.mean(np.abs(f_obl - f_sph) > 1e-6) > 0.1


def test_training_converges_and_table_is_finite(trained):
    m, table, hist, _ = trained
    assert hist[-1] < 0.5 * hist[0]
    assert np.all(table[np.isfinite(table)] >= 0)
    assert np.isfinite(table).sum() >= 8


def _walkers(n):
    wl = inputs.injected_curve(n_walkers=n)
    p = {k: torch.tensor(np.ascontiguousarray(wl["walkers"][k]), dtype=torch.float64,
                         device="cuda") for k in PARAM_NAMES}
    return wl, p


def test_surrogate_lightcurves_within_1ppm_of_oracle(ctx, trained):
    import oracle
    m, table, _, _ = trained
    wl, p = _walkers(6)
    t = torch.tensor(wl["t"], device="cuda")
    exp = torch.full((6,), wl["exptime"], dtype=torch.float64, device="cuda")
    out = torch.empty(6 * len(wl["t"]), dtype=torch.float64, device="cuda")
    stats = binding.gl_lightcurve_surrogate(ctx.handle, m, p, t, out, table, 1e-6, exptime=exp,
                                            nsuper_all=15)
    ref = oracle.lightcurve({k: wl["walkers"][k] for k in PARAM_NAMES}, wl["t"], wl["exptime"], 15)
    err = np.max(np.abs(out.cpu().numpy() - ref.ravel()))
    assert err <= 1e-6, err
    assert stats["items"] > 0


def test_all_fallback_equals_exact_fp32c(ctx, trained):
    m, table, _, _ = trained
    wl, p = _walkers(8)
    t = torch.tensor(wl["t"], device="cuda")
    exp = torch.full((8,), wl["exptime"], dtype=torch.float64, device="cuda")
    out = torch.empty(8 * len(wl["t"]), dtype=torch.float64, device="cuda")
    stats = binding.gl_lightcurve_surrogate(ctx.handle, m, p, t, out, table, 0.0, exptime=exp,
                                            nsuper_all=15)
    exact = torch.empty_like(out)
    ctx.lightcurve(p, t, exact, exp, nsuper_all=15, precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    assert stats["fallback"] > 0
    assert float((out - exact).abs().max()) <= 1e-7


def test_gain_of_the_network_over_the_exact_path(ctx, trained):
    """Times the surrogate path and the exact FP32C path on the injected-transit
    workload (1024 walkers x 3000 exposures x 15) and reports the ratio and the
    fallback fraction; the gain itself is measured, not asserted."""
    m, table, _, _ = trained
    wl, p = _walkers(1024)
    t = torch.tensor(wl["t"], device="cuda")
    exp = torch.full((1024,), wl["exptime"], dtype=torch.float64, device="cuda")
    out_s = torch.empty(1024 * len(wl["t"]), dtype=torch.float64, device="cuda")
    out_e = torch.empty_like(out_s)
    for _ in range(2):
        stats = binding.gl_lightcurve_surrogate(ctx.handle, m, p, t, out_s, table, 1e-6,
                                                exptime=exp, nsuper_all=15)
        ctx.lightcurve(p, t, out_e, exp, nsuper_all=15, precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        binding.gl_lightcurve_surrogate(ctx.handle, m, p, t, out_s, table, 1e-6, exptime=exp,
                                        nsuper_all=15)
    torch.cuda.synchronize()
    ts = (time.perf_counter() - t0) / 3
    t0 = time.perf_counter()
    for _ in range(3):
        ctx.lightcurve(p, t, out_e, exp, nsuper_all=15, precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / 3
    diff = float((out_s - out_e).abs().max())
    print(f"surrogate {ts * 1e3:.3f} ms, exact FP32C {te * 1e3:.3f} ms, gain {te / ts:.3f}x, "
          f"fallback {stats['fallback']}/{stats['items']}, max|diff| {diff:.2e}")
    assert diff <= 2e-6
