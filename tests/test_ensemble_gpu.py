"""GPU: the (mu, nu) kernels of Appendix A and the device-resident stretch-move
ensemble against the oracle (oracle/munu.py and the FP64 oracle light curves):
element-wise maps and prior draws; initial log posteriors; one full sweep with
the same random numbers (same proposals, same decisions, same states); and
sampling the prior alone, whose (f, eta) must come out uniform in f and
cos-distributed in eta."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2410_05408_b300 import binding

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_munu_kernels_match_oracle(ctx):
    from oracle import munu as M
    rng = np.random.default_rng(1)
    f, eta = rng.uniform(0.01, 0.99, 4096), rng.uniform(0.01, 1.55, 4096)
    u, w = rng.uniform(0.001, 0.999, 4096), rng.uniform(0.001, 0.999, 4096)
    out = [torch.empty(4096, dtype=torch.float64, device="cuda") for _ in range(6)]
    binding.gl_munu(ctx.handle, "to_munu", _dev(f), _dev(eta), out[0], out[1])
    binding.gl_munu(ctx.handle, "to_feta", out[0], out[1], out[2], out[3])
    binding.gl_munu(ctx.handle, "prior", _dev(u), _dev(w), out[4], out[5])
    got = [o.cpu().numpy() for o in out]
    np.testing.assert_allclose(got[0], M.mu_of(f, eta), atol=1e-13)
    np.testing.assert_allclose(got[1], M.nu_of(f, eta), atol=1e-12)
    np.testing.assert_allclose(got[2], f, atol=1e-12)
    np.testing.assert_allclose(got[3], eta, atol=1e-7)
    mu, nu = M.prior_draw(u, w)
    np.testing.assert_allclose(got[4], mu, atol=1e-12)
    np.testing.assert_allclose(got[5], nu, atol=1e-12)


# The fit: a C0-like single transit, 200 exposures over +-10 h, x 3.
TRUTH = np.array([0.0, 542.0, 230.0, 0.2, 0.066, 0.0, 0.5, 0.785, 0.42, 0.31])
LO = np.array([-0.1, 541.0, 150.0, 0.0, 0.03, -1.0, 0.0, 0.0, 0.0, 0.0])
HI = np.array([0.1, 543.0, 300.0, 0.9, 0.12, 1.0, 1.0, math.pi, 1.0, 1.0])
EXPTIME, NSUPER = 0.02, 3


def _oracle_lnpost(X, t, data, sigma):
    import oracle
    from oracle import munu as M
    X = np.atleast_2d(X)
    out = np.full(len(X), -np.inf)
    for i, x in enumerate(X):
        t0, P, a, b, k, mu, nu, xi, q1, q2 = x
        inside = (np.all(x >= LO) and np.all(x <= HI) and -1 < mu <= 1 and 0 <= nu < 1
                  and 0 <= q1 <= 1 and 0 <= q2 <= 1 and P > 0 and a > 1 and k > 0
                  and 0 <= b < a)
        if not inside:
            continue
        f, eta = M.f_eta_of(mu, nu)
        u1, u2 = oracle.q_to_u(q1, q2)
        p = dict(t0=[t0], period=[P], a_rs=[a], b=[b], ecc=[0.0], omega=[0.5 * math.pi],
                 k=[k], f=[f], eta=[eta], xi=[xi], u1=[u1], u2=[u2])
        flux = oracle.lightcurve(p, t, EXPTIME, NSUPER)[0]
        out[i] = math.log(M.p_munu(mu, nu)) - 0.5 * np.sum(((flux - data) / sigma) ** 2)
    return out


@pytest.fixture(scope="module")
def fit():
    import oracle
    from oracle import munu as M
    t = np.linspace(-10.0 / 24.0, 10.0 / 24.0, 200)
    t0, P, a, b, k, mu, nu, xi, q1, q2 = TRUTH
    f, eta = M.f_eta_of(mu, nu)
    u1, u2 = oracle.q_to_u(q1, q2)
    p = dict(t0=[t0], period=[P], a_rs=[a], b=[b], ecc=[0.0], omega=[0.5 * math.pi], k=[k],
             f=[f], eta=[eta], xi=[xi], u1=[u1], u2=[u2])
    rng = np.random.default_rng(2)
    sigma = np.full(t.size, 1e-4)
    data = oracle.lightcurve(p, t, EXPTIME, NSUPER)[0] + rng.normal(0, 1e-4, t.size)
    walkers = TRUTH + rng.normal(0, 1, (16, 10)) * np.array(
        [1e-3, 1e-3, 0.5, 0.01, 5e-4, 0.05, 0.05, 0.05, 0.02, 0.02])
    walkers[3, 1] = 600.0   # one walker outside the prior box
    return t, data, sigma, walkers


def test_init_and_one_sweep_match_the_oracle(ctx, fit):
    from oracle import munu as M
    t, data, sigma, walkers = fit
    dw = _dev(walkers)
    ens = binding.Ensemble(ctx, dw, _dev(LO), _dev(HI), _dev(t), _dev(data), _dev(sigma),
                           EXPTIME, NSUPER, precision=binding.GL_FP64)
    ens.init()
    torch.cuda.synchronize()
    lp0 = ens.logpost.cpu().numpy()
    ref0 = _oracle_lnpost(walkers, t, data, sigma)
    assert np.isneginf(lp0[3]) and np.isneginf(ref0[3])
    fin = np.isfinite(ref0)
    np.testing.assert_allclose(lp0[fin], ref0[fin], rtol=0, atol=1e-6)

    rng = np.random.default_rng(3)
    rnd = rng.uniform(0.0, 1.0, 3 * 16)
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    ens.sweep(_dev(rnd), acc)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    W, LP = walkers.copy(), lp0.copy()
    n_acc = 0
    for h in (0, 1):
        r = rnd[h * 24:(h + 1) * 24]
        act, oth = np.arange(h, 16, 2), np.arange(1 - h, 16, 2)
        W, LP, ok, _ = M.stretch_half(W, LP, act, oth, r[:8], r[8:16], r[16:24],
                                      lambda y: _oracle_lnpost(y, t, data, sigma))
        n_acc += int(ok.sum())
    np.testing.assert_allclose(dw.cpu().numpy(), W, rtol=1e-13, atol=1e-15)
    got_lp = ens.logpost.cpu().numpy()
    fin = np.isfinite(LP)
    np.testing.assert_array_equal(np.isfinite(got_lp), fin)
    np.testing.assert_allclose(got_lp[fin], LP[fin], rtol=0, atol=1e-6)
    assert int(acc.item()) == n_acc


def test_prior_only_sampling_gives_the_target_prior(ctx, fit):
    """With data carrying no information (sigma 1e6) the ensemble samples the
    prior: (f, eta) from the final (mu, nu) of 2048 walkers after 300 sweeps,
    starting from prior draws of every coordinate."""
    from oracle import munu as M
    t, data, _, _ = fit
    n = 2048
    rng = np.random.default_rng(4)
    u, w = rng.uniform(size=n), rng.uniform(size=n)
    mu, nu = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(
        n, dtype=torch.float64, device="cuda")
    binding.gl_munu(ctx.handle, "prior", _dev(u), _dev(w), mu, nu)
    # a full-rank ensemble (the stretch move's z^(D-1) assumes walkers spanning all
    # D dimensions): every coordinate drawn from its prior
    X = rng.uniform(LO, HI, (n, 10))
    X[:, 5], X[:, 6] = mu.cpu().numpy(), nu.cpu().numpy()
    dw = _dev(X)
    ens = binding.Ensemble(ctx, dw, _dev(LO), _dev(HI), _dev(t), _dev(data),
                           _dev(np.full(t.size, 1e6)), EXPTIME, NSUPER,
                           precision=binding.GL_FP32C)
    ens.init()
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    for _ in range(300):
        ens.sweep(torch.rand(3 * n, dtype=torch.float64, device="cuda", generator=gen), acc)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    frac = int(acc.item()) / (300 * n)
    assert 0.1 < frac < 0.95
    final = dw.cpu().numpy()
    f, eta = M.f_eta_of(final[:, 5], final[:, 6])
    assert stats.kstest(f, "uniform").pvalue > 1e-4
    assert stats.kstest(eta, lambda x: np.sin(np.clip(x, 0, math.pi / 2))).pvalue > 1e-4
