"""GPU: general triaxial ellipsoid (Sec. 2: semi-axes a, b, c along x', y', z'
and all three rotation angles), passed as the optional g and zeta of the
parameter sets, against the FP64 oracle's triaxial light curves; g = 0 must
reproduce the oblate call bit for bit (zeta has no effect there); invalid g
gives NaN and the invalid-set status."""
import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

from _common import PARAM_NAMES, nsuper_array, oracle_params, product_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {binding.GL_FP64: 1e-10, binding.GL_FP32C: 1e-7}


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.array(a, copy=True)).to(device="cuda", dtype=dtype).contiguous()


def _run(ctx, wl, prec, extra=None):
    p = product_params(wl)
    for key in ("g", "zeta"):
        if key in wl["params"]:
            p[key] = np.asarray(wl["params"][key], dtype=np.float64)
    if extra is not None:
        p.update(extra)
    n_sets = len(p["t0"])
    dp = {k: _dev(v) for k, v in p.items()}
    exptime = np.broadcast_to(wl["exptime"], (n_sets,))
    out = torch.empty(n_sets * len(wl["t"]), dtype=torch.float64, device="cuda")
    ctx.lightcurve(dp, _dev(wl["t"]), out, _dev(exptime),
                   nsuper=_dev(nsuper_array(wl, n_sets), torch.int32), precision=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def tri():
    import oracle
    wl = inputs.triaxial_batch()
    op = oracle_params(wl)
    op["g"], op["zeta"] = wl["params"]["g"], wl["params"]["zeta"]
    assert set(PARAM_NAMES) <= set(op)
    ref = oracle.lightcurve(op, wl["t"], wl["exptime"], wl["nsuper"]).reshape(-1)
    return wl, ref


@pytest.mark.parametrize("prec", [binding.GL_FP64, binding.GL_FP32C])
def test_triaxial_light_curves_match_oracle(ctx, tri, prec):
    wl, ref = tri
    got = _run(ctx, wl, prec)
    assert ctx.sync() == binding.GL_OK
    assert np.mean(ref < 1.0) > 0.3
    err = float(np.max(np.abs(got - ref)))
    assert err <= TOL[prec], f"max |dflux| {err:.3e}"
    assert np.all(got[ref == 1.0] == 1.0)


def test_zero_g_is_the_oblate_call(ctx, tri):
    wl, _ = tri
    n = len(wl["params"]["t0"])
    base = {k: v for k, v in wl["params"].items() if k not in ("g", "zeta")}
    wl0 = dict(wl, params=base)
    plain = _run(ctx, wl0, binding.GL_FP64)
    zero = _run(ctx, wl0, binding.GL_FP64,
                extra={"g": np.zeros(n), "zeta": np.linspace(0.1, 3.0, n)})
    assert ctx.sync() == binding.GL_OK
    assert np.array_equal(plain, zero)


def test_invalid_g_gives_nan_and_status(ctx, tri):
    wl, _ = tri
    n = len(wl["params"]["t0"])
    g = np.array(wl["params"]["g"], copy=True)
    g[0] = 1.0
    got = _run(ctx, wl, binding.GL_FP64, extra={"g": g})
    per = len(wl["t"])
    assert np.all(np.isnan(got[:per]))
    assert np.all(np.isfinite(got[per:]))
    assert ctx.sync() == binding.GL_ENUMERIC
