"""GPU: tidally locked bodies (Appendix B) -- the projection recomputed for every
sub-exposure from the orbital angle -- against the FP64 oracle's locked light
curves (printed Eqs. dx-locked, dy1-locked, dy2-locked), and a sphere, whose
projection cannot depend on the orbital angle, against the unlocked path."""
import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

from _common import nsuper_array, oracle_params, product_params

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


def _run(ctx, wl, prec, locked, params=None):
    p = params if params is not None else product_params(wl)
    if params is None:
        for key in ("g", "zeta"):
            if key in wl["params"]:
                p[key] = np.asarray(wl["params"][key], dtype=np.float64)
    n_sets = len(p["t0"])
    dp = {k: _dev(v) for k, v in p.items()}
    out = torch.empty(n_sets * len(wl["t"]), dtype=torch.float64, device="cuda")
    ctx.lightcurve(dp, _dev(wl["t"]), out, _dev(np.broadcast_to(wl["exptime"], (n_sets,))),
                   nsuper=_dev(nsuper_array(wl, n_sets), torch.int32), precision=prec,
                   locked=locked)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def locked():
    import oracle
    wl = inputs.locked_batch()
    op = oracle_params(wl)
    op["g"], op["zeta"] = wl["params"]["g"], wl["params"]["zeta"]
    ref = oracle.lightcurve(op, wl["t"], wl["exptime"], wl["nsuper"], locked=True).reshape(-1)
    unlocked = oracle.lightcurve(op, wl["t"], wl["exptime"], wl["nsuper"]).reshape(-1)
    return wl, ref, unlocked


@pytest.mark.parametrize("prec", [binding.GL_FP64, binding.GL_FP32C])
def test_locked_light_curves_match_oracle(ctx, locked, prec):
    wl, ref, unlocked = locked
    got = _run(ctx, wl, prec, locked=True)
    assert np.mean(ref < 1.0) > 0.3
    assert np.max(np.abs(ref - unlocked)) > 1e-4   # locking changes these curves
    err = float(np.max(np.abs(got - ref)))
    assert err <= TOL[prec], f"max |dflux| {err:.3e}"
    assert np.all(got[ref == 1.0] == 1.0)


def test_sphere_is_the_same_locked_or_not(ctx, locked):
    wl, _, _ = locked
    p = product_params(wl)
    p["f"] = np.zeros_like(p["f"])
    a = _run(ctx, wl, binding.GL_FP64, locked=True, params=dict(p))
    b = _run(ctx, wl, binding.GL_FP64, locked=False, params=dict(p))
    assert float(np.max(np.abs(a - b))) <= 1e-13
