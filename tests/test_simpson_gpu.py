"""GPU: the paper's own scheme (Sec. 2) -- composite Simpson over the ellipse
angle with the boundary snapped onto the limb, no crossings -- against the FP64
oracle.  Its error is set by the kink where the boundary meets the limb (there
f_lin behaves like the square root of the distance along the curve), so it falls
roughly as N^-1.5: the test checks parity at a fine N, the rate of convergence,
exact flux 1 out of transit, and argument checks."""
import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def geo():
    import oracle
    g = inputs.geometry_sample(3000, seed=31)
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(g["q1"], g["q2"])])
    g["u1"], g["u2"] = u[:, 0].copy(), u[:, 1].copy()
    g["z"][:100] = 0.5   # behind the star
    ref = oracle.flux_sky_batch(g["x0"], g["y0"], g["z"], g["k"], g["f"], g["eta"], g["xi"],
                                g["u1"], g["u2"])
    return g, ref


def _out_checks(g, got, ref):
    """Exactly 1 where the planet is behind the star or beyond rho >= 1 + 2.2 k
    (2.2 k bounds R_eq for f <= 0.9); near the limb without overlap the snapped
    curve retraces a limb arc and the integrals cancel only to rounding."""
    far = (g["z"] > 0) | (np.hypot(g["x0"], g["y0"]) >= 1.0 + 2.2 * g["k"])
    assert np.all(got[far] == 1.0)
    assert np.all(np.abs(got[ref == 1.0] - 1.0) <= 1e-7)


def _run(ctx, g, n_int, prec):
    args = [torch.as_tensor(np.ascontiguousarray(g[q]), device="cuda")
            for q in ("x0", "y0", "z", "k", "f", "eta", "xi", "u1", "u2")]
    out = torch.empty(len(g["k"]), dtype=torch.float64, device="cuda")
    ctx.flux_sky_simpson(*args, out, n_int, precision=prec)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    return out.cpu().numpy()


def test_fine_simpson_matches_oracle_and_converges(ctx, geo):
    g, ref = geo
    errs = {}
    for n_int in (1024, 4096, 16384, 65536):
        got = _run(ctx, g, n_int, binding.GL_FP64)
        _out_checks(g, got, ref)
        errs[n_int] = float(np.max(np.abs(got - ref)))
    assert errs[65536] <= 2e-6, errs
    assert errs[1024] / errs[16384] >= 8.0, errs       # 16x the nodes: N^-1.5 gives 64x
    assert errs[4096] > errs[16384] > errs[65536], errs


def test_single_precision_simpson(ctx, geo):
    g, ref = geo
    got = _run(ctx, g, 4096, binding.GL_FP32C)
    _out_checks(g, got, ref)
    assert float(np.max(np.abs(got - ref))) <= 1e-4


def test_bad_interval_counts_are_rejected(ctx, geo):
    g, _ = geo
    for bad in (0, 3, 1 << 25):
        with pytest.raises(binding.GLError):
            _run(ctx, g, bad, binding.GL_FP64)
