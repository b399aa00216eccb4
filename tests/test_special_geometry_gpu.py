"""GPU: special geometries that random sampling rarely reaches, through the
geometry-level entry point gl_flux_sky.

Orientations on the axes and the diagonal (xi = 0, pi/4, pi/2; eta = 0, small,
pi/2 for a face-on circle), flattening from 0 to 0.9, and centres placed exactly on
the symmetry lines (x0 = 0, y0 = 0, x0 = y0), at the disk centre, at inner and
outer tangency of the bounding circle and with the centre on the limb.  The
FP32C path must stay within 1e-7 of the FP64 path everywhere, and the FP64 path
within 1e-10 of the oracle on a seeded subsample.  (A split of the turn built
from frame parameters once failed here: two inner maxima exactly opposite each
other, one of them at the frame's t = infinity.)
"""
import math

import numpy as np
import pytest

from paper_2410_05408_b300 import binding

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _req(k, f):
    return k / (1.0 - f) ** (1.0 / 3.0)


def _cases():
    rows = []
    for k in (0.05, 0.12, 0.2):
        for f in (0.0, 0.3, 0.6, 0.9):
            for eta in (0.0, 1e-3, 0.3, 0.5 * math.pi):
                for xi in (0.0, 0.25 * math.pi, 0.5 * math.pi):
                    req = _req(k, f)
                    line = np.linspace(-1.0 - req * 1.05, 1.0 + req * 1.05, 161)
                    pts = [(0.0, y) for y in line] + [(x, 0.0) for x in line]
                    pts += [(d / math.sqrt(2.0), d / math.sqrt(2.0)) for d in line]
                    pts += [(0.0, 0.0), (0.0, 1.0), (1.0, 0.0), (0.0, -1.0),
                            (0.0, 1.0 - req), (0.0, 1.0 + req), (1.0 - req, 0.0), (1.0 + req, 0.0),
                            (0.0, -(1.0 - req)), (-(1.0 + req), 0.0)]
                    for x, y in pts:
                        rows.append((x, y, k, f, eta, xi))
    return np.array(rows)


def _flux(ctx, rows, prec):
    n = len(rows)
    cols = [rows[:, 0], rows[:, 1], np.full(n, -1.0), rows[:, 2], rows[:, 3], rows[:, 4],
            rows[:, 5], np.full(n, 0.4), np.full(n, 0.25)]
    d = [torch.as_tensor(np.ascontiguousarray(c), device="cuda") for c in cols]
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    binding.gl_flux_sky(ctx.handle, *d, out, prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_fp32c_matches_fp64_on_special_geometries(ctx):
    rows = _cases()
    f64 = _flux(ctx, rows, binding.GL_FP64)
    f32 = _flux(ctx, rows, binding.GL_FP32C)
    err = np.abs(f32 - f64)
    worst = int(np.argmax(err))
    assert err[worst] <= 1e-7, f"max |dflux| {err[worst]:.3e} at {rows[worst]}"
    assert np.all(f32[f64 == 1.0] == 1.0)


def test_fp64_matches_oracle_on_special_geometries(ctx):
    import oracle
    rows = _cases()
    rng = np.random.default_rng(7)
    idx = rng.choice(len(rows), 1500, replace=False)
    sub = rows[idx]
    got = _flux(ctx, sub, binding.GL_FP64)
    ref = oracle.flux_sky_batch(sub[:, 0], sub[:, 1], np.full(len(sub), -1.0), sub[:, 2],
                                sub[:, 3], sub[:, 4], sub[:, 5], np.full(len(sub), 0.4),
                                np.full(len(sub), 0.25))
    err = np.abs(got - ref)
    worst = int(np.argmax(err))
    assert err[worst] <= 1e-10, f"max |dflux| {err[worst]:.3e} at {sub[worst]}"
