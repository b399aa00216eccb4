"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the tensor-core kernels' mbarrier wait is
  made to poll a phase that nothing completes (gl_mlp_wait_probe), before any
  MMA is issued.  The kernels give up, free their tensor memory and return;
  gl_mlp_status reports GL_ETIMEOUT once; with the probe off the same network
  gives the same outputs as before, bit for bit (the context stayed usable).
* An allocation that fails: the context refuses to grow its workspace
  (gl_debug_alloc_limit), gl_lightcurve_batch returns GL_ENOMEM with a message,
  and once the limit is lifted the same call succeeds with the same light curve.
"""
import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

from _common import product_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_network_recovers():
    assert torch.cuda.is_available()
    m = binding.Mlp(0)
    m.init(5)
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.uniform(-1, 1, (700, 7)).astype(np.float32), device="cuda")
    y0 = torch.empty(700, dtype=torch.float32, device="cuda")
    m.forward(x, y0)
    torch.cuda.synchronize()
    assert m.status() == binding.GL_OK
    m.wait_probe(64)
    y1 = torch.empty_like(y0)
    m.forward(x, y1)
    torch.cuda.synchronize()
    assert m.status() == binding.GL_ETIMEOUT
    assert m.status() == binding.GL_OK          # read once, then cleared
    m.wait_probe(0)
    y2 = torch.empty_like(y0)
    m.forward(x, y2)
    torch.cuda.synchronize()
    assert m.status() == binding.GL_OK
    assert torch.equal(y0, y2)
    with pytest.raises(binding.GLError):
        m.wait_probe(-1)
    m.close()


def test_allocation_failure_is_reported_and_recovered():
    wl = inputs.mcmc_batch(n_sets=16, n_times=400, seed=9)
    p = {k: torch.tensor(v, dtype=torch.float64, device="cuda")
         for k, v in product_params(wl).items()}
    t = torch.tensor(wl["t"], dtype=torch.float64, device="cuda")
    ex = torch.tensor(np.broadcast_to(wl["exptime"], (16,)).copy(), dtype=torch.float64,
                      device="cuda")
    ref = torch.empty(16 * 400, dtype=torch.float64, device="cuda")
    c = binding.Context(0)
    c.lightcurve(p, t, ref, ex, nsuper_all=wl["nsuper"], precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    c.close()
    ctx = binding.Context(0)          # fresh: no workspace yet
    ctx.alloc_limit(1024)
    out = torch.full_like(ref, -1.0)
    with pytest.raises(binding.GLError) as err:
        ctx.lightcurve(p, t, out, ex, nsuper_all=wl["nsuper"], precision=binding.GL_FP32C)
    assert err.value.code == binding.GL_ENOMEM
    assert "refused" in ctx.last_error()
    ctx.alloc_limit(0)
    ctx.lightcurve(p, t, out, ex, nsuper_all=wl["nsuper"], precision=binding.GL_FP32C)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    assert torch.equal(out, ref)
    ctx.close()
