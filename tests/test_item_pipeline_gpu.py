"""GPU: the item pipeline of the light-curve kernel gives bit-identical output.

With the pipeline on, tiles of exposures hand their in-window sub-exposures to a
global queue that a second kernel integrates and a third sums per exposure; with
it off each tile integrates its own; with a small workspace some tiles do one and
some the other.  Every item is evaluated with the same arithmetic and every
exposure is summed in sub-exposure order, so all three must agree bit for bit, on
both precisions, for a shared time grid, a ragged CSR batch and eccentric orbits.
"""
import numpy as np
import pytest

from paper_2410_05408_b300 import binding, inputs

from _common import nsuper_array, product_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [binding.GL_FP64, binding.GL_FP32C]


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.array(a, copy=True)).to(device="cuda", dtype=dtype).contiguous()


def _prepare(wl):
    p = product_params(wl)
    n_sets = len(p["t0"])
    exptime = np.ascontiguousarray(np.broadcast_to(wl["exptime"], (n_sets,)), dtype=np.float64)
    offsets = wl.get("offsets")
    n_total = n_sets * len(wl["t"]) if offsets is None else int(offsets[-1])
    return dict(p={k: _dev(v) for k, v in p.items()}, t=_dev(wl["t"]), exptime=_dev(exptime),
                ns=_dev(nsuper_array(wl, n_sets), torch.int32),
                offsets=None if offsets is None else _dev(offsets, torch.int64), n_total=n_total)


def _run(ctx, d, prec):
    out = torch.empty(d["n_total"], dtype=torch.float64, device="cuda")
    for _ in range(2):   # eager first call, then the captured graph
        ctx.lightcurve(d["p"], d["t"], out, d["exptime"], nsuper=d["ns"], offsets=d["offsets"],
                       precision=prec)
    torch.cuda.synchronize()
    assert ctx.sync() == binding.GL_OK
    return out.cpu().numpy()


def _items(ctx, d, prec):
    ctx.counts(True)
    _run(ctx, d, prec)
    n = ctx.counts_read()["items"]
    ctx.counts(False)
    return n


WORKLOADS = {
    "mcmc_batch": lambda: inputs.mcmc_batch(seed=11),
    "uneven_batch": lambda: inputs.uneven_batch(seed=12),
    "extreme_orbits": lambda: inputs.extreme_orbits(seed=13),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
@pytest.mark.parametrize("prec", PRECS)
def test_pipeline_local_and_mixed_are_bit_identical(ctx, name, prec):
    d = _prepare(WORKLOADS[name]())
    try:
        ctx.item_pipeline(True)
        on = _run(ctx, d, prec)
        items = _items(ctx, d, prec)
        ctx.item_pipeline(False)
        off = _run(ctx, d, prec)
        # a workspace smaller than the batch's items but larger than one tile's
        # (256 exposures x 15): the first tiles queue, later ones integrate locally
        cap = max(4000, items // 3)
        ctx.item_pipeline(True, cap)
        mixed = _run(ctx, d, prec)
    finally:
        ctx.item_pipeline(True)
    assert items > 0
    for other in (off, mixed):
        same = (on == other) | (np.isnan(on) & np.isnan(other))
        assert same.all(), (int((~same).sum()), float(np.nanmax(np.abs(on - other))))
    assert (on < 1.0).sum() > 0


def test_pipeline_setting_is_validated(ctx):
    with pytest.raises(binding.GLError):
        ctx.item_pipeline(True, -1)
    with pytest.raises(binding.GLError):
        ctx.item_pipeline(True, 1 << 31)
    ctx.item_pipeline(True)


def test_pipeline_kernels_are_profiled(ctx):
    d = _prepare(inputs.mcmc_batch(seed=14))
    ctx.profile(True)
    _run(ctx, d, binding.GL_FP32C)
    got = {k: ctx.profile_read(k)[1] for k in (binding.GL_KERNEL_SETUP, binding.GL_KERNEL_WINDOW,
                                                binding.GL_KERNEL_CURVE, binding.GL_KERNEL_QUAD)}
    ctx.profile(False)
    assert all(n == 2 for n in got.values()), got


def _boundary_batch(csr):
    """Curve lengths around the window kernel's pass and warp widths (0, 1, 31-33,
    255-257, 511-513, 1023-1025 exposures) or a shared grid of 777 times; three
    invalid sets (unbound orbits) and three whole-orbit sets (a/R* = 1.05) mixed in."""
    wl = inputs.uneven_batch(n_curves=240, seed=21, min_len=100, max_len=2000)
    p = {k: np.array(v, copy=True) for k, v in wl["params"].items()}
    n = len(p["t0"])
    for s in (5, 77, 200):
        p["ecc"][s] = 1.5
    for s in (9, 110, 233):   # an orbit inside 1 + R_eq: no window, every time kept
        p["a_rs"][s], p["b"][s], p["ecc"][s] = 1.05, 0.1, 0.0
    if csr:
        pattern = [0, 1, 2, 31, 32, 33, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 0, 3]
        lengths = np.array([pattern[s % len(pattern)] for s in range(n)], dtype=np.int64)
        off = np.zeros(n + 1, dtype=np.int64)
        off[1:] = np.cumsum(lengths)
        t = np.concatenate([(np.arange(m) - 0.5 * (m - 1)) * wl["exptime"][s]
                            for s, m in enumerate(lengths)])
        return dict(wl, params=p, t=t, offsets=off), lengths
    t = (np.arange(777) - 388.0) * 900.0 / 86400.0
    out = dict(wl, params=p, t=t, exptime=np.full(n, 900.0 / 86400.0), nsuper=15)
    out.pop("offsets")
    return out, np.full(n, 777, dtype=np.int64)


@pytest.mark.parametrize("csr", [True, False])
@pytest.mark.parametrize("prec", PRECS)
def test_window_kernel_set_boundaries(ctx, csr, prec):
    """The window kernel's per-thread set cursor and its fast and general passes,
    on ranges that start and end at every offset within a pass: the pipeline must
    equal the tile path bit for bit, invalid sets must be NaN throughout and the
    others finite."""
    wl, lengths = _boundary_batch(csr)
    d = _prepare(wl)

    def run():
        out = torch.empty(d["n_total"], dtype=torch.float64, device="cuda")
        for _ in range(2):   # eager first call, then the captured graph
            ctx.lightcurve(d["p"], d["t"], out, d["exptime"], nsuper=d["ns"],
                           offsets=d["offsets"], precision=prec)
        torch.cuda.synchronize()
        assert ctx.sync() == binding.GL_ENUMERIC   # the invalid sets are reported
        return out.cpu().numpy()

    try:
        ctx.item_pipeline(True)
        on = run()
        ctx.item_pipeline(False)
        off = run()
    finally:
        ctx.item_pipeline(True)
    same = (on == off) | (np.isnan(on) & np.isnan(off))
    assert same.all(), (int((~same).sum()), float(np.nanmax(np.abs(on - off))))
    starts = np.concatenate([[0], np.cumsum(lengths)])
    bad = np.zeros(len(on), dtype=bool)
    for s in (5, 77, 200):
        bad[starts[s]:starts[s + 1]] = True
    assert np.isnan(on[bad]).all()
    assert np.isfinite(on[~bad]).all()
    assert (on[~bad] < 1.0).sum() > 0


@pytest.mark.parametrize("prec", PRECS)
def test_non_finite_times_give_flux_one(ctx, prec):
    """A time that is NaN (either sign bit) or infinite lies outside every transit
    window (documented in the header): flux exactly 1, on the pipeline, on the
    tile path and with the graph replay, while the finite times around it keep
    their values."""
    wl = inputs.single_transit(n_times=200)
    t = np.array(wl["t"], copy=True)
    nan_neg = np.frombuffer(np.uint64(0xFFF8000000000000).tobytes(), dtype=np.float64)[0]
    bad = [7, 100, 101, 150]
    t[bad] = [np.nan, nan_neg, np.inf, -np.inf]
    wl_bad = dict(wl, t=t)
    ref = _run(ctx, _prepare(wl), prec)
    assert np.any(ref[0, bad] < 1.0) if ref.ndim == 2 else np.any(ref[bad] < 1.0)
    for on in (True, False):
        ctx.item_pipeline(on)
        got = _run(ctx, _prepare(wl_bad), prec).reshape(-1)
        assert np.all(got[bad] == 1.0)
        keep = np.setdiff1d(np.arange(got.size), bad)
        assert np.array_equal(got[keep], ref.reshape(-1)[keep])
    ctx.item_pipeline(True)


@pytest.mark.parametrize("prec", PRECS)
def test_graph_profiling_times_kernels_inside_the_replay(ctx, prec):
    """Profiling mode 2 keeps the graph replay and times every kernel of the step
    with event-record nodes inside the graph: each profiled replay yields one span
    per kernel, the spans add up to the step's span, and the light curve is bit
    for bit the unprofiled one."""
    d = _prepare(inputs.mcmc_batch(n_sets=32, n_times=600, seed=3))
    ref = _run(ctx, d, prec)
    out = torch.empty(d["n_total"], dtype=torch.float64, device="cuda")
    call = lambda: ctx.lightcurve(d["p"], d["t"], out, d["exptime"], nsuper=d["ns"],  # noqa: E731
                                  offsets=d["offsets"], precision=prec)
    ctx.profile(binding.PROFILE_GRAPH)
    call()                               # capture of the profiled graph
    torch.cuda.synchronize()
    ctx.profile(binding.PROFILE_GRAPH)   # reset
    g0 = ctx.graph_launches()
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    assert ctx.graph_launches() - g0 == 5
    kinds = {"setup": binding.GL_KERNEL_SETUP, "window": binding.GL_KERNEL_WINDOW,
             "exposures": binding.GL_KERNEL_CURVE, "quad_sum": binding.GL_KERNEL_QUAD,
             "quad": binding.GL_KERNEL_ITEMS, "step": binding.GL_KERNEL_STEP}
    got = {k: ctx.profile_read(v) for k, v in kinds.items()}
    ctx.profile(False)
    assert all(n == 5 for _, n in got.values()), got
    assert all(ms > 0.0 for ms, _ in got.values()), got
    parts = sum(got[k][0] for k in ("setup", "window", "exposures", "quad_sum"))
    assert abs(parts - got["step"][0]) <= 1e-3 * 5 + 1e-3 * got["step"][0], got
    assert got["quad"][0] <= got["quad_sum"][0] + 1e-3
    assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref)
    assert ctx.sync() == binding.GL_OK
