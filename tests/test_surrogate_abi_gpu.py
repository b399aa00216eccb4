"""The surrogate's C-ABI: initialisation, training with its schedule and shuffle,
the held-out error table and the checkpoint, called through ctypes.

* A training run split into several calls, or saved after some steps and resumed
  in a fresh network from the checkpoint, ends with the parameters of one
  uninterrupted call, bit for bit (the shuffle and the learning rate of a step
  follow from the seed and the step number; the checkpoint carries the Adam
  moments and step).
* The error table equals the per-bin maximum of |network - target| computed here
  from the network's own forward pass, with +inf for empty bins.
* gl_mlp_init draws within the He bounds, reproducibly per seed.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_2410_05408_b300 import binding, surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, 7)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) * x[:, 1] + 0.3 * x[:, 2] ** 2).astype(np.float32)
    bins = rng.integers(-1, binding.SUR_BINS - 3, n).astype(np.int32)   # 3 bins left empty
    return (torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"),
            torch.tensor(bins, device="cuda"))


@pytest.fixture(scope="module")
def data():
    assert torch.cuda.is_available()
    return _data(5000, 1)


def _cfg(n, seed=5):
    return surrogate.config(n, epochs=3, batch=1024, lr=3e-3, lr_end=1e-4, seed=seed)


def test_resume_from_checkpoint_is_bit_identical(data, tmp_path):
    x, t, _ = data
    n = t.numel()
    cfg = _cfg(n)
    total = cfg.epochs * surrogate.steps_per_epoch(n, cfg)   # 3 x 5 = 15 steps
    a = binding.Mlp(0)
    a.init(7)
    la = a.train(x, t, cfg, 0, total)
    pa = a.get_params()
    # the same run in three calls
    b = binding.Mlp(0)
    b.init(7)
    for s0, s1 in ((0, 4), (4, 11), (11, total)):
        b.train(x, t, cfg, s0, s1 - s0)
    assert np.array_equal(b.get_params(), pa)
    # 7 steps, checkpoint, a fresh network resumes from it
    c = binding.Mlp(0)
    c.init(7)
    c.train(x, t, cfg, 0, 7)
    table = np.arange(binding.SUR_BINS, dtype=np.float32)
    path = str(tmp_path / "sur.ckpt")
    surrogate.save(path, c, table, cfg, 7)
    d = binding.Mlp(0)
    d.init(99)                        # different start, all overwritten by the load
    tbl, cfg2, step = surrogate.load(path, d)
    assert step == 7 and np.array_equal(tbl, table) and cfg2.as_dict() == cfg.as_dict()
    d.train(x, t, cfg2, step, total - step)
    assert np.array_equal(d.get_params(), pa)
    # a different seed shuffles differently (so the test above is not vacuous)
    e = binding.Mlp(0)
    e.init(7)
    e.train(x, t, _cfg(n, seed=6), 0, total)
    assert not np.array_equal(e.get_params(), pa)
    # and training lowers the loss on the whole set (against the initial network)
    f = binding.Mlp(0)
    f.init(7)
    assert np.isfinite(la)
    assert a.loss_grad(x, t) < 0.5 * f.loss_grad(x, t)
    for m in (a, b, c, d, e, f):
        assert m.status() == binding.GL_OK
        m.close()


def test_error_table_is_the_per_bin_maximum(data):
    x, t, bins = data
    m = binding.Mlp(0)
    m.init(3)
    m.train(x, t, _cfg(t.numel()), 0, 5)
    err = torch.empty_like(t)
    table = m.error_table(x, t, bins, err)
    y = surrogate.predict(m, x)
    torch.cuda.synchronize()
    e = (y - t).abs().cpu().numpy()
    assert np.array_equal(err.cpu().numpy(), e)
    b = bins.cpu().numpy()
    for k in range(binding.SUR_BINS):
        sel = b == k
        want = e[sel].max() if sel.any() else np.inf
        assert table[k] == want, (k, table[k], want)
    assert np.isinf(table[-3:]).all()
    m.close()


def test_init_bounds_and_reproducibility():
    m = binding.Mlp(0)
    m.init(11)
    p = m.get_params()
    m.init(11)
    assert np.array_equal(m.get_params(), p)
    m.init(12)
    assert not np.array_equal(m.get_params(), p)
    widths = (7, 256, 256, 256, 256, 1)
    o = 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        w = p[o:o + fi * fo]
        o += fi * fo
        bvec = p[o:o + fo]
        o += fo
        lim = np.sqrt(6.0 / fi)
        assert np.abs(w).max() <= lim and np.abs(bvec).max() <= 0.1
        if w.size > 1000:   # roughly uniform: mean near 0, variance near lim^2 / 3
            assert abs(w.mean()) < 0.05 * lim and abs(w.var() / (lim * lim / 3) - 1) < 0.05
    assert o == p.size
    m.close()


def test_checkpoint_errors(tmp_path):
    m = binding.Mlp(0)
    bad = tmp_path / "not_a_checkpoint"
    bad.write_bytes(b"x" * 100)
    lib = binding.load()
    assert lib.gl_surrogate_load(m.handle, os.fsencode(str(bad)), None, None, None) == binding.GL_EIO
    assert lib.gl_surrogate_load(m.handle, os.fsencode(str(tmp_path / "missing")), None, None,
                                 None) == binding.GL_EIO
    cfg = _cfg(10)
    table = np.zeros(binding.SUR_BINS, dtype=np.float32)
    assert lib.gl_surrogate_save(m.handle, os.fsencode(str(tmp_path / "no_dir" / "f")),
                                 table.ctypes.data, ctypes.byref(cfg), 0) == binding.GL_EIO
    # a step range beyond the run is refused
    x, t, _ = _data(10, 2)
    assert lib.gl_surrogate_train(m.handle, 10, x.data_ptr(), t.data_ptr(), ctypes.byref(cfg),
                                  0, 1000, None, None) == binding.GL_EINVAL
    m.close()
