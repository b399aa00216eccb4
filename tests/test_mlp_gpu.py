"""Surrogate network kernels (tcgen05) against the FP64 MLP oracle.

The GPU network keeps BF16 copies of the three hidden weight matrices, BF16
hidden activations and BF16 gradients at the hidden pre-activations; the oracle
gets the same BF16-rounded hidden weights and rounds the same quantities to BF16
(its ``round_act`` hook), in FP64 otherwise.  What remains between the two is the
FP32 accumulation and the rare BF16 rounding that lands on the other side of a
tie point, so every output and every gradient element is held to
4 x 2^-8 x sum |a_i b_i| of its own dot product (the BF16 half-ulp scale of each
term; a single flipped rounding moves one term by at most 2^-7 of itself).  A
wrong row, column or tile would miss this by orders of magnitude.  The former
norm-wise checks (1.5e-2 on outputs and loss against the unrounded FP64
network, 5e-2 per layer's gradient) are kept beside them."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2410_05408_b300 import binding

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def flatten(params):
    parts = []
    for W, b in params:
        parts += [W.reshape(-1), b.reshape(-1)]
    return np.concatenate(parts).astype(np.float32)


def unflatten(v):
    out, o = [], 0
    for fi, fo in zip(omlp.WIDTHS[:-1], omlp.WIDTHS[1:]):
        W = v[o:o + fi * fo].reshape(fi, fo).astype(np.float64)
        o += fi * fo
        b = v[o:o + fo].astype(np.float64)
        o += fo
        out.append((W, b))
    return out


def bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def as_gpu_sees(params):
    """The hidden layers' weights as the tensor cores see them (BF16)."""
    return [(bf16(W) if 0 < li < 4 else W, b) for li, (W, b) in enumerate(params)]


ELEM = 4.0 * 2.0 ** -8


def _out_scale(params, x):
    """sum_k |h4_k w5_k| + |b5| per sample, on the BF16-aware oracle."""
    _, (acts, _) = omlp.forward(params, x, round_act=bf16)
    return np.abs(acts[4]) @ np.abs(params[4][0][:, 0]) + abs(params[4][1][0])


def _grad_scales(params, x, t):
    """Per gradient element, the sum over samples of |input activation x dz| (and
    of |dz| for the biases), on the BF16-aware oracle."""
    y, (acts, pres) = omlp.forward(params, x, round_act=bf16)
    n = y.shape[0]
    dz = (2.0 / n) * (y - t)[:, None]
    out = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        out[li] = (np.abs(acts[li]).T @ np.abs(dz), np.abs(dz).sum(axis=0))
        if li > 0:
            dz = bf16((dz @ W.T) * omlp.silu_grad(pres[li - 1]))
    return out


def _elementwise(got, ref, scale, what):
    bad = np.abs(got - ref) > ELEM * scale + 1e-30
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - ref) / (scale + 1e-300))))


@pytest.fixture(scope="module")
def net():
    assert torch.cuda.is_available()
    m = binding.Mlp(0)
    yield m
    m.close()


def _setup(net, seed, n):
    rng = np.random.default_rng(seed)
    params = omlp.init_params(rng)
    flat = flatten(params)
    net.set_params(flat)
    params = unflatten(flat)           # float32-rounded master values
    x = rng.uniform(-1, 1, (n, 7)).astype(np.float32)
    t = (np.sin(x[:, 0] * 2) * x[:, 1] + 0.3 * x[:, 2] ** 2).astype(np.float32)
    return params, x, t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n", [1, 200, 1000])
def test_forward_matches_oracle(net, n):
    params, x, _ = _setup(net, 1, n)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(x, device="cuda"), y)
    torch.cuda.synchronize()
    gp = as_gpu_sees(params)
    ref, _ = omlp.forward(gp, x.astype(np.float64))
    assert _rel(y.cpu().numpy(), ref) < 1.5e-2
    ref_b, _ = omlp.forward(gp, x.astype(np.float64), round_act=bf16)
    _elementwise(y.cpu().numpy(), ref_b, _out_scale(gp, x.astype(np.float64)), "y")
    assert net.status() == binding.GL_OK


def _grads_match_oracle(net, seed, n):
    params, x, t = _setup(net, seed, n)
    loss = net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = unflatten(net.get_grads())
    gp = as_gpu_sees(params)
    xd, td = x.astype(np.float64), t.astype(np.float64)
    ref_loss, ref_g = omlp.loss_and_grads(gp, xd, td)
    assert abs(loss - ref_loss) / ref_loss < 1.5e-2
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(g, ref_g)):
        assert _rel(gW, rW) < 5e-2, (li, _rel(gW, rW))
        assert _rel(gb, rb) < 5e-2, (li, _rel(gb, rb))
    # element by element against the BF16-aware oracle
    lb, gb_ref = omlp.loss_and_grads(gp, xd, td, round_act=bf16)
    yb, _ = omlp.forward(gp, xd, round_act=bf16)
    ls = np.mean(2.0 * np.abs(yb - td) * _out_scale(gp, xd))   # d loss = mean 2 r dy
    assert abs(loss - lb) <= ELEM * ls, (loss, lb, ls)
    scales = _grad_scales(gp, xd, td)
    for li, ((gW, gbias), (rW, rb), (sW, sb)) in enumerate(zip(g, gb_ref, scales)):
        _elementwise(gW, rW, sW, f"dW{li + 1}")
        _elementwise(gbias, rb, sb, f"db{li + 1}")
    assert net.status() == binding.GL_OK


def test_gradients_match_oracle(net):
    _grads_match_oracle(net, 2, 700)   # several 128-row tiles and a ragged tail


def test_large_batch_gradients_match_oracle(net):
    """More than one 128-row tile per SM: the forward runs one tensor-core kernel
    per layer (training epilogue), the weight gradients take several tiles per
    CTA; a ragged tail as well."""
    n = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 + 300
    net.profile(True)
    _grads_match_oracle(net, 5, n)
    _, launches = net.profile_read(binding.GL_MLP_KERNEL_GEMM_FWD)
    net.profile(False)
    assert launches == 3                      # one per layer


def test_adam_step_matches_oracle(net):
    params, x, t = _setup(net, 3, 256)
    net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = unflatten(net.get_grads())
    net.adam(1e-3)
    torch.cuda.synchronize()
    got = unflatten(net.get_params())
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    ref, _, _ = omlp.adam_update(params, g, zeros, zeros, 1, 1e-3)
    for (W, b), (rW, rb) in zip(got, ref):
        np.testing.assert_allclose(W, rW, rtol=0, atol=2e-6)
        np.testing.assert_allclose(b, rb, rtol=0, atol=2e-6)


def test_training_reduces_loss(net):
    params, x, t = _setup(net, 4, 4096)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    first = net.loss_grad(xd, td)
    for _ in range(200):
        net.adam(2e-3)
        last = net.loss_grad(xd, td)
    assert last < 0.1 * first, (first, last)


def test_kernel_timing_counts_every_launch(net):
    """gl_mlp_profile brackets every launch of each kernel kind with events: one
    forward (the three-layer tensor-core kernel, input and output layers) and one
    loss-and-gradient call (another forward, 3 backward layer GEMMs, 3
    weight-gradient GEMMs)."""
    n = 700
    _, x, t = _setup(net, 3, n)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    net.profile(True)
    net.forward(xd, y)
    net.loss_grad(xd, td)
    got = [net.profile_read(k) for k in range(5)]
    net.profile(False)
    assert [c for _, c in got] == [2, 3, 3, 2, 2], got
    assert all(ms > 0.0 for ms, _ in got), got
    net.profile(True)   # enabling resets the accumulated times
    assert net.profile_read(binding.GL_MLP_KERNEL_GEMM_FWD) == (0.0, 0)
    net.profile(False)
    with pytest.raises(binding.GLError):
        net.profile_read(5)
    assert net.status() == binding.GL_OK


def test_large_batch_rows_match_the_fused_kernel(net):
    """Batches of more than one 128-row tile per SM run one tensor-core kernel per
    layer; at most one, a single kernel for the three layers.  Both do the same
    arithmetic on each row, so a row's output is the same bits either way."""
    props = torch.cuda.get_device_properties(0)
    n_big = props.multi_processor_count * 128 + 1000
    _, x, _ = _setup(net, 4, n_big)
    xd = torch.tensor(x, device="cuda")
    y_big = torch.empty(n_big, dtype=torch.float32, device="cuda")
    y_small = torch.empty(1000, dtype=torch.float32, device="cuda")
    net.profile(True)
    net.forward(xd, y_big)
    _, launches = net.profile_read(binding.GL_MLP_KERNEL_GEMM_FWD)
    net.profile(False)
    assert launches == 3                      # one per layer
    net.forward(xd[:1000], y_small)
    assert np.array_equal(y_big[:1000].cpu().numpy(), y_small.cpu().numpy())
    assert np.isfinite(y_big.cpu().numpy()).all()
    assert net.status() == binding.GL_OK
