"""Surrogate network kernels (tcgen05) against the FP64 MLP oracle.

The GPU network keeps BF16 copies of the three hidden weight matrices and BF16
activations; the oracle gets the same BF16-rounded hidden weights and runs in
FP64, so the comparison measures the kernels' arithmetic (BF16 activations,
FP32 accumulation) and layout, not a weight mismatch.  Tolerances are relative:
1.5e-2 on outputs and loss, 5e-2 on each layer's gradient (norm-wise)."""
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
    ref, _ = omlp.forward(as_gpu_sees(params), x.astype(np.float64))
    assert _rel(y.cpu().numpy(), ref) < 1.5e-2
    assert net.status() == binding.GL_OK


def test_gradients_match_oracle(net):
    n = 700                            # several 128-row tiles and a ragged tail
    params, x, t = _setup(net, 2, n)
    loss = net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = unflatten(net.get_grads())
    ref_loss, ref_g = omlp.loss_and_grads(as_gpu_sees(params), x.astype(np.float64), t)
    assert abs(loss - ref_loss) / ref_loss < 1.5e-2
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(g, ref_g)):
        assert _rel(gW, rW) < 5e-2, (li, _rel(gW, rW))
        assert _rel(gb, rb) < 5e-2, (li, _rel(gb, rb))
    assert net.status() == binding.GL_OK


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
