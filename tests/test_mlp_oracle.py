"""Pins of the FP64 MLP oracle (no GPU): central finite differences of the loss
for every parameter of a narrow network and sampled parameters of the full-width
one; forward pass and Adam step against torch's own CPU implementations."""
import numpy as np
import pytest

from oracle import mlp


def _fd_check(params, x, t, picks, h=1e-6, rtol=1e-6):
    _, grads = mlp.loss_and_grads(params, x, t)
    for li, which, idx in picks:
        W, b = params[li]
        arr = W if which == 0 else b
        old = arr[idx]
        arr[idx] = old + h
        lp, _ = mlp.loss_and_grads(params, x, t)
        arr[idx] = old - h
        lm, _ = mlp.loss_and_grads(params, x, t)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        an = grads[li][which][idx]
        assert abs(fd - an) <= rtol * max(1.0, abs(fd)) + 1e-9, (li, which, idx, fd, an)


def test_backward_matches_finite_differences_narrow_all_parameters():
    rng = np.random.default_rng(0)
    widths = (7, 8, 8, 1)
    params = mlp.init_params(rng, widths)
    x = rng.uniform(-1, 1, (16, 7))
    t = rng.normal(size=16)
    picks = []
    for li, (W, b) in enumerate(params):
        picks += [(li, 0, ij) for ij in np.ndindex(W.shape)]
        picks += [(li, 1, (j,)) for j in range(b.shape[0])]
    _fd_check(params, x, t, picks)


def test_backward_matches_finite_differences_full_width_sampled():
    rng = np.random.default_rng(1)
    params = mlp.init_params(rng)
    x = rng.uniform(-1, 1, (32, 7))
    t = rng.normal(size=32) * 0.1
    picks = []
    for li, (W, b) in enumerate(params):
        for _ in range(6):
            picks.append((li, 0, tuple(rng.integers(0, s) for s in W.shape)))
        picks.append((li, 1, (int(rng.integers(0, b.shape[0])),)))
    _fd_check(params, x, t, picks)


def test_forward_and_adam_match_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    params = mlp.init_params(rng)
    x = rng.uniform(-1, 1, (20, 7))
    t = rng.normal(size=20)
    layers = []
    for li, (W, b) in enumerate(params):
        lin = torch.nn.Linear(W.shape[0], W.shape[1]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W.T))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
        if li + 1 < len(params):
            layers.append(torch.nn.SiLU())
    net = torch.nn.Sequential(*layers)
    y, _ = mlp.forward(params, x)
    yt = net(torch.from_numpy(x)).detach().numpy()[:, 0]
    np.testing.assert_allclose(y, yt, rtol=1e-12, atol=1e-12)
    # one Adam step
    opt = torch.optim.Adam(net.parameters(), lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    loss = ((net(torch.from_numpy(x))[:, 0] - torch.from_numpy(t)) ** 2).mean()
    opt.zero_grad()
    loss.backward()
    opt.step()
    l0, grads = mlp.loss_and_grads(params, x, t)
    assert abs(l0 - float(loss)) < 1e-12
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    newp, _, _ = mlp.adam_update(params, grads, zeros, zeros, 1, 1e-3)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (W, b), lin in zip(newp, lins):
        np.testing.assert_allclose(W, lin.weight.detach().numpy().T, rtol=0, atol=1e-12)
        np.testing.assert_allclose(b, lin.bias.detach().numpy(), rtol=0, atol=1e-12)


def test_rounded_network_matches_torch_autograd():
    """The BF16 rounding hook, pinned against torch autograd of the same network
    built independently: hidden activations rounded to BF16 in the forward pass
    (identity gradient), and the gradient at each hidden pre-activation rounded to
    BF16 in the backward pass (a function that is the identity forward).  Also:
    every rounded quantity is a BF16 number, and the hook set to the identity
    reproduces the plain network bit for bit."""
    torch = pytest.importorskip("torch")

    def rnd_np(a):
        return torch.from_numpy(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()

    class RoundFwd(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            return a.to(torch.bfloat16).double()

        @staticmethod
        def backward(ctx, g):
            return g

    class RoundGrad(torch.autograd.Function):
        @staticmethod
        def forward(ctx, z):
            return z.clone()

        @staticmethod
        def backward(ctx, g):
            return g.to(torch.bfloat16).double()

    rng = np.random.default_rng(5)
    params = mlp.init_params(rng)
    x = rng.uniform(-1, 1, (24, 7))
    t = rng.normal(size=24) * 0.3
    tw = [(torch.from_numpy(W.copy()).requires_grad_(), torch.from_numpy(b.copy()).requires_grad_())
          for W, b in params]
    a = torch.from_numpy(x)
    for li, (W, b) in enumerate(tw):
        z = a @ W + b
        if li + 1 < len(tw):
            a = RoundFwd.apply(torch.nn.functional.silu(RoundGrad.apply(z)))
        else:
            a = z
    loss_t = ((a[:, 0] - torch.from_numpy(t)) ** 2).mean()
    loss_t.backward()
    y, (acts, _) = mlp.forward(params, x, round_act=rnd_np)
    np.testing.assert_allclose(y, a.detach().numpy()[:, 0], rtol=1e-12, atol=1e-12)
    for h in acts[1:-1]:
        assert np.array_equal(h, rnd_np(h))
    loss, grads = mlp.loss_and_grads(params, x, t, round_act=rnd_np)
    assert abs(loss - float(loss_t)) < 1e-12
    for (gW, gb), (W, b) in zip(grads, tw):
        np.testing.assert_allclose(gW, W.grad.numpy(), rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-14)
    l0, g0 = mlp.loss_and_grads(params, x, t)
    l1, g1 = mlp.loss_and_grads(params, x, t, round_act=lambda v: v)
    assert l0 == l1 and all(np.array_equal(p, q) for u, v in zip(g0, g1) for p, q in zip(u, v))
