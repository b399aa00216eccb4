"""Plain FP64 multilayer perceptron: the oracle of the surrogate network kernels.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

The surrogate is a fully connected network 7 -> 256 -> 256 -> 256 -> 256 -> 1 with
SiLU activations between layers and a linear output, trained on the mean squared
error.  This module computes, in float64 and with no blocking or fusion, the
forward pass, the loss and the backward pass (gradients of every weight and
bias) by the chain rule written out layer by layer.  The surrogate is not part of
the paper; it follows the statement of the workload (network shape, activation,
loss).

Parameters are a list of (W, b) per layer, W of shape (fan_in, fan_out), so a
layer computes z = x @ W + b.

``round_act`` (optional) is a rounding applied, as the workload's BF16 network
does, to every hidden activation SiLU(z) before the next layer uses it and to
every gradient with respect to a hidden pre-activation z before it is used (the
output layer's z and its gradient are not rounded).  With ``round_act`` None the
computation is the plain FP64 network.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (7, 256, 256, 256, 256, 1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(rng: np.random.Generator, widths=WIDTHS):
    """He-style uniform initialisation (for tests only)."""
    params = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / fi)
        params.append((rng.uniform(-lim, lim, (fi, fo)), rng.uniform(-0.1, 0.1, fo)))
    return params


def _identity(a):
    return a


def forward(params, x, round_act=None):
    """Returns the output (n,) and the per-layer inputs and pre-activations."""
    rnd = round_act or _identity
    a = np.asarray(x, dtype=np.float64)
    acts, pres = [a], []
    for li, (W, b) in enumerate(params):
        z = a @ W + b
        pres.append(z)
        a = rnd(silu(z)) if li + 1 < len(params) else z
        acts.append(a)
    return a[:, 0], (acts, pres)


def loss_and_grads(params, x, target, round_act=None):
    """Mean squared error over the batch and its gradient for every (W, b)."""
    rnd = round_act or _identity
    y, (acts, pres) = forward(params, x, round_act)
    n = y.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    dz = (2.0 / n) * r[:, None]                  # d loss / d z of the output layer
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (acts[li].T @ dz, dz.sum(axis=0))
        if li > 0:
            dz = rnd((dz @ W.T) * silu_grad(pres[li - 1]))
    return loss, grads


def adam_update(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), returns new params, m, v (float64)."""
    new_p, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p_, g_, m_, v_ in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m2 = beta1 * m_ + (1.0 - beta1) * g_
            v2 = beta2 * v_ + (1.0 - beta2) * g_ * g_
            mh = m2 / (1.0 - beta1 ** step)
            vh = v2 / (1.0 - beta2 ** step)
            out.append((p_ - lr * mh / (np.sqrt(vh) + eps), m2, v2))
        new_p.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_p, new_m, new_v
