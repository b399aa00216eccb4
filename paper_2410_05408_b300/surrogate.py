"""Oblate-minus-spherical flux surrogate: data, training, error table, checkpoint.

Every number here is computed by the library's kernels through the C-ABI:
the training targets come from the exact FP64 GPU integrator (gl_flux_sky for
the oblate planet, gl_flux_sphere for the sphere of equal projected area), the
features from gl_surrogate_features, the network's forward, backward and Adam
steps from the tcgen05 kernels of gl_mlp.  PyTorch only holds device memory and
shuffles sample indices.

The surrogate is not part of the paper; it serves the light-curve path as a
cheaper replacement of the quadrature wherever its held-out error bound allows
(gl_lightcurve_surrogate), with the exact FP32 path as fallback.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import binding, inputs

N_BINS = binding.SUR_BINS
WIDTHS = (7, 256, 256, 256, 256, 1)


def init_params(seed: int = 0, widths=WIDTHS) -> np.ndarray:
    """He-style uniform initial parameters in the layout gl_mlp expects: per layer
    the weights (fan_in x fan_out, row-major, U(-sqrt(6 / fan_in), +)) then the
    biases (U(-0.1, 0.1)), layers in order, as one float32 vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        lim = math.sqrt(6.0 / fi)
        parts.append(rng.uniform(-lim, lim, (fi, fo)).ravel())
        parts.append(rng.uniform(-0.1, 0.1, fo))
    return np.concatenate(parts).astype(np.float32)


def make_dataset(ctx: binding.Context, n: int, seed: int, chunk: int = 2_000_000) -> dict:
    """n samples of the surrogate box (inputs.surrogate_samples): features, targets
    (F_oblate - F_sphere) / R_eq^2, scale R_eq^2 and error-table bin, on the GPU."""
    import torch
    s = inputs.surrogate_samples(n, seed)
    u1, u2 = binding.gl_q_to_u(s["q1"], s["q2"])
    # the box is uniform in cos(eta) and in the position angle of the axis
    cols = dict(x0=s["x"], y0=s["y"], k=s["k"], f=s["f"], eta=np.arccos(s["cos_tilt"]),
                xi=s["psi"], u1=u1, u2=u2)
    feat = torch.empty((n, 7), dtype=torch.float32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    scale = torch.empty(n, dtype=torch.float32, device="cuda")
    bins = torch.empty(n, dtype=torch.int32, device="cuda")
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        d = {k: torch.tensor(v[a:b], dtype=torch.float64, device="cuda") for k, v in cols.items()}
        r_area = torch.empty(b - a, dtype=torch.float64, device="cuda")
        binding.gl_surrogate_features(ctx.handle, d["x0"], d["y0"], d["k"], d["f"], d["eta"],
                                      d["xi"], d["u1"], d["u2"], feat[a:b], scale[a:b], r_area,
                                      bins[a:b])
        z = torch.full((b - a,), -1.0, dtype=torch.float64, device="cuda")
        f_obl = torch.empty(b - a, dtype=torch.float64, device="cuda")
        f_sph = torch.empty(b - a, dtype=torch.float64, device="cuda")
        ctx.flux_sky(d["x0"], d["y0"], z, d["k"], d["f"], d["eta"], d["xi"], d["u1"], d["u2"],
                     f_obl, precision=binding.GL_FP64)
        ctx.flux_sphere(d["x0"], d["y0"], z, r_area, d["u1"], d["u2"], f_sph,
                        precision=binding.GL_FP64)
        binding.gl_surrogate_targets(ctx.handle, f_obl, f_sph, scale[a:b], t[a:b])
    torch.cuda.synchronize()
    return dict(feat=feat, t=t, scale=scale, bins=bins)


def train(mlp: binding.Mlp, data: dict, epochs: int, batch: int = 16384, lr: float = 2e-3,
          lr_end: float = 5e-5, seed: int = 0, log=None) -> list:
    """Mini-batch Adam with a cosine learning-rate schedule; returns the mean
    training loss of each epoch."""
    import torch
    n = data["t"].numel()
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    steps_per_epoch = (n + batch - 1) // batch
    total = epochs * steps_per_epoch
    step, history = 0, []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        acc, cnt = 0.0, 0
        for a in range(0, n, batch):
            idx = perm[a:a + batch]
            x = data["feat"].index_select(0, idx).contiguous()
            t = data["t"].index_select(0, idx).contiguous()
            loss = mlp.loss_grad(x, t)
            frac = step / max(1, total - 1)
            mlp.adam(lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * frac)))
            acc += loss
            cnt += 1
            step += 1
        history.append(acc / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {history[-1]:.3e}")
    return history


def predict(mlp: binding.Mlp, feat, chunk: int = 1 << 20):
    import torch
    n = feat.shape[0]
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        mlp.forward(feat[a:b], out[a:b])
    return out


def error_table(mlp: binding.Mlp, data: dict) -> np.ndarray:
    """Per bin, the largest |predicted - exact| normalised residual on the data
    (held-out samples); bins without samples get +inf (always fall back)."""
    import torch
    err = (predict(mlp, data["feat"]) - data["t"]).abs()
    b = data["bins"].long()
    keep = b >= 0
    table = torch.full((N_BINS,), -1.0, dtype=torch.float32, device="cuda")
    table.scatter_reduce_(0, b[keep], err[keep], reduce="amax", include_self=True)
    out = table.cpu().numpy()
    out[out < 0] = np.inf
    return out.astype(np.float32)


def flux_error_quantiles(mlp: binding.Mlp, data: dict, qs=(0.5, 0.99, 0.999, 1.0)) -> dict:
    """Quantiles of |error| in flux units (normalised error x R_eq^2) over the
    samples that overlap the star."""
    import torch
    err = ((predict(mlp, data["feat"]) - data["t"]).abs() * data["scale"])[data["bins"] >= 0]
    v = torch.quantile(err.double()[: 1 << 24], torch.tensor(qs, dtype=torch.float64,
                                                              device="cuda"))
    return {str(q): float(x) for q, x in zip(qs, v.cpu())}


def save(path: str, mlp: binding.Mlp, table: np.ndarray, meta: dict) -> None:
    """Checkpoint: FP32 parameters (.npy), error table and metadata (.json)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.save(path + ".params.npy", mlp.get_params())
    with open(path + ".json", "w") as fh:
        json.dump(dict(meta, table=[float(x) for x in table]), fh, indent=1)


def load(path: str, mlp: binding.Mlp):
    """Restore parameters into `mlp` (Adam state restarts); returns (table, meta)."""
    mlp.set_params(np.load(path + ".params.npy"))
    with open(path + ".json") as fh:
        meta = json.load(fh)
    return np.asarray(meta.pop("table"), dtype=np.float32), meta
