"""Oblate-minus-spherical flux surrogate: argument marshalling over the C-ABI.

Every number is computed by the library (include/gl.h): the training targets by
the exact FP64 GPU integrator (gl_flux_sky for the oblate planet, gl_flux_sphere
for the sphere of equal projected area) and gl_surrogate_targets, the features
by gl_surrogate_features, the initial parameters by gl_mlp_init, the training
(shuffle, learning-rate schedule, forward, backward, Adam) by gl_surrogate_train,
the held-out error table by gl_surrogate_error_table, the checkpoint by
gl_surrogate_save / gl_surrogate_load.  This module only moves arrays and loops
over epochs.  PyTorch holds device memory.

The surrogate is not part of the paper; it serves the light-curve path as a
cheaper replacement of the quadrature wherever its held-out error bound allows
(gl_lightcurve_surrogate), with the exact FP32 path as fallback.
"""
from __future__ import annotations

import json

import numpy as np

from . import binding, inputs

N_BINS = binding.SUR_BINS


def make_dataset(ctx: binding.Context, n: int, seed: int, chunk: int = 2_000_000) -> dict:
    """n samples of the surrogate box (inputs.surrogate_samples): features, targets
    (F_oblate - F_sphere) / R_eq^2, scale R_eq^2 and error-table bin, on the GPU."""
    import torch
    s = inputs.surrogate_samples(n, seed)
    u1, u2 = binding.gl_q_to_u(s["q1"], s["q2"])
    cols = dict(x0=s["x"], y0=s["y"], k=s["k"], f=s["f"], eta=s["eta"], xi=s["psi"], u1=u1,
                u2=u2)
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


def config(n: int, epochs: int, batch: int = 16384, lr: float = 2e-3, lr_end: float = 5e-5,
           seed: int = 0) -> binding.TrainConfig:
    """The gl_train_config of a run (Adam's usual betas and epsilon)."""
    return binding.TrainConfig(epochs=epochs, batch=batch, lr=lr, lr_end=lr_end, beta1=0.9,
                               beta2=0.999, eps=1e-8, seed=seed)


def steps_per_epoch(n: int, cfg: binding.TrainConfig) -> int:
    return -(-n // cfg.batch)


def train(mlp: binding.Mlp, data: dict, epochs: int, batch: int = 16384, lr: float = 2e-3,
          lr_end: float = 5e-5, seed: int = 0, log=None) -> list:
    """A whole run of gl_surrogate_train, one call per epoch; returns the mean
    training loss of each epoch."""
    n = data["t"].numel()
    cfg = config(n, epochs, batch, lr, lr_end, seed)
    spe = steps_per_epoch(n, cfg)
    history = []
    for ep in range(epochs):
        history.append(mlp.train(data["feat"], data["t"], cfg, ep * spe, spe))
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


def error_table(mlp: binding.Mlp, data: dict, err=None) -> np.ndarray:
    """Per bin, the largest |predicted - exact| normalised residual on the data
    (held-out samples), +inf for bins without samples (gl_surrogate_error_table);
    `err` (n float32 on the GPU, optional) receives the per-sample error."""
    return mlp.error_table(data["feat"], data["t"], data["bins"], err)


def save(path: str, mlp: binding.Mlp, table, cfg: binding.TrainConfig, train_step: int,
         meta: dict | None = None) -> None:
    """Checkpoint (gl_surrogate_save); `meta` (run notes, optional) goes to a JSON
    file beside it."""
    mlp.save(path, table, cfg, train_step)
    if meta is not None:
        with open(path + ".json", "w") as fh:
            json.dump(meta, fh, indent=1)


def load(path: str, mlp: binding.Mlp):
    """Restore a checkpoint into `mlp`; returns (table, TrainConfig, train_step)."""
    return mlp.load(path)
