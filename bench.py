"""Benchmark: oblate-planet transit flux evaluations per second on one B300.

Workload (default): the MCMC batch - 256 parameter sets x 2000 shared exposure
times (29.4-min cadence) x 15 sub-exposures = 7.68e6 flux evaluations per step,
parameters drawn uniformly over the MCMC box (seed 1).  A step is one call of
gl_lightcurve_batch over the whole batch with inputs resident in HBM; the timed
path is the FP32-compensated one (FP64 Kepler, roots and exposure sums), whose
max |delta flux| against the plain FP64 GPU path is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mcmc_batch|uneven_batch|single_transit|peaks|
                                surrogate_train|surrogate_mcmc|simpson_variant|
                                locked_batch|ensemble]

Under torchrun (N > 1) every rank evaluates its own batch (different seeds):
the work units are independent, so the ranks share no data-path collective
(weak scaling); the timed region is bracketed by barriers and the max over
ranks is reported.  ``--impl reference`` times the FP64 CPU oracle on this
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_05408_b300 import inputs  # noqa: E402

METRIC = "oblate flux evals/sec at |dflux|<=1e-7 (FP32) vs FP64 GPU path"
UNIT = "evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 / FP64 non-tensor peaks.  Measured in the same run by the pipe probes of
# libglpeaks.so (include/gl_peaks.h: independent FMA chains over 8 CTAs per SM,
# best of 5 launches); if the probe cannot run, derived from unit counts x
# maximum SM clock (148 SMs, 128 FP32 lanes and 2 FP64 lanes per SM, FMA = 2).
SM_COUNT = 148


def alu_peaks(sm_mhz: float):
    fp32 = SM_COUNT * 128 * 2 * sm_mhz * 1e6 / 1e12
    fp64 = SM_COUNT * 2 * 2 * sm_mhz * 1e6 / 1e12
    return fp32, fp64


def measured_alu_peaks(device: int, sm_mhz_fallback: float):
    """(FP32 TFLOP/s, FP64 TFLOP/s, MUFU Top/s, source) from the probes."""
    from paper_2410_05408_b300 import binding
    try:
        f32 = binding.glp_measure(device, binding.GLP_FFMA)["flops_per_s"] / 1e12
        f64 = binding.glp_measure(device, binding.GLP_DFMA)["flops_per_s"] / 1e12
        mufu = binding.glp_measure(device, binding.GLP_MUFU)["flops_per_s"] / 1e12
        return f32, f64, mufu, "of measured (FFMA/DFMA probe, libglpeaks, same run)"
    except Exception as e:   # noqa: BLE001 - reported in the line
        f32, f64 = alu_peaks(sm_mhz_fallback)
        return f32, f64, None, f"of derived (probe failed: {e}): unit counts x max SM clock"


# Algorithmic work per unit of the FP32C light-curve step (flops, FMA = 2),
# counted from the source, by kernel:
#   window (gl_win_kernel): HBM-bound; algorithmic bytes = the distinct times read
#         (8 B each: the shared grid once, or every exposure of a CSR batch) + 8 B
#         of flux written per exposure outside the window + 8 B of kept-list
#         entry per kept exposure; FP32 window test 12 per exposure, no FP64
#   exposures (gl_expgeo_kernel): FP64 per kept exposure 10 (exact window),
#         midpoint Kepler state 90 (one Halley step with its series, second-order
#         update, sky position); per sub-exposure FP32 position and class 40, and
#         FP64 Kepler 90 for sets without the Taylor expansion
#   quadrature (gl_items_quad_kernel, then gl_items_sum_kernel): FP32 whole-ellipse
#         item 840 (geometry and limb polynomial 35, Newton for the maximum 150,
#         16 nodes x 40, closed forms 15), crossing item 1590 (frame 90, FP32
#         Ferrari 290, Newton steps settling two roots on the frame's quartic 50,
#         breakpoints 40, closed forms 160, arcs 110, one inside arc of 16 nodes
#         x 56; the few items whose g may have two maxima add a 310-flop quartic);
#         no FP64 in a crossing item (the FP64 quartic runs only where the FP32
#         roots cannot be trusted: none on the MCMC batch); FP64 exposure sums 2
#         per sub-exposure
F32_EXPOSURE, F32_ITEM, F32_FULL, F32_PARTIAL = 12, 40, 840, 1590
F64_WINDOW, F64_KEPLER, F64_PARTIAL, F64_SUM = 10, 90, 0, 2


def kernel_flops(c: dict) -> dict:
    """(FP32, FP64) algorithmic flops of one step, per ALU-bound kernel group."""
    return {
        "exposures": (c["items"] * F32_ITEM,
                      c["kept"] * F64_WINDOW + (c["kepler"] + c["item_kepler"]) * F64_KEPLER),
        "quadrature": (c["full"] * F32_FULL + c["partial"] * F32_PARTIAL,
                       c["partial"] * F64_PARTIAL + c["items"] * F64_SUM),
    }


def window_bytes(c: dict, time_bytes: int) -> int:
    """Algorithmic DRAM bytes of one window-kernel launch."""
    return time_bytes + 8 * (c["exposures"] - c["kept"]) + 8 * c["kept"]


def alu_roofline(f32: float, f64: float, ms: float, fp32_peak: float, fp64_peak: float,
                 peak_source: str = "derived: 148 SMs x (128 FP32 | 2 FP64) lanes x 2 flops x "
                                    "max SM clock") -> dict:
    """Algorithmic FP32 and FP64 flops over a CUDA-event duration, against the
    pipe that bounds them (the larger of flops/peak)."""
    t = ms * 1e-3
    a32, a64 = f32 / t / 1e12, f64 / t / 1e12
    pipe = "fp64" if f64 / fp64_peak >= f32 / fp32_peak else "fp32"
    ach, peak = (a64, fp64_peak) if pipe == "fp64" else (a32, fp32_peak)
    return {"bound": "alu", "pipe": pipe, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak,
            "fp32": {"achieved": a32, "peak": fp32_peak, "frac": a32 / fp32_peak,
                     "flops_per_launch": f32},
            "fp64": {"achieved": a64, "peak": fp64_peak, "frac": a64 / fp64_peak,
                     "flops_per_launch": f64},
            "kernel_ms": ms,
            "peak_source": peak_source}


def hbm_roofline(nbytes: float, ms: float, hbm_peak) -> dict:
    """Algorithmic bytes over a CUDA-event duration against the copy bandwidth
    (the measured one, else the fallback 6.4 TB/s)."""
    src = "of measured (STREAM-style copy)" if hbm_peak else "of fallback (6.4 TB/s)"
    hbm_peak = hbm_peak or 6400.0
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": ach / hbm_peak, "bytes_per_launch": nbytes, "kernel_ms": ms,
            "peak_source": src}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, summed over
# the kernels of the group) from one ncu capture of the current kernels on the
# workload named (the launch lists under profiles/); None where no capture of the
# current kernel exists, and for other workloads.
TRAFFIC = {("mcmc_batch", "window"): 0.083e6,
           ("mcmc_batch", "exposures"): 0.337e6,
           ("mcmc_batch", "quadrature"): 3.148e6 + 1.763e6,
           ("uneven_batch", "window"): 471.2e6,
           ("uneven_batch", "exposures"): 81.9e6,
           ("uneven_batch", "quadrature"): 74.7e6 + 41.5e6}

KERNEL_NAMES = {"window": "gl_win_kernel", "exposures": "gl_expgeo_kernel",
                "quadrature": "gl_items_quad_kernel+gl_items_sum_kernel"}


def roofline(c: dict, kern: dict, fp32_peak: float, fp64_peak: float, hbm_peak: float,
             time_bytes: int, workload: str = "", peak_source: str = None) -> dict:
    """Roofline of the dominant kernel of the FP32C step (the one with the largest
    measured time), with every kernel's own figures beside it."""
    extra = {"peak_source": peak_source} if peak_source else {}
    per = {k: alu_roofline(*f, kern[k], fp32_peak, fp64_peak, **extra)
           for k, f in kernel_flops(c).items() if kern.get(k)}
    if kern.get("window"):
        per["window"] = hbm_roofline(window_bytes(c, time_bytes), kern["window"], hbm_peak)
    top = max(per, key=lambda k: per[k]["kernel_ms"])
    line = dict(per[top])
    line.update({"kernel": KERNEL_NAMES[top], "traffic": TRAFFIC.get((workload, top)),
                 "kernels": {KERNEL_NAMES[k]: {"ms": v["kernel_ms"], "bound": v["bound"],
                                               "pipe": v.get("pipe"), "frac": v["frac"],
                                               "traffic": TRAFFIC.get((workload, k))}
                             for k, v in per.items()}})
    return line


def workload(name: str, seed_offset: int = 0):
    if name == "mcmc_batch":
        return inputs.mcmc_batch(seed=1 + 1000 * seed_offset)
    if name == "uneven_batch":
        return inputs.uneven_batch(seed=2 + 1000 * seed_offset)
    if name == "single_transit":
        return inputs.single_transit()
    raise SystemExit(f"unknown workload {name}")


def n_evals(wl) -> int:
    n_sets = len(wl["params"]["t0"])
    ns = wl["nsuper"]
    if wl.get("offsets") is None:
        per = np.full(n_sets, len(wl["t"]), dtype=np.int64)
    else:
        per = np.diff(wl["offsets"])
    nsa = np.broadcast_to(np.asarray(ns, dtype=np.int64), (n_sets,))
    return int(np.sum(per * nsa))


def n_exposures(wl) -> int:
    n_sets = len(wl["params"]["t0"])
    return n_sets * len(wl["t"]) if wl.get("offsets") is None else int(wl["offsets"][-1])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(1.0)   # nvidia-smi's start-up stays out of the timed region
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup(backend: str = None):
    """Rank layout from the torchrun environment; NCCL on GPUs, gloo otherwise."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    """Max over ranks (timing only: the work units share no data)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world: int, evals_per_rank_step: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank evaluates its own batch of the same size."""
    return world * evals_per_rank_step * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_sample(wl, max_sets: int):
    """A bounded, seeded sample of the workload's parameter sets."""
    n_sets = len(wl["params"]["t0"])
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(n_sets, min(max_sets, n_sets), replace=False))
    return idx


def run_oracle(wl, idx, nthreads=0):
    import oracle
    p = {k: np.asarray(v, dtype=np.float64)[idx] for k, v in wl["params"].items()}
    if "u1" not in p:
        u = np.array([oracle.q_to_u(a, b) for a, b in zip(p.pop("q1"), p.pop("q2"))])
        p["u1"], p["u2"] = u[:, 0].copy(), u[:, 1].copy()
    exptime = np.broadcast_to(np.asarray(wl["exptime"], dtype=np.float64),
                              (len(wl["params"]["t0"]),))[idx]
    ns = wl["nsuper"]
    ns_sub = ns if np.ndim(ns) == 0 else np.asarray(ns)[idx]
    if wl.get("offsets") is None:
        t_sub, off_sub = wl["t"], None
        evals = len(idx) * len(wl["t"]) * int(ns)
    else:
        off = wl["offsets"]
        lengths = np.diff(off)[idx]
        off_sub = np.zeros(len(idx) + 1, dtype=np.int64)
        off_sub[1:] = np.cumsum(lengths)
        t_sub = np.concatenate([wl["t"][off[s]:off[s + 1]] for s in idx])
        evals = int(np.sum(lengths * np.asarray(ns_sub)))
    t0 = time.perf_counter()
    ref = oracle.lightcurve(p, t_sub, exptime, ns_sub, offsets=off_sub, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return evals, dt, oracle.max_threads(), np.asarray(ref).reshape(-1)


def sample_outputs(wl, idx, out: np.ndarray) -> np.ndarray:
    """The GPU outputs of the sampled parameter sets, in the oracle's layout."""
    if wl.get("offsets") is None:
        return out.reshape(len(wl["params"]["t0"]), len(wl["t"]))[idx].reshape(-1)
    off = wl["offsets"]
    return np.concatenate([out[off[s]:off[s + 1]] for s in idx])


def cpu_baseline(wl, sample_sets: int, min_seconds: float = 10.0, gpu_out=None):
    """The oracle on a seeded sample of the workload's parameter sets (all their
    exposures and sub-exposures), repeated until at least min_seconds of CPU work.
    With gpu_out (the timed path's output), also the max |dflux| of that path
    against the oracle over the sample."""
    idx = oracle_sample(wl, sample_sets)
    evals, dt, reps = 0, 0.0, 0
    ref = None
    while dt < min_seconds or reps == 0:
        e, t, cores, ref = run_oracle(wl, idx)
        evals += e
        dt += t
        reps += 1
    res = {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(idx)} of {len(wl['params']['t0'])} parameter sets, all their "
                     f"exposures and sub-exposures, {reps} passes ({evals} evals, {dt:.1f} s)"}
    if gpu_out is not None:
        got = sample_outputs(wl, idx, gpu_out)
        res["max_dflux_vs_oracle"] = float(np.max(np.abs(got - ref)))
        res["sample_exposures"] = int(ref.size)
        res["sample_in_transit"] = int(np.sum(ref < 1.0))
    return res


def peaks_arm(args):
    """Measured non-tensor pipe throughput of this GPU (libglpeaks probes), with
    the SM clock sampled while they run: the denominators of the ALU rooflines."""
    from paper_2410_05408_b300 import binding, build
    build.build()
    world, rank, local = dist_setup()
    res = {}
    with ClockSampler(local) as clk:
        for name, kind in (("ffma", binding.GLP_FFMA), ("dfma", binding.GLP_DFMA),
                           ("mufu_rsqrt", binding.GLP_MUFU)):
            res[name] = binding.glp_measure(local, kind, repeats=max(3, args.steps))
    clocks = clk.summary()
    if rank != 0:
        return
    line = {"metric": "non-tensor pipe throughput", "unit": "TFLOP/s (FMA = 2 flops; MUFU: Top/s)",
            "value": res["ffma"]["flops_per_s"] / 1e12, "n_gpus": 1, "steps": max(3, args.steps),
            "warmup": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "peaks", "grid": "8 x 256-thread CTAs per SM",
                       "chains": "FFMA 8, DFMA 4, MUFU 8 independent chains per thread"},
            "fp32_tflops": res["ffma"]["flops_per_s"] / 1e12,
            "fp64_tflops": res["dfma"]["flops_per_s"] / 1e12,
            "mufu_tops": res["mufu_rsqrt"]["flops_per_s"] / 1e12,
            "fp32_to_fp64": res["ffma"]["flops_per_s"] / res["dfma"]["flops_per_s"],
            "best_ms": {k: v["best_ms"] for k, v in res.items()},
            "clocks": clocks}
    print(json.dumps(line))


def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    wl = workload(args.workload)
    sample = args.ref_sets
    idx = oracle_sample(wl, sample)
    for _ in range(args.warmup):
        run_oracle(wl, idx[:1])
    tot_evals, tot_t, cores = 0, 0.0, 1
    for _ in range(args.steps):
        e, dt, cores, _ = run_oracle(wl, idx)
        tot_evals += e
        tot_t += dt
    value = tot_evals / tot_t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "parallelism": "cpu-openmp"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(idx)} parameter sets per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ surrogate workloads
MLP_TRAIN_FLOPS = 3 * 2 * (7 * 256 + 3 * 256 * 256 + 256)   # forward + 2x backward, per sample
MLP_TC_TRAIN_FLOPS = 3 * 2 * 3 * 256 * 256                # the tensor-core part of it


def stretch_move(logp, walkers: np.ndarray, rng, a: float = 2.0):
    """One sweep of the affine-invariant stretch move (Goodman and Weare 2010):
    each half of the ensemble proposes moves along lines through members of the
    other half; `logp` evaluates all proposals at once on the GPU."""
    n, d = walkers.shape
    lp = logp(walkers)
    acc = 0
    for half in (0, 1):
        act = np.arange(half, n, 2)
        oth = np.arange(1 - half, n, 2)
        zz = ((a - 1.0) * rng.uniform(size=act.size) + 1.0) ** 2 / a
        partner = walkers[rng.choice(oth, act.size)]
        prop = partner + zz[:, None] * (walkers[act] - partner)
        full = walkers.copy()
        full[act] = prop
        lp_new = logp(full)[act]
        logr = (d - 1) * np.log(zz) + lp_new - lp[act]
        ok = np.log(rng.uniform(size=act.size)) < logr
        walkers[act[ok]] = prop[ok]
        lp[act[ok]] = lp_new[ok]
        acc += int(ok.sum())
    return walkers, acc / n


def flux_error_quantiles(err, data, qs=(0.5, 0.99, 0.999, 1.0)) -> dict:
    """Quantiles of the held-out |error| in flux units (normalised error x R_eq^2)
    over the samples that overlap the star (reporting only)."""
    e = (err * data["scale"])[data["bins"] >= 0].double().cpu().numpy()
    return {str(q): float(np.quantile(e, q)) for q in qs}


def surrogate_train_arm(args):
    import torch
    from paper_2410_05408_b300 import binding, build, surrogate
    build.build()
    ctx = binding.Context(0)
    mlp = binding.Mlp(0)
    mlp.init(0)
    t0 = time.perf_counter()
    train = surrogate.make_dataset(ctx, args.sur_train, seed=3)
    held = surrogate.make_dataset(ctx, args.sur_held, seed=1003)
    gen_s = time.perf_counter() - t0
    # timed training: CUDA events around every step (forward + backward + Adam)
    batch = args.sur_batch
    n = train["t"].numel()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    hist = surrogate.train(mlp, train, epochs=args.sur_epochs, batch=batch, lr=args.sur_lr)
    ev1.record()
    torch.cuda.synchronize()
    train_s = ev0.elapsed_time(ev1) * 1e-3
    samples = args.sur_epochs * n
    err = torch.empty_like(held["t"])
    table = surrogate.error_table(mlp, held, err)
    q = flux_error_quantiles(err, held)
    if args.sur_save:
        cfg = surrogate.config(n, args.sur_epochs, batch, args.sur_lr)
        surrogate.save(args.sur_save, mlp, table, cfg,
                       args.sur_epochs * surrogate.steps_per_epoch(n, cfg),
                       dict(train=n, epochs=args.sur_epochs, batch=batch, history=hist))
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    tc = samples * MLP_TC_TRAIN_FLOPS / train_s / 1e12
    # inference forward of one training batch (its three 256 x 256 layers run on
    # the tensor cores; the 7-wide input and 1-wide output layers on CUDA cores),
    # CUDA events around 50 calls after 5 untimed ones
    fb = min(batch, held["t"].numel())
    fx, fy = held["feat"][:fb], torch.empty(fb, dtype=torch.float32, device="cuda")
    for _ in range(5):
        mlp.forward(fx, fy)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(50):
        mlp.forward(fx, fy)
    f1.record()
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / 50
    fwd_tf = fb * 3 * 2 * 256 * 256 / (fwd_ms * 1e-3) / 1e12
    # the layer GEMM kernel alone: CUDA events around each launch (gl_mlp_profile)
    mlp.profile(True)
    for _ in range(20):
        mlp.forward(fx, fy)
    torch.cuda.synchronize()
    g_ms, g_n = mlp.profile_read(binding.GL_MLP_KERNEL_GEMM_FWD)
    i_ms, i_n = mlp.profile_read(binding.GL_MLP_KERNEL_IN)
    o_ms, o_n = mlp.profile_read(binding.GL_MLP_KERNEL_OUT)
    mlp.profile(False)
    gemm_ms = g_ms / 20            # per forward (one launch at this batch)
    gemm_tf = fb * 3 * 2 * 256 * 256 / (gemm_ms * 1e-3) / 1e12
    burst = peaks.get("bf16_tflops", 1718.5)
    line = {"metric": "surrogate training samples/sec (forward + backward + Adam)",
            "value": samples / train_s, "unit": "samples/s", "n_gpus": 1,
            "steps": args.sur_epochs * ((n + batch - 1) // batch), "warmup": 0,
            "higher_is_better": True, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": "surrogate_train", "train_samples": n,
                       "heldout_samples": held["t"].numel(), "epochs": args.sur_epochs,
                       "batch": batch, "network": "7-256-256-256-256-1 SiLU"},
            "data_generation_s": gen_s, "train_s": train_s, "loss_history": hist,
            "tensor_core": {"achieved_tflops": tc,
                            "peak": peaks.get("bf16_tflops_sustained", 1407.5),
                            "frac": tc / peaks.get("bf16_tflops_sustained", 1407.5),
                            "note": "3 hidden 256x256 layers, forward + 2 backward GEMMs, "
                                    "whole training step time (incl. CUDA-core layers, Adam)"},
            "forward_batch": {"rows": fb, "ms": fwd_ms, "tensor_tflops": fwd_tf,
                              "peak": burst, "frac": fwd_tf / burst,
                              "note": "the three-layer tensor-core kernel plus the CUDA-core "
                                      "input and output layers, against the burst BF16 peak"},
            "gemm_kernel": {"kernel": "gl_mlp_fwd3_kernel (the three hidden layers)", "rows": fb,
                            "ms": gemm_ms, "launches": g_n, "bound": "tensor",
                            "tensor_tflops": gemm_tf, "peak": burst, "frac": gemm_tf / burst,
                            "input_layer_ms": i_ms / max(i_n, 1),
                            "output_layer_ms": o_ms / max(o_n, 1),
                            "note": "CUDA events around each launch, back-to-back forwards "
                                    "(weights and activations in L2), against the burst "
                                    "BF16 peak"},
            "heldout_flux_error_quantiles": q,
            "error_table_normalised": [float(x) for x in table]}
    print(json.dumps(line))


def surrogate_mcmc_arm(args):
    import torch
    from paper_2410_05408_b300 import binding, build, surrogate
    build.build()
    ctx = binding.Context(0)
    mlp = binding.Mlp(0)
    if args.sur_load:
        table, _, _ = surrogate.load(args.sur_load, mlp)
    else:   # no saved surrogate: train one here (untimed), as the training arm does
        mlp.init(0)
        train = surrogate.make_dataset(ctx, args.sur_train, seed=3)
        held = surrogate.make_dataset(ctx, args.sur_held, seed=1003)
        surrogate.train(mlp, train, epochs=args.sur_epochs, batch=args.sur_batch, lr=args.sur_lr)
        table = surrogate.error_table(mlp, held)
        del train, held
    wl = inputs.injected_curve(n_walkers=args.walkers)
    names = binding.PARAM_NAMES
    nt = len(wl["t"])
    t = torch.tensor(wl["t"], device="cuda")
    exp = torch.full((args.walkers,), wl["exptime"], dtype=torch.float64, device="cuda")
    p = {k: torch.tensor(np.ascontiguousarray(wl["walkers"][k]), dtype=torch.float64,
                         device="cuda") for k in names}
    out_s = torch.empty(args.walkers * nt, dtype=torch.float64, device="cuda")
    out_e = torch.empty_like(out_s)
    evals = args.walkers * nt * wl["nsuper"]

    def run_s():
        return binding.gl_lightcurve_surrogate(ctx.handle, mlp, p, t, out_s, table,
                                               args.sur_limit, exptime=exp,
                                               nsuper_all=wl["nsuper"])

    def run_e():
        ctx.lightcurve(p, t, out_e, exp, nsuper_all=wl["nsuper"], precision=binding.GL_FP32C)

    for _ in range(args.warmup):
        stats = run_s()
        run_e()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        stats = run_s()
    torch.cuda.synchronize()
    ts = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run_e()
    torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / args.steps
    # accuracy against the FP64 GPU path (the path the GPU tests hold to the oracle)
    out_64 = torch.empty_like(out_s)
    run_s()
    ctx.lightcurve(p, t, out_64, exp, nsuper_all=wl["nsuper"], precision=binding.GL_FP64)
    torch.cuda.synchronize()
    max_err = float((out_s - out_64).abs().max().item())
    # a few sweeps of an ensemble sampler on the injected data, likelihood on the GPU
    truth = {k: float(wl["truth"][k][0]) for k in names}
    flux_true = torch.empty(nt, dtype=torch.float64, device="cuda")
    ctx.lightcurve({k: torch.tensor([truth[k]], dtype=torch.float64, device="cuda")
                    for k in names}, t, flux_true, exp[:1], nsuper_all=wl["nsuper"],
                   precision=binding.GL_FP64)
    data = flux_true + torch.tensor(wl["noise"], device="cuda")
    sigma = torch.full((nt,), 1e-4, dtype=torch.float64, device="cuda")
    free = ["t0", "b", "k", "f", "eta", "xi"]
    ll = torch.empty(args.walkers, dtype=torch.float64, device="cuda")

    def logp(wk):
        for i, name in enumerate(free):
            p[name].copy_(torch.tensor(wk[:, i]))
        bad = (wk[:, 3] < 0) | (wk[:, 3] > 0.9) | (wk[:, 1] < 0) | (wk[:, 2] <= 0)
        run_s()
        binding.gl_loglike(ctx.handle, out_s, data, sigma, ll)
        v = ll.cpu().numpy().copy()
        v[bad] = -np.inf
        return v

    walkers = np.stack([wl["walkers"][n_] for n_ in free], axis=1)
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    accs = []
    for _ in range(args.sweeps):
        walkers, a = stretch_move(logp, walkers, rng)
        accs.append(a)
    sweep_s = (time.perf_counter() - t0) / max(args.sweeps, 1)
    line = {"metric": "surrogate-in-the-loop likelihood evals/sec", "value": evals / ts,
            "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ts * 1e3, "higher_is_better": True, "dtype": "bf16+f32+f64",
            "data": "synthetic", "config": {"workload": "surrogate_mcmc",
                                            "walkers": args.walkers, "exposures": nt,
                                            "nsuper": wl["nsuper"],
                                            "bound_limit": args.sur_limit},
            "exact_fp32c": {"value": evals / te, "ms_per_step": te * 1e3},
            "gain_vs_exact": te / ts, "fallback": stats,
            "fallback_fraction": stats["fallback"] / max(stats["items"], 1),
            "max_dflux_vs_fp64_gpu": max_err,
            "sampler": {"sweeps": args.sweeps, "acceptance": accs, "s_per_sweep": sweep_s}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
def simpson_arm(args):
    """Geometry-level comparison of the split Gauss-Legendre path (gl_flux_sky)
    with the paper's snapped Simpson scheme (gl_flux_sky_simpson) at several N:
    evaluations/s over a large geometry sample (device-resident, CUDA events) and
    max |dflux| against the FP64 split path (the path the GPU tests hold to the
    oracle within 1e-10) over the whole sample."""
    import torch
    from paper_2410_05408_b300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    n = 200_000
    g = inputs.geometry_sample(n, seed=41)
    g["u1"], g["u2"] = binding.gl_q_to_u(g["q1"], g["q2"])
    d = [torch.as_tensor(np.ascontiguousarray(g[q]), device=dev)
         for q in ("x0", "y0", "z", "k", "f", "eta", "xi", "u1", "u2")]
    out = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ref_d = torch.empty(n, dtype=torch.float64, device=dev)
    ctx.flux_sky(*d, ref_d, precision=binding.GL_FP64, stream=stream)
    torch.cuda.synchronize(dev)

    def measure(call):
        for _ in range(args.warmup):
            call()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            call()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / args.steps
        err = float((out - ref_d).abs().max().item())
        return {"evals_per_s": n / (ms * 1e-3), "ms": ms, "max_dflux_vs_fp64_split": err}

    rows = {}
    for name, prec in (("fp32", binding.GL_FP32C), ("fp64", binding.GL_FP64)):
        rows[f"split_gauss_legendre_{name}"] = measure(
            lambda: ctx.flux_sky(*d, out, precision=prec, stream=stream))
        for n_int in (64, 256, 1024, 4096, 16384):
            rows[f"simpson_{name}_N{n_int}"] = measure(
                lambda: ctx.flux_sky_simpson(*d, out, n_int, precision=prec, stream=stream))
    best = rows["split_gauss_legendre_fp32"]
    line = {"metric": "geometry-level flux evals/s, split Gauss-Legendre vs the paper's snapped "
                      "Simpson scheme", "value": best["evals_per_s"], "unit": "evals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": best["ms"], "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "simpson_variant", "geometries": n,
                       "sample": "geometry_sample(seed=41)"},
            "paths": rows}
    print(json.dumps(line))
    ctx.close()


def locked_arm(args):
    """Tidally locked light curves (gl_lightcurve_locked, projection per
    sub-exposure) against the unlocked item pipeline on the same close-in,
    triaxial planets: evals/s of each, L2 flushed before every step."""
    import torch
    from paper_2410_05408_b300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    wl = inputs.locked_batch(n_sets=256, n_times=2000, seed=61)
    p = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in wl["params"].items()}
    p["u1"], p["u2"] = binding.gl_q_to_u(p.pop("q1"), p.pop("q2"))
    n_sets, n_t = len(p["t0"]), len(wl["t"])
    dp = {k: torch.as_tensor(v, device=dev) for k, v in p.items()}
    d_t = torch.as_tensor(np.ascontiguousarray(wl["t"]), device=dev)
    d_exp = torch.as_tensor(np.ascontiguousarray(wl["exptime"]), device=dev)
    out = torch.empty(n_sets * n_t, dtype=torch.float64, device=dev)
    evals = n_sets * n_t * int(wl["nsuper"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = {}
    for name, prec, locked in (("locked_fp32c", binding.GL_FP32C, True),
                               ("locked_fp64", binding.GL_FP64, True),
                               ("unlocked_fp32c", binding.GL_FP32C, False),
                               ("unlocked_fp64", binding.GL_FP64, False)):
        def step():
            ctx.lightcurve(dp, d_t, out, d_exp, nsuper_all=int(wl["nsuper"]), precision=prec,
                           stream=stream, locked=locked)
        for _ in range(args.warmup):
            step()
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms += a.elapsed_time(b)
        rows[name] = {"evals_per_s": evals / (ms / args.steps * 1e-3), "ms": ms / args.steps}
    line = {"metric": "tidally locked light-curve evals/s (projection per sub-exposure)",
            "value": rows["locked_fp32c"]["evals_per_s"], "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": rows["locked_fp32c"]["ms"], "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "locked_batch", "parameter_sets": n_sets, "exposures": n_t,
                       "nsuper": int(wl["nsuper"]), "evals_per_step": evals,
                       "l2": "flushed between steps (256 MB write)"},
            "paths": rows}
    print(json.dumps(line))
    ctx.close()


def ensemble_arm(args):
    """The device-resident stretch-move ensemble (gl_ensemble_sweep) on the
    injected single-transit curve: 1024 walkers in the (mu, nu) parameterisation
    of Appendix A, 3000 exposures x 15; sweeps/s and light-curve evaluations/s
    (two half-ensembles of proposals per sweep), CUDA events around the sweeps."""
    import torch
    from paper_2410_05408_b300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    ctx = binding.Context(0)
    inj = inputs.injected_curve(n_walkers=args.walkers)
    tr = {k: float(v[0]) for k, v in inj["truth"].items()}
    u1, u2 = tr["u1"], tr["u2"]
    q1 = (u1 + u2) ** 2
    q2 = u1 / (2.0 * (u1 + u2))
    # (mu, nu) of the truth, through the library's own kernel
    f_d = torch.tensor([tr["f"]], dtype=torch.float64, device=dev)
    e_d = torch.tensor([tr["eta"]], dtype=torch.float64, device=dev)
    mu_d, nu_d = torch.empty_like(f_d), torch.empty_like(f_d)
    binding.gl_munu(ctx.handle, "to_munu", f_d, e_d, mu_d, nu_d)
    truth = np.array([tr["t0"], tr["period"], tr["a_rs"], tr["b"], tr["k"], float(mu_d.item()),
                      float(nu_d.item()), tr["xi"], q1, q2])
    lo = np.array([-0.2, 540.0, 150.0, 0.0, 0.03, -1.0, 0.0, 0.0, 0.0, 0.0])
    hi = np.array([0.2, 544.0, 300.0, 0.9, 0.12, 1.0, 1.0, np.pi, 1.0, 1.0])
    rng = np.random.default_rng(8)
    n = args.walkers
    scale = np.array([1e-3, 1e-3, 0.5, 0.01, 1e-4, 0.01, 0.01, 0.01, 0.01, 0.01])
    X = np.clip(truth + scale * rng.standard_normal((n, 10)), lo + 1e-9, hi - 1e-9)
    # data: the model at the truth (library FP64 path) plus the seeded noise
    t = np.ascontiguousarray(inj["t"])
    d_t = torch.as_tensor(t, device=dev)
    p_true = {k: torch.tensor([float(v[0])], dtype=torch.float64, device=dev)
              for k, v in inj["truth"].items()}
    model = torch.empty(t.size, dtype=torch.float64, device=dev)
    ctx.lightcurve(p_true, d_t, model, torch.full((1,), inj["exptime"], dtype=torch.float64,
                                                  device=dev),
                   nsuper_all=inj["nsuper"], precision=binding.GL_FP64)
    data = model + torch.as_tensor(inj["noise"], device=dev)
    sigma = torch.full_like(data, 1e-4)
    walkers = torch.as_tensor(X, device=dev).contiguous()
    ens = binding.Ensemble(ctx, walkers, torch.as_tensor(lo, device=dev),
                           torch.as_tensor(hi, device=dev), d_t, data, sigma, inj["exptime"],
                           inj["nsuper"], precision=binding.GL_FP32C)
    ens.init()
    gen = torch.Generator(device=dev)
    gen.manual_seed(9)
    acc = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        ens.sweep(torch.rand(3 * n, dtype=torch.float64, device=dev, generator=gen), acc)
    rnd = [torch.rand(3 * n, dtype=torch.float64, device=dev, generator=gen)
           for _ in range(args.sweeps)]
    acc.zero_()
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for r in rnd:
        ens.sweep(r, acc, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.sweeps
    evals = n * t.size * inj["nsuper"]
    status = ctx.sync()
    line = {"metric": "device-resident stretch-move sweeps: light-curve evals/s", "value":
            evals / (ms * 1e-3), "unit": "evals/s", "n_gpus": 1, "steps": args.sweeps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "ensemble", "walkers": n, "exposures": int(t.size),
                       "nsuper": int(inj["nsuper"]), "parameterisation": "(mu, nu) Appendix A"},
            "sweeps_per_s": 1e3 / ms, "acceptance": int(acc.item()) / (n * args.sweeps),
            "status": status}
    print(json.dumps(line))
    ctx.close()


def pin_config(ctx, spec: str) -> None:
    """Pin the kernel configuration from 'nodes=N,quad=C,exp=B,quad64=C,exp64=B'."""
    from paper_2410_05408_b300 import binding
    kv = dict(item.split("=") for item in spec.split(","))
    ctx.configure(binding.GL_FP32C, nodes=int(kv.get("nodes", 0)),
                  quad_ctas=int(kv.get("quad", 0)), exposure_block=int(kv.get("exp", 0)))
    ctx.configure(binding.GL_FP64, quad_ctas=int(kv.get("quad64", 0)),
                  exposure_block=int(kv.get("exp64", 0)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mcmc_batch")
    ap.add_argument("--ref-sets", type=int, default=96)
    ap.add_argument("--cpu-sets", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="",
                    help="pin the configuration instead of autotuning it, as "
                         "'nodes=N,quad=C,exp=B,quad64=C,exp64=B' (a previous run's "
                         "autotune reports)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run warm-up + steps FP32C steps of the workload and exit "
                         "(a profiler's target; prints no bench line)")
    ap.add_argument("--sur-train", type=int, default=10_000_000)
    ap.add_argument("--sur-held", type=int, default=1_000_000)
    ap.add_argument("--sur-epochs", type=int, default=6)
    ap.add_argument("--sur-batch", type=int, default=16384)
    ap.add_argument("--sur-lr", type=float, default=2e-3)
    ap.add_argument("--sur-save", default="")
    ap.add_argument("--sur-load", default="")
    ap.add_argument("--sur-limit", type=float, default=1e-6)
    ap.add_argument("--walkers", type=int, default=1024)
    ap.add_argument("--sweeps", type=int, default=5)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "surrogate_train":
        return surrogate_train_arm(args)
    if args.workload == "surrogate_mcmc":
        return surrogate_mcmc_arm(args)
    if args.workload == "simpson_variant":
        return simpson_arm(args)
    if args.workload == "locked_batch":
        return locked_arm(args)
    if args.workload == "ensemble":
        return ensemble_arm(args)
    if args.workload == "peaks":
        return peaks_arm(args)

    import torch
    from paper_2410_05408_b300 import binding, build

    world, rank, local = dist_setup()
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(local)

    wl = workload(args.workload, seed_offset=rank)
    p = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in wl["params"].items()}
    if "u1" not in p:
        p["u1"], p["u2"] = binding.gl_q_to_u(p.pop("q1"), p.pop("q2"))
    p = {k: p[k] for k in binding.PARAM_NAMES}
    n_sets = len(p["t0"])
    exptime = np.ascontiguousarray(np.broadcast_to(wl["exptime"], (n_sets,)), dtype=np.float64)
    ns = np.ascontiguousarray(np.broadcast_to(np.asarray(wl["nsuper"], dtype=np.int32), (n_sets,)))
    t = np.ascontiguousarray(wl["t"], dtype=np.float64)
    offsets = wl.get("offsets")
    offsets = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
    n_tot = n_exposures(wl)
    evals = n_evals(wl)

    # device-resident inputs
    dp = {k: torch.as_tensor(v, device=dev) for k, v in p.items()}
    d_t = torch.as_tensor(t, device=dev)
    d_exp = torch.as_tensor(exptime, device=dev)
    d_ns = torch.as_tensor(ns, device=dev)
    d_off = None if offsets is None else torch.as_tensor(offsets, device=dev)
    out32 = torch.empty(n_tot, dtype=torch.float64, device=dev)
    out64 = torch.empty(n_tot, dtype=torch.float64, device=dev)

    def step(out, prec):
        ctx.lightcurve(dp, d_t, out, d_exp, nsuper=d_ns, offsets=d_off, precision=prec,
                       stream=stream)

    if args.profile_case:
        # A short run for a profiler's launch list or capture: the configuration
        # pinned by --config, then warm-up + K FP32C steps through the same call
        # (graph replays), and nothing else: no FP64 path, no timing, no autotune.
        if args.config:
            pin_config(ctx, args.config)
        for _ in range(args.warmup + args.steps):
            step(out32, binding.GL_FP32C)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": args.workload, "config": args.config,
                          "steps": args.warmup + args.steps, "status": ctx.sync(stream)}))
        ctx.close()
        return

    # accuracy of the timed path against the FP64 GPU path
    step(out64, binding.GL_FP64)
    step(out32, binding.GL_FP32C)
    torch.cuda.synchronize(dev)
    status = ctx.sync(stream)
    max_dflux = float((out32 - out64).abs().max().item())
    in_transit = int((out64 < 1.0).sum().item())

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    step_stats = {}

    def timed(prec, out, k, profile):
        """k steps, L2 flushed before each, CUDA events on the launch stream around
        each step (the flush is outside them).  With profile=True the library also
        times each kernel with CUDA events recorded inside the replayed step graph
        (event-record nodes at the kernel boundaries, on the same stream)."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        l0 = ctx.launches()
        ctx.profile(binding.PROFILE_GRAPH if profile else False)
        if profile:
            step(out, prec)   # capture of the profiled graph, untimed
            torch.cuda.synchronize(dev)
            ctx.profile(binding.PROFILE_GRAPH)   # reset the accumulated times
        gc_was = gc.isenabled()
        gc.disable()   # no collector pause between a step's events
        torch.cuda.nvtx.range_push(f"timed steps (precision {prec}, profile {profile})")
        try:
            for i in range(k):
                flush.zero_()
                evs[i][0].record(stream)
                step(out, prec)
                evs[i][1].record(stream)
            torch.cuda.synchronize(dev)
        finally:
            torch.cuda.nvtx.range_pop()
            if gc_was:
                gc.enable()
        per_step = [a.elapsed_time(b) for a, b in evs]
        step_stats[prec if not profile else -1] = per_step
        ms = sum(per_step)
        kern = {}
        if profile:
            for name, kind in (("window", binding.GL_KERNEL_WINDOW),
                               ("exposures", binding.GL_KERNEL_CURVE),
                               ("quadrature", binding.GL_KERNEL_QUAD),
                               ("quadrature_kernel", binding.GL_KERNEL_ITEMS),
                               ("setup", binding.GL_KERNEL_SETUP),
                               ("step", binding.GL_KERNEL_STEP)):
                t_ms, n = ctx.profile_read(kind)
                kern[name] = t_ms / n if n else None
            kern["timed_steps"] = k
            ctx.profile(False)
        return ms, ctx.launches() - l0, kern

    # autotuner: kernel shape and FP32 quadrature order for this batch (untimed)
    if args.config:
        pin_config(ctx, args.config)
        tune = tune64 = {"pinned": args.config}
    else:
        tune = ctx.autotune(dp, d_t, out32, d_exp, nsuper=d_ns, offsets=d_off,
                            precision=binding.GL_FP32C, stream=stream)
        tune64 = ctx.autotune(dp, d_t, out64, d_exp, nsuper=d_ns, offsets=d_off,
                              precision=binding.GL_FP64, stream=stream)
    step(out32, binding.GL_FP32C)
    torch.cuda.synchronize(dev)
    max_dflux = float((out32 - out64).abs().max().item())

    # workload counts of one FP32C step (instrumented kernel instance, untimed)
    ctx.counts(True)
    step(out32, binding.GL_FP32C)
    counts = ctx.counts_read()
    ctx.counts(False)

    # The clock sampler starts (and settles) before the warm-up steps.  Its second
    # of start-up leaves the GPU idle, and a GPU that has idled that long ran this
    # short, latency-bound step up to twice as slow for a while afterwards (with or
    # without the sampler; the sampled SM clock stayed at its maximum), so 0.3 s
    # of L2-flush writes bring it back to its working state before the warm-up.
    with ClockSampler(local) as clk:
        t_busy = time.perf_counter()
        while time.perf_counter() - t_busy < 0.3:
            flush.zero_()
            torch.cuda.synchronize(dev)
        for _ in range(args.warmup):
            step(out32, binding.GL_FP32C)
            step(out64, binding.GL_FP64)
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        ms32, launches, _ = timed(binding.GL_FP32C, out32, args.steps, profile=False)
    barrier(world)
    ms32 = allreduce_max(ms32, world)
    clocks = clk.summary()
    k_prof = max(3, min(args.steps, 20))
    _, _, kern32 = timed(binding.GL_FP32C, out32, k_prof, profile=True)
    k64 = max(3, min(args.steps, 20))
    ms64, _, _ = timed(binding.GL_FP64, out64, k64, profile=False)
    ms64 = allreduce_max(ms64, world)
    _, _, kern64 = timed(binding.GL_FP64, out64, 3, profile=True)

    value = aggregate_value(world, evals, args.steps, ms32)
    fp64_value = aggregate_value(world, evals, k64, ms64)
    # end to end: pinned host inputs and output through the same public call
    hp = {k: torch.as_tensor(v).pin_memory() for k, v in p.items()}
    h_t = torch.as_tensor(t).pin_memory()
    h_exp = torch.as_tensor(exptime).pin_memory()
    h_ns = torch.as_tensor(ns).pin_memory()
    h_off = None if offsets is None else torch.as_tensor(offsets).pin_memory()
    h_out = torch.empty(n_tot, dtype=torch.float64).pin_memory()
    for _ in range(2):
        ctx.lightcurve(hp, h_t, h_out, h_exp, nsuper=h_ns, offsets=h_off,
                       precision=binding.GL_FP32C, stream=stream)
    barrier(world)
    k_e2e = max(3, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        ctx.lightcurve(hp, h_t, h_out, h_exp, nsuper=h_ns, offsets=h_off,
                       precision=binding.GL_FP32C, stream=stream)
    e2e_s = allreduce_max(time.perf_counter() - t0, world)
    h2d = sum(v.numel() * v.element_size() for v in hp.values()) + h_t.numel() * 8 + \
        h_exp.numel() * 8 + h_ns.numel() * 4 + (0 if h_off is None else h_off.numel() * 8)
    d2h = h_out.numel() * 8

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    with ClockSampler(local) as clk_probe:
        fp32_peak, fp64_peak, mufu_peak, peak_src = measured_alu_peaks(
            local, peaks.get("sm_max_mhz", 2032.0))
    probe_clocks = clk_probe.summary()
    if rank != 0:
        return
    step_s = ms32 / args.steps * 1e-3
    on_disk = counts["full"] + counts["partial"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_sets, gpu_out=out32.cpu().numpy())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps,
        "ms_per_step_median": statistics.median(step_stats[binding.GL_FP32C]),
        "ms_per_step_max": max(step_stats[binding.GL_FP32C]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "evals_per_step": evals,
                   "exposures_per_step": n_tot, "parameter_sets": n_sets,
                   "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MB write)",
                   "graphs": "step replayed as a CUDA graph"},
        "max_dflux_vs_fp64_gpu": max_dflux, "in_transit_exposures": in_transit,
        "max_dflux_vs_oracle": None if cpu is None else cpu["max_dflux_vs_oracle"],
        "in_transit_evals_per_s": world * on_disk / step_s,
        "in_window_evals_per_s": world * counts["items"] / step_s,
        "rates_note": "in_transit = sub-exposures whose planet overlaps the star (the "
                      "quadrature's items); in_window = sub-exposures of exposures inside "
                      "the exact transit window; value counts every evaluation",
        "alu_peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak,
                      "mufu_tops": mufu_peak, "source": peak_src, "clocks": probe_clocks},
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": ms64 / k64},
        "kernel_ms": {"fp32c": kern32, "fp64": kern64},
        "workload_counts": counts,
        "autotune": tune,
        "autotune_fp64": tune64,
        "roofline": roofline(counts, kern32, fp32_peak, fp64_peak,
                             peaks.get("hbm_gbs"), 8 * len(t) if offsets is None
                             else 8 * n_tot, args.workload, peak_src),
        "gpu_launches": launches,
        "status": status,
        "clocks": clocks,
        "e2e": {"value": world * evals * k_e2e / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
