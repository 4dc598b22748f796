#!/usr/bin/env python
"""Correlator benchmark on GB300.

Headline: correlator TOPS of the tcgen05 tensor path on the precision
workload (256 stations, 2 pols, 480 channels, 1024 samples per integration,
complex int8 samples, bit-exact INT32 visibilities), one kernel launch per
step, inputs resident in HBM. The same run also times the FP16 tensor path
and the FP32 CUDA-core path on the same samples, the production FP32
workload, the ragged batch and the gain adjoint, and reports the roofline
of the dominant kernel, clocks during the timed region, an end-to-end figure
with host buffers, and the FP64 CPU oracle on a bounded sample.

Correlator ops = 32 per baseline per sample (8 per complex multiply-add,
4 polarisation pairs), baselines S(S+1)/2 (Section 2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--split none|channels]

Under torchrun each rank correlates on its own GPU with no collective on the
data path. --split none (default): every rank runs the whole workload (weak
scaling); --split channels: the workload's channels are divided over the
ranks (strong scaling, the partition of Sections 2 and 7). Either way the
line reports the ops of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

S3, C3, T3 = 256, 480, 1024
METRIC = "correlator TOPS & % of roofline: FP32 vs INT8/FP16 tensor path, same GB300"
UNIT = "TOPS"
WORKLOAD = ("precision: 256 stations, 2 pols, 480 channels, 1024 samples per integration, "
            "complex int8 N(0,32^2) clipped to +-127, INT32 visibilities (bit-exact)")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "tc_pair_kernel_int8_precision.txt")
TC_SOURCES = [os.path.join(ROOT, "paper_1702_00844_gb300", "csrc", f)
              for f in ("corr_tc.cu", "ptx.cuh", "corr_tc_internal.h")]


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["precision", "precision-f16", "production", "production-tf32",
                                           "ragged"],
                    default="precision",
                    help="precision: int8 tensor path at 256 stations (the headline); "
                         "precision-f16: the same samples on the f16 tensor path; "
                         "production: the 64-station FP32 workload on the FP32 path; "
                         "production-tf32: the same on the tensor cores (tf32 value + remainder split); "
                         "ragged: the 32-sub-array f16 batch alone")
    ap.add_argument("--ragged-scale", type=float, default=1.0,
                    help="channels of each ragged sub-array scaled by this factor")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the FP16/FP32/batch/adjoint side measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--split", choices=["none", "channels"], default="none",
                    help="none: every rank runs the whole workload (weak scaling); channels: the "
                         "workload's channels are divided over the ranks (strong scaling)")
    return ap.parse_args(argv)


def ops_of(S, T, units):
    return 32.0 * S * (S + 1) / 2 * T * units


# ------------------------------------------------------------- rank logic
def rank_channels(split: str, n_channels: int, world: int, rank: int):
    """[lo, hi) of the workload's channels this rank correlates: all of them
    for split "none" (weak scaling), a contiguous share for "channels"
    (strong scaling; the first n_channels % world ranks take one more)."""
    from paper_1702_00844_gb300.shard import channel_range
    if split == "channels":
        return channel_range(n_channels, world, rank)
    return 0, n_channels


def job_throughput(ops_rank: float, ms_rank: float, steps: int, device=None):
    """Job-wide correlator TOPS and ms per step: the ops of all ranks over
    the slowest rank's time for `steps` steps (ms_rank is that rank's total
    over the steps). Returns (TOPS, ms per step, total ops per step)."""
    from paper_1702_00844_gb300.shard import max_over_ranks, sum_over_ranks
    ops = sum_over_ranks(ops_rank, device=device)
    ms = max_over_ranks(ms_rank, device=device)
    return ops * steps / (ms * 1e-3) / 1e12, ms / steps, ops


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- profile data
def tc_source_hash() -> str:
    h = hashlib.sha256()
    for f in TC_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None if the summary is absent or the kernel changed since."""
    try:
        kv = {}
        for ln in open(PROFILE_SUMMARY):
            if ":" in ln:
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != tc_source_hash():
            return None
        return float(kv["dram_bytes_per_launch_full"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------- oracle
def oracle_sample(n_channels: int, passes: int = 1):
    """Times the FP64 oracle on the first n_channels channels of the precision
    workload (host data), `passes` times over. Returns (TOPS, seconds, threads)."""
    import oracle
    import synth
    d = synth.precision(channels=list(range(n_channels)))
    t0 = time.perf_counter()
    for _ in range(passes):
        oracle.correlate(d["x"], "ci8")
    dt = time.perf_counter() - t0
    return ops_of(S3, T3, n_channels) * passes / dt / 1e12, dt, oracle.threads()


def cpu_baseline(target_s: float = 12.0):
    """About target_s of oracle work: a channel sample sized from a first
    timing on one channel per thread, up to all 480 channels, repeated when
    the whole workload takes less than half of target_s."""
    import oracle
    nthr = max(1, oracle.threads())
    tops, dt, _ = oracle_sample(nthr)
    per_channel = max(dt, 1e-3) / nthr
    n = int(min(C3, max(nthr, target_s / per_channel)))
    n = max(nthr, (n // nthr) * nthr) if n < C3 else C3
    passes = max(1, min(4, int(round(target_s / (per_channel * n)))))
    tops, dt, _ = oracle_sample(n, passes)
    what = f"{n} of 480 channels" + (f", {passes} passes" if passes > 1 else "")
    return {"value": tops, "unit": UNIT, "cores": nthr, "kind": "oracle",
            "sample": f"{what} of the precision workload (all 32896 baselines x 4 pol pairs x "
                      f"1024 samples each), FP64, {dt:.1f} s"}


def _rel_frob(got, ref):
    """Largest per-unit relative Frobenius error."""
    import numpy as np
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    den = np.linalg.norm(r, axis=1)
    return float((np.linalg.norm(g - r, axis=1) / np.where(den == 0, 1.0, den)).max())


def _coef_err(got, ref, S):
    """max |V - V_ref| / sqrt(V_ref_aa V_ref_bb): the error in the
    normalised correlation coefficient."""
    import numpy as np
    auto = np.array([s * (s + 1) // 2 + s for s in range(S)])
    a = np.stack([ref[:, auto, 0, 0].real, ref[:, auto, 1, 1].real], axis=-1)
    s2 = np.concatenate([np.full(j + 1, j) for j in range(S)])
    s1 = np.concatenate([np.arange(j + 1) for j in range(S)])
    na = np.sqrt(np.maximum(a[:, s1, :], 1e-300))
    nb = np.sqrt(np.maximum(a[:, s2, :], 1e-300))
    return float((np.abs(got - ref) / (na[:, :, :, None] * nb[:, :, None, :])).max())


def oracle_errors(torch):
    """Errors against the FP64 oracle, stated per workload, on sampled
    channels of host-generated data: the precision workload on the int8
    (mismatched elements), f16 and FP32 paths; the production FP32 workload;
    sub-arrays of the ragged batch in one batched f16 call; and the
    differentiation workload's loss and gradients."""
    import numpy as np

    import oracle
    import synth
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    res = {}

    def vis(t):
        a = t.detach().cpu().numpy()
        if a.dtype == np.int32:
            return a.astype(np.int64)
        return a.astype(np.complex128).reshape((-1,) + a.shape[-3:])

    # precision: channels 0, 137, 479
    picks = [0, 137, 479]
    x8 = synth.precision(channels=picks)["x"]
    ref = oracle.correlate(x8, "ci8")
    p8 = Plan(S3, len(picks), T3, dtype="ci8", path="tensor")
    got8 = vis(p8.correlate(torch.from_numpy(x8).cuda())).reshape(ref.shape + (2,))
    mism = int((got8[..., 0] != ref.real.astype(np.int64)).sum() + (got8[..., 1] != ref.imag.astype(np.int64)).sum())
    res["precision_int8"] = {"channels": picks, "mismatched_elements": mism, "elements": int(ref.size * 2)}
    p16 = Plan(S3, len(picks), T3, dtype="cf16", path="tensor")
    got16 = vis(p16.correlate(torch.from_numpy(synth.int8_as_cf16(x8)).cuda()))
    res["precision_f16"] = {"channels": picks, "rel_frobenius_max": _rel_frob(got16, ref),
                            "coef_error_max": _coef_err(got16, ref, S3), "bound": "2e-3 relative"}
    xc = (x8[..., 0].astype(np.float32) + 1j * x8[..., 1].astype(np.float32)).astype(np.complex64)
    p32 = Plan(S3, len(picks), T3, dtype="cf32", path="fp32")
    got32 = vis(p32.correlate(torch.from_numpy(xc).cuda()))
    res["precision_fp32"] = {"channels": picks, "rel_frobenius_max": _rel_frob(got32, ref),
                             "coef_error_max": _coef_err(got32, ref, S3), "bound": "1e-5 relative"}
    del p8, p16, p32
    # production (one integration of 256 channels): channels 0, 100, 255
    xp = synth.production(n_integrations=1)["x"][0]
    pp = Plan(64, xp.shape[0], xp.shape[2], dtype="cf32", path="fp32")
    gotp = vis(pp.correlate(torch.from_numpy(xp).cuda()))
    cp = [0, 100, 255]
    refp = oracle.correlate(xp[cp])
    res["production_fp32"] = {"channels": cp, "rel_frobenius_max": _rel_frob(gotp[cp], refp),
                              "coef_error_max": _coef_err(gotp[cp], refp, 64), "bound": "1e-5 relative"}
    ptt = Plan(64, xp.shape[0], xp.shape[2], dtype="cf32", path="tensor")
    gott = vis(ptt.correlate(torch.from_numpy(xp).cuda()))
    res["production_tf32_split"] = {"channels": cp, "rel_frobenius_max": _rel_frob(gott[cp], refp),
                                    "coef_error_max": _coef_err(gott[cp], refp, 64), "bound": "1e-5 relative"}
    del pp, ptt, xp
    # ragged batch: three sub-arrays (the smallest, a long integration and a
    # partial last block) in one batched f16 call; two channels each
    shapes = synth.batching_shapes()
    pick = [min(range(len(shapes)), key=lambda k: shapes[k][0] * shapes[k][1] * shapes[k][2]),
            next(k for k, s in enumerate(shapes) if s[2] >= 3000 and s[0] < 120),
            next(k for k, s in enumerate(shapes) if s[0] % 64 and 120 < s[0] < 200)]
    subs, outs, sh = [], [], []
    for k in pick:
        S, C, T = shapes[k]
        subs.append(synth.batching_subarray_device(S, C, T, k, "cuda"))
        outs.append(torch.empty((C, S * (S + 1) // 2, 2, 2), dtype=torch.complex64, device="cuda"))
        sh.append((S, C, T))
    pb = Plan(1, 1, 1, dtype="cf16", path="tensor")
    pb.correlate_batched(list(zip(subs, outs)), sh)
    torch.cuda.synchronize()
    worst_f, worst_c = 0.0, 0.0
    for (S, C, T), xs, o in zip(sh, subs, outs):
        for c in (0, C - 1):
            xh = xs[c].cpu().numpy()
            r = oracle.correlate(xh[None], "cf16")
            g = o[c].cpu().numpy().astype(np.complex128)[None]
            worst_f = max(worst_f, _rel_frob(g, r))
            worst_c = max(worst_c, _coef_err(g, r, S))
    res["ragged_f16"] = {"sub_arrays": [list(s) for s in sh], "channels": "first and last of each",
                         "rel_frobenius_max": worst_f, "coef_error_max": worst_c, "bound": "2e-3 relative"}
    del subs, outs, pb
    # differentiation: loss and gradients on channels 0, 31, 63
    d = synth.differentiation()
    pg = Plan(d["S"], d["C"], d["T"], dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = (torch.from_numpy(d[k]).cuda() for k in ("x", "g", "M"))
    R = pg.correlate(xd)
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    gg, gx = pg.gain_backward(xd, gd, Md, R=R, loss=loss)
    torch.cuda.synchronize()
    gg, gx = gg.cpu().numpy(), gx.cpu().numpy()
    Lref, _ = oracle.gain_loss(oracle.correlate(d["x"]), d["g"], d["M"])
    eg, ex = 0.0, 0.0
    for c in (0, 31, 63):
        Rc = oracle.correlate(d["x"][c][None])
        gr = oracle.gain_grad(Rc, d["g"][c][None], d["M"][c][None])
        xr = oracle.input_grad(d["x"][c][None], Rc, d["g"][c][None], d["M"][c][None])
        eg = max(eg, float(np.abs(gg[c][None] - gr).max() / np.abs(gr).max()))
        ex = max(ex, float(np.abs(gx[c][None] - xr).max() / np.abs(xr).max()))
    res["differentiation_fp32"] = {"channels": [0, 31, 63], "loss_rel": abs(float(loss) - Lref) / Lref,
                                   "grad_gain_max_rel": eg, "grad_samples_max_rel": ex,
                                   "bound": "1e-4 (gradients)"}
    # the same with the forward correlation on the tensor cores (tf32 split)
    pt = Plan(d["S"], d["C"], d["T"], dtype="cf32", path="tensor", flags=FLAG_GAINS)
    Rt = pt.correlate(xd)
    gg, gx = pt.gain_backward(xd, gd, Md, R=Rt, loss=loss)
    torch.cuda.synchronize()
    gg, gx = gg.cpu().numpy(), gx.cpu().numpy()
    eg, ex = 0.0, 0.0
    for c in (0, 31, 63):
        Rc = oracle.correlate(d["x"][c][None])
        gr = oracle.gain_grad(Rc, d["g"][c][None], d["M"][c][None])
        xr = oracle.input_grad(d["x"][c][None], Rc, d["g"][c][None], d["M"][c][None])
        eg = max(eg, float(np.abs(gg[c][None] - gr).max() / np.abs(gr).max()))
        ex = max(ex, float(np.abs(gx[c][None] - xr).max() / np.abs(xr).max()))
    res["differentiation_tf32_forward"] = {"channels": [0, 31, 63], "loss_rel": abs(float(loss) - Lref) / Lref,
                                           "grad_gain_max_rel": eg, "grad_samples_max_rel": ex,
                                           "bound": "1e-4 (gradients)"}
    del pg, pt
    torch.cuda.empty_cache()
    return res


def cpu_fp32_correlator(target_s: float = 6.0):
    """The multithreaded FP32 CPU correlator (Section 4.1's design) on the
    precision workload's samples as complex64: channels sized from a first
    timing on one channel per thread for about target_s, up to all 480."""
    import numpy as np

    import cpu_baseline
    import synth
    nthr = max(1, cpu_baseline.threads())

    def samples(n):   # the first n channels, (n, S, T, 2) complex64
        x = synth.precision(channels=list(range(n)))["x"]
        return (x[..., 0].astype(np.float32) + 1j * x[..., 1].astype(np.float32)).astype(np.complex64)

    xc = samples(nthr)
    cpu_baseline.correlate(xc)                       # warm-up
    t0 = time.perf_counter()
    cpu_baseline.correlate(xc)
    per_channel = max(time.perf_counter() - t0, 1e-4) / nthr
    n = int(min(C3, max(nthr, target_s / per_channel)))
    xc = samples(n)
    t0 = time.perf_counter()
    cpu_baseline.correlate(xc)
    dt = time.perf_counter() - t0
    return {"value": ops_of(S3, T3, n) / dt / 1e12, "unit": UNIT, "cores": nthr,
            "kind": "multithreaded FP32 CPU correlator (2x2 station tiles, time loop vectorised, "
                    "Section 4.1 design)",
            "sample": f"{n} of 480 channels of the precision workload as complex64, {dt:.1f} s"}


# ---------------------------------------------------------------- reference
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    nthr = oracle.threads()
    n = max(1, nthr)
    oracle_sample(n)  # warm-up: page in the oracle and the sample
    times = []
    for _ in range(args.steps):
        tops, dt, _ = oracle_sample(n)
        times.append(dt)
    total = sum(times)
    value = ops_of(S3, T3, n) * len(times) / total / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_channels_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                         "sample": f"{n} channels of the precision workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours
def time_launches(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps  # ms


def ragged_shapes(scale=1.0):
    """The ragged-batch workload's 32 (stations, channels, samples) shapes,
    channels scaled by ``scale`` (at least one per sub-array)."""
    import synth
    return [(S, max(1, int(round(C * scale))), T) for S, C, T in synth.batching_shapes()]


def ragged_batch(torch, scale=1.0, steps=5, warmup=2):
    """The ragged batch (32 sub-arrays of 16-576 stations and 256-4096
    samples, complex f16) correlated by one corr_correlate_batched call,
    captured in a CUDA graph and replayed: ms per replay, TOPS, the clocks
    during the replays and the tile configuration the batch tuner chose.
    A replay of the full batch lasts about 45 ms, so the replays are a
    sustained load: the fraction is also given against the sustained bf16
    peak."""
    import synth
    from paper_1702_00844_gb300 import Plan
    shapes = ragged_shapes(scale)
    xs, outs = [], []
    for k, (S, C, T) in enumerate(shapes):
        xs.append(synth.batching_subarray_device(S, C, T, k, "cuda"))
        outs.append(torch.empty((C, S * (S + 1) // 2, 2, 2), dtype=torch.complex64, device="cuda"))
    pb = Plan(1, 1, 1, dtype="cf16", path="tensor")
    pairs = list(zip(xs, outs))
    pb.correlate_batched(pairs, shapes)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pb.correlate_batched(pairs, shapes, stream=s)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = time_launches(g.replay, steps, warmup, torch.cuda.current_stream())
    opsb = sum(ops_of(S, T, C) for S, C, T in shapes)
    peaks, _ = measured_peaks()
    res = {"ms": ms, "TOPS": opsb / ms / 1e9, "ops": opsb, "steps": steps, "clocks": clk.summary(),
           "frac_sustained": opsb / ms / 1e9 / float(peaks.get("bf16_tflops_sustained", 1700.0)),
           "input_GB": sum(x.numel() * 2 for x in xs) / 1e9,
           "channel_scale": scale,
           "variant": pb.batch_tile_variant(),
           "tuned": [["/".join(map(str, c)), round(t, 3)] for c, t in pb.tune_results(batch=True)]}
    pb.check_error()
    del xs, outs, pairs, g, pb
    return res


def run_ragged(args):
    """--workload ragged: the ragged batch alone on one GPU (rank 0), one
    JSON line; --ragged-scale shrinks its channels for profiler captures."""
    import torch
    if int(os.environ.get("RANK", "0")) != 0:
        return
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    r = ragged_batch(torch, args.ragged_scale, max(1, args.steps), max(3, args.warmup))
    line = {"metric": METRIC, "value": r["TOPS"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic (seeded device Philox)",
            "config": {"workload": "ragged batch: 32 sub-arrays, 16-576 stations, 256-4096 samples, "
                                   f"channels x {args.ragged_scale:g}, complex f16, one batched call "
                                   "replayed as a CUDA graph",
                       "l2": f"inputs {r['input_GB']:.2f} GB"},
            "clocks": r["clocks"],
            "roofline": {"bound": "tensor", "achieved": r["TOPS"], "peak": peak, "unit": "TFLOP/s",
                         "frac": r["TOPS"] / peak, "traffic": None,
                         "peak_source": f"{peak_src} bf16 dense burst"},
            "batch": r}
    print(json.dumps(line), flush=True)


def secondary(x8, torch):
    """Side measurements on one GPU: FP16 and FP32 paths on the same samples,
    the production FP32 workload, the ragged batch and the gain adjoint."""
    import synth
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    res = {}
    st = torch.cuda.current_stream()
    ops3 = ops_of(S3, T3, C3)
    x16 = x8.to(torch.float16)
    p16 = Plan(S3, C3, T3, dtype="cf16", path="tensor")
    o16 = p16.empty_out()
    ms = time_launches(lambda: p16.correlate(x16, o16), 10, 3, st)
    res["tensor_fp16_precision"] = {"ms": ms, "TOPS": ops3 / ms / 1e9}
    # the same for about a second of back-to-back steps: a sustained load
    # like the ragged batch's replays (the power limit lowers the clocks)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = time_launches(lambda: p16.correlate(x16, o16), 2000, 3, st)
    peaks, _ = measured_peaks()
    res["tensor_fp16_precision_sustained"] = {
        "ms": ms, "TOPS": ops3 / ms / 1e9, "steps": 2000, "clocks": clk.summary(),
        "frac_sustained": ops3 / ms / 1e9 / float(peaks.get("bf16_tflops_sustained", 1700.0))}
    # the same shape on complex N(0,1) f16 samples, the ragged batch's value
    # distribution (full mantissas: the tensor cores draw more power on them
    # than on small integers), again for about a second
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 6)
    xg = torch.randn(x16.shape, generator=gen, device="cuda", dtype=torch.float32).to(torch.float16)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = time_launches(lambda: p16.correlate(xg, o16), 2000, 3, st)
    res["tensor_fp16_gaussian_sustained"] = {
        "ms": ms, "TOPS": ops3 / ms / 1e9, "steps": 2000, "clocks": clk.summary(),
        "frac_sustained": ops3 / ms / 1e9 / float(peaks.get("bf16_tflops_sustained", 1700.0)),
        "data": "256 st. x 480 ch. x 1024, complex f16 N(0,1)"}
    del xg
    del o16, x16, p16
    xc = torch.view_as_complex(x8.to(torch.float32).contiguous())
    p32 = Plan(S3, C3, T3, dtype="cf32", path="fp32")
    o32 = p32.empty_out()
    ms = time_launches(lambda: p32.correlate(xc, o32), 3, 1, st)
    res["fp32_cuda_core_precision"] = {"ms": ms, "TOPS": ops3 / ms / 1e9}
    # the same FP32 samples on the tensor cores (tf32 value + remainder
    # split, three products per term, FP32 accumulation)
    pt = Plan(S3, C3, T3, dtype="cf32", path="tensor")
    ms = time_launches(lambda: pt.correlate(xc, o32), 3, 1, st)
    res["tensor_tf32_split_fp32_precision"] = {"ms": ms, "TOPS": ops3 / ms / 1e9}
    del o32, xc, p32, pt
    torch.cuda.empty_cache()
    # production FP32 workload: 64 stations, 256 channels, 768 samples, 10 integrations
    S2, C2, T2, I2 = 64, 256, 768, 10
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 2)
    x2 = torch.randn((I2, C2, S2, T2, 2), dtype=torch.complex64, device="cuda", generator=gen)
    p2 = Plan(S2, C2, T2, I2, dtype="cf32", path="fp32")
    o2 = p2.empty_out()
    ms = time_launches(lambda: p2.correlate(x2, o2), 5, 2, st)
    res["fp32_cuda_core_production"] = {"ms": ms, "TOPS": ops_of(S2, T2, C2 * I2) / ms / 1e9}
    pt2 = Plan(S2, C2, T2, I2, dtype="cf32", path="tensor")
    ms = time_launches(lambda: pt2.correlate(x2, o2), 5, 2, st)
    res["tensor_tf32_split_fp32_production"] = {"ms": ms, "TOPS": ops_of(S2, T2, C2 * I2) / ms / 1e9}
    del x2, o2, p2, pt2
    torch.cuda.empty_cache()
    # ragged batch: 32 sub-arrays, one persistent launch (graph replay)
    res["tensor_fp16_ragged_batch"] = ragged_batch(torch, steps=20)
    torch.cuda.empty_cache()
    # gain adjoint: 64 stations, 64 channels, 1024 samples
    d = synth.differentiation()
    pg = Plan(d["S"], d["C"], d["T"], dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd = torch.from_numpy(d["x"]).cuda()
    gd = torch.from_numpy(d["g"]).cuda()
    Md = torch.from_numpy(d["M"]).cuda()
    R = pg.correlate(xd)
    gg = torch.empty_like(gd)
    gx = torch.empty_like(xd)

    def step():
        pg.correlate(xd, R)
        pg.gain_backward(xd, gd, Md, R=R)

    ms = time_launches(step, 10, 3, st)
    res["gain_forward_backward_differentiation"] = {"ms": ms, "forward": "FP32 CUDA cores"}
    # the same step with the forward correlation on the tensor cores (tf32
    # value + remainder split)
    pt = Plan(d["S"], d["C"], d["T"], dtype="cf32", path="tensor", flags=FLAG_GAINS)

    def step_t():
        pt.correlate(xd, R)
        pt.gain_backward(xd, gd, Md, R=R)

    ms = time_launches(step_t, 10, 3, st)
    res["gain_forward_backward_differentiation_tf32_forward"] = {"ms": ms, "forward": "tensor cores, tf32 split"}
    del pg, pt, xd, gd, Md, R, gg, gx
    torch.cuda.empty_cache()
    # one polarisation: the int8 samples read as 512 stations of one pol (the
    # same bytes, and the same products per channel as 256 two-pol stations)
    p1 = Plan(2 * S3, C3, T3, dtype="ci8", path="tensor", n_pols=1)
    x1 = x8.view(C3, 2 * S3, T3, 1, 2)
    o1 = p1.empty_out()
    ms = time_launches(lambda: p1.correlate(x1, o1), 10, 3, st)
    ops1 = 8.0 * (2 * S3) * (2 * S3 + 1) / 2 * T3 * C3
    res["tensor_int8_single_pol_512_stations"] = {"ms": ms, "TOPS": ops1 / ms / 1e9,
                                                  "variant": p1.tile_variant()}
    del p1, o1
    torch.cuda.empty_cache()
    # the first 120 channels' bytes read as 30 channels of 1024 stations (the
    # same correlator ops as the 256-station workload): the tile triangle's
    # diagonal blocks weigh less (524800 of the 589824 station pairs the pair
    # tiles compute are needed, against 32896 of 49152 at 256 stations)
    Sw, Cw = 4 * S3, C3 // 16
    pw = Plan(Sw, Cw, T3, dtype="ci8", path="tensor")
    xw = x8[: Cw * Sw // S3].view(Cw, Sw, T3, 2, 2)
    ow = pw.empty_out()
    ms = time_launches(lambda: pw.correlate(xw, ow), 10, 3, st)
    opsw = ops_of(Sw, T3, Cw)
    pk, _ = measured_peaks()
    res["tensor_int8_1024_stations"] = {
        "ms": ms, "TOPS": opsw / ms / 1e9,
        "frac": opsw / ms / 1e9 / float(pk.get("bf16_tflops", 1893.4)),
        "useful_fraction": (Sw * (Sw + 1) / 2) / (((Sw // 64) // 2) * ((Sw // 64) // 2 + 1) / 2 * 4 * 4096),
        "variant": pw.tile_variant()}
    del pw, ow
    torch.cuda.empty_cache()
    # sample layouts (corr_reorder) on the int8 precision samples: the
    # time-major layout of Section 4.4 and the per-station streams before the
    # corner turn of Section 7, each into the correlator's layout. HBM-bound:
    # every byte read once and written once.
    from paper_1702_00844_gb300 import reorder
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    nbytes = x8.numel() * x8.element_size()
    x6 = x8.view(1, C3, S3, T3, 2, 2)
    for L in ("cts", "sct"):
        other = reorder(x6, S3, C3, T3, 1, "ci8", "cst", L)
        back = torch.empty_like(x6)
        ms = time_launches(lambda: reorder(other, S3, C3, T3, 1, "ci8", L, "cst", out=back), 10, 3, st)
        gbs = 2 * nbytes / (ms * 1e-3) / 1e9
        res[f"reorder_{L}_to_cst_int8"] = {"ms": ms, "GB/s": gbs, "hbm_frac": gbs / hbm,
                                           "peak": f"{src} hbm_gbs {hbm:.0f}"}
        del other, back
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_1702_00844_gb300 import Plan
    from paper_1702_00844_gb300.shard import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()

    wl = args.workload
    prod = wl in ("production", "production-tf32")
    # this rank's channels of the workload (all of them unless --split channels)
    c_lo, c_hi = rank_channels(args.split, 256 if prod else C3, world, rank)
    # weak scaling: a workload of its own per rank; strong: this rank's
    # share of the one workload
    split = args.split == "channels"
    x8 = synth.precision_device(c_hi - c_lo if not prod else C3, S3, T3, "cuda",
                                rank=0 if split else rank, first_channel=c_lo if split else 0)
    if prod:
        S, C, T, I = 64, c_hi - c_lo, 768, 10
        gen = torch.Generator(device="cuda")
        gen.manual_seed(synth.BASE_SEED + 2 + 7919 * rank)
        x = torch.randn((I, C, S, T, 2), dtype=torch.complex64, device="cuda", generator=gen)
        tf32 = wl == "production-tf32"
        plan = Plan(S, C, T, I, dtype="cf32", path="tensor" if tf32 else "fp32")
        units, dtype_label = C * I, "f32"
        workload = ("production: 64 stations, 2 pols, 256 channels, 768 samples, 10 integrations, "
                    "complex64 N(0,1), " + ("tensor cores, tf32 value + remainder split" if tf32
                                            else "FP32 CUDA-core path"))
    else:
        S, C, T, I = S3, c_hi - c_lo, T3, 1
        if wl == "precision-f16":
            x = x8.to(torch.float16)
            plan = Plan(S, C, T, dtype="cf16", path="tensor")
            dtype_label = "f16"
            workload = WORKLOAD.replace("INT32 visibilities (bit-exact)",
                                        "cast to f16, FP32 accumulation")
        else:
            x = x8
            plan = Plan(S, C, T, dtype="ci8", path="tensor")
            dtype_label = "s8"
            workload = WORKLOAD
        units = C
    out = plan.empty_out()
    stream = torch.cuda.current_stream()

    def step():
        plan.correlate(x, out)

    for _ in range(max(3, args.warmup)):
        step()
    # one pair of events per timed step around the plan's main kernel launch
    # (corr_set_kernel_events), for the roofline's per-launch duration
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        time.sleep(0.3)
        # the timed steps: nothing between the launches (an event between the
        # int8 path's checked launch and its redo launch would keep the redo
        # launch from being scheduled ahead as a programmatic dependent)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        # the same steps again with a pair of events around each step's main
        # kernel launch (corr_set_kernel_events): the roofline's per-launch
        # duration of the dominant kernel
        for a, b in kev:
            plan.set_kernel_events(a, b)
            step()
        torch.cuda.synchronize()
    plan.set_kernel_events()
    kernel_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in kev) / len(kev), device="cuda")
    ops = ops_of(S, T, units)
    value, ms_step, ops_job = job_throughput(ops, e0.elapsed_time(e1), args.steps, device="cuda")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    plan.check_error()

    # end to end through the public API with host buffers: corr_correlate_host
    # streams the step's samples from page-locked memory in chunks, with the
    # copies overlapping the kernels, and copies the visibilities back.
    from paper_1702_00844_gb300 import FLAG_HOST_IO
    plan_io = Plan(S, C, T, I, dtype=plan.dtype, path="fp32" if wl == "production" else "tensor",
                   flags=FLAG_HOST_IO)
    xh = x.cpu().pin_memory()
    oh = plan_io.empty_out("cpu").pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    e2e_ms = time_launches(lambda: plan_io.correlate_host(xh, oh), e2e_steps, 1, stream)
    plan_io.check_error()
    e2e_val, e2e_ms, _ = job_throughput(ops, e2e_ms, 1, device="cuda")
    # the host link's own bound for this step (Section 3.6's perf_max with
    # the link as the bandwidth): the same bytes copied both ways at once,
    # H2D and D2H on two streams, no kernel
    xd_, od_ = torch.empty_like(xh, device="cuda"), torch.empty_like(oh, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def copies():
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        with torch.cuda.stream(s_in):
            xd_.copy_(xh, non_blocking=True)
        with torch.cuda.stream(s_out):
            oh.copy_(od_, non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    link_ms = time_launches(copies, e2e_steps, 1, stream)
    link_ms = max_over_ranks(link_ms, device="cuda")
    e2e = {"value": e2e_val, "unit": UNIT,
           "h2d_bytes_per_step": xh.numel() * xh.element_size(),
           "d2h_bytes_per_step": oh.numel() * oh.element_size(), "ms_per_step": e2e_ms,
           "api": "corr_correlate_host (chunked, copies overlapped with kernels)",
           "link_only_ms": link_ms,
           "link_bound_TOPS": ops / (link_ms * 1e-3) / 1e12,
           "frac_of_link_bound": link_ms / e2e_ms}
    del xh, oh, plan_io, xd_, od_

    peaks, peak_src = measured_peaks()
    in_bps = {"s8": 4, "f16": 8, "f32": 16}[dtype_label]
    alg_bytes = units * (S * T * in_bps + S * (S + 1) // 2 * 32)
    # the dominant kernel's own launches (events around the main launch of
    # each step), as the roofline asks; ms_per_step also holds the int8 path's
    # redo launch (empty on this data)
    achieved = ops / (kernel_ms * 1e-3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if wl == "production-tf32":
        # tf32 dense (the measured bf16 rate x the nominal tf32 : bf16 ratio
        # 1.1 : 2.25), divided by the three tf32 products per correlator term
        peak = float(peaks.get("bf16_tflops", 1900.0)) * 1.1 / 2.25 / 3
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "tf32_correlate_kernel",
                "peak_source": f"{peak_src} bf16 dense burst x 1.1/2.25 (tf32) / 3 (split products)"}
    elif wl == "production":
        # FP32 FMA pipe: this device's SMs x 128 FP32 lanes x 2 flops x maximum SM clock
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "fp32_correlate_kernel",
                "peak_source": f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flops x max SM clock"}
    else:
        peak = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic() if wl == "precision" else None,
                "kernel": (f"tc_pair_kernel<{dtype_label}> (CTA pairs)" if plan.tile_variant() == "pair"
                           else f"tc_correlate_kernel<{dtype_label}, {plan.tile_variant()}>"),
                "peak_source": f"{peak_src} bf16 dense burst (f16 dense runs at the bf16 rate)"}
    roof["algorithmic_bytes"] = alg_bytes
    roof["kernel_ms"] = kernel_ms
    roof["timing"] = ("CUDA events around the main kernel launch of each step of a second pass "
                      "over the timed steps inside the clock-sampled region "
                      "(corr_set_kernel_events), averaged")
    roof["hbm_bound_TOPS"] = ops / (alg_bytes / (hbm * 1e9)) / 1e12

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong" if args.split == "channels" else "weak",
            "vs_baseline": None,
            "dtype": dtype_label,
            "data": "synthetic (seeded device Philox, same recipe as the workload)",
            "config": {"workload": workload, "stations": S, "pols": 2, "channels": C,
                       "integrations": I, "samples": T,
                       "path": {"s8": "tcgen05 kind::f16 with exact int8->f16 widening; exact "
                                      "FP32 sums by a station-power bound, chunked INT32 fold "
                                      "for tiles that fail it",
                                "f16": "tcgen05 kind::f16, FP32 accumulation in TMEM",
                                "f32": "FP32 CUDA cores, TMA-staged samples"}[dtype_label]
                       if wl != "production-tf32" else
                       "tcgen05 kind::tf32, value + remainder split (three products per term), FP32 "
                       "accumulation in TMEM in 256-sample chunks summed in FP32",
                       "l2": f"inputs {units * S * T * in_bps / 1e6:.0f} MB and outputs "
                             f"{units * S * (S + 1) // 2 * 32 / 1e6:.0f} MB; inputs exceed L2 "
                             "(129 MB): no flush",
                       "parallelism": (f"{world} GPU(s), the workload's channels split over them "
                                       f"(this rank: {c_hi - c_lo} of {c_hi - c_lo if args.split == 'none' else (256 if prod else C3)}), no collective"
                                       if args.split == "channels" else
                                       f"channels per GPU fixed, {world} GPU(s), no collective")},
            "clocks": clk.summary(), "e2e": e2e, "roofline": roof,
            "tile_config": (dict(plan.tile_config(),
                                 tuned=[["/".join(map(str, c)), round(t, 4)] for c, t in plan.tune_results()])
                            if not prod else None),
            # one tensor launch per step, plus the (usually empty) redo launch
            # of the int8 path when T exceeds one 512-sample chunk
            "gpu_launches": args.steps * (2 if dtype_label == "s8" and T > 512 else 1)}
    if rank == 0 and world == 1 and not args.no_secondary and wl == "precision":
        line["paths"] = secondary(x8, torch)
        fp32 = line["paths"]["fp32_cuda_core_precision"]["TOPS"]
        line["paths"]["tensor_int8_vs_fp32_same_samples"] = value / fp32
    if rank == 0 and world == 1 and not args.no_cpu and wl == "precision":
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_fp32_correlator"] = cpu_fp32_correlator()
        line["oracle_errors"] = oracle_errors(torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged":
        run_ragged(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
