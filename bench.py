#!/usr/bin/env python3
"""Benchmark of the FX correlator hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole hot path over one block of synthetic
LOFAR-shaped input already resident in HBM, through the C ABI:
fx_channelize_correct (FP64 phase table, then the fused PPF FIR + FFT + delay /
bandpass correction with the transposing write) and fx_correlate (X-stage).

Default workload (the headline): 64 stations x 2 pols, 244 subbands, complex
int16 noise (sigma 100) + 3 point sources with seeded delays (+-5 us) and
per-station bandpass ripple, 16-tap PPF to 64 channels, 3072 spectra per block
(1.00663 s of sky), FP32-accurate path: the X-stage runs on the tcgen05 tensor
cores with each FP32 operand split into hi + lo, hi hi' as TF32 MMAs and the
cross terms hi lo' + lo hi' as BF16 MMAs (FX_TF32_SPLIT).
The CUDA-core FFMA FP32 X-stage and the FP16 / BF16 / split-FP16 tensor-core
X-stages are timed on the same block, and the 8-bit precision workload (64
stations, 488 subbands, 256 channels, 768 spectra) is timed at its own shape;
every result's error is stated against the FP64 oracle on sampled subbands of
the benchmarked block itself. Inputs (24.7 GB raw) are far larger than L2.

value  = real-time factor = seconds of sky processed by all ranks / wall second
e2e    = the same through fx_process_host, with the raw block copied
         host->device from pinned memory and the visibilities copied back
         inside the timed region
Multi-GPU (torchrun): every rank processes its own 244-subband block (subbands
are independent; weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload. Besides that arm and the cpu_baseline leg, the oracle runs here only
to state the error of the benchmarked visibilities on sampled subbands.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FX real-time factor & X-stage TFLOP/s at 64 stations; TC FP16 vs FP32 at stated err"
UNIT = "x real time (sky s / wall s)"
FS = 195312.5

WORKLOADS = {
    "lofar16_fp32": dict(N=64, SB=244, C=64, S=3072, T=16, fmt=0, precision=4, sigma=100.0,
                         ntones=3, ripple=True, seed_index=1,
                         desc="LOFAR 16-bit, FP32-accurate path (hi/lo split X-stage on tensor cores: hi hi' in TF32, "
                              "hi lo' + lo hi' in BF16): "
                              "64 stations x 2 pols, 244 subbands, 16-tap PPF to 64 channels, "
                              "3072 spectra (1.00663 s) per block"),
    "lofar16_ffma": dict(N=64, SB=244, C=64, S=3072, T=16, fmt=0, precision=0, sigma=100.0,
                         ntones=3, ripple=True, seed_index=1,
                         desc="LOFAR 16-bit, FP32 path with the CUDA-core FFMA X-stage: 64 stations x 2 pols, "
                              "244 subbands, 16-tap PPF to 64 channels, 3072 spectra (1.00663 s) per block"),
    "lofar8_fp16": dict(N=64, SB=488, C=256, S=768, T=16, fmt=1, precision=1, sigma=20.0,
                        ntones=1, ripple=False, seed_index=2,
                        desc="LOFAR 8-bit, FP16 X-stage: 64 stations x 2 pols, 488 subbands, "
                             "16-tap PPF to 256 channels, 768 spectra (1.00663 s) per block"),
    "lofar16_fp32_small": dict(N=64, SB=8, C=64, S=3072, T=16, fmt=0, precision=4, sigma=100.0,
                               ntones=3, ripple=True, seed_index=1,
                               desc="LOFAR 16-bit FP32-accurate path on 8 subbands (profiling size, ~4 GB)"),
    "lofar16_ffma_small": dict(N=64, SB=8, C=64, S=3072, T=16, fmt=0, precision=0, sigma=100.0,
                               ntones=3, ripple=True, seed_index=1,
                               desc="LOFAR 16-bit FFMA FP32 path on 8 subbands (profiling size, ~4 GB)"),
    "lofar8_fp16_small": dict(N=64, SB=16, C=256, S=768, T=16, fmt=1, precision=1, sigma=20.0,
                              ntones=1, ripple=False, seed_index=2,
                              desc="LOFAR 8-bit FP16 X-stage on 16 subbands (profiling size, ~2.5 GB)"),
    "tiny_fp32": dict(N=8, SB=1, C=64, S=768, T=16, fmt=0, precision=4, sigma=100.0,
                      ntones=1, ripple=False, seed_index=0,
                      desc="8 stations x 2 pols, 1 subband, 64 channels, 768 spectra"),
}

PRECISION_NAMES = {0: "fp32_ffma", 1: "fp16", 2: "bf16", 3: "split_fp16", 4: "tf32_split"}
DTYPE_NAMES = {0: "f32", 1: "f16", 2: "bf16", 3: "f16 hi+lo", 4: "f32 as hi+lo: tf32 hi hi', bf16 cross terms"}
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def sky_seconds(w):
    return w["S"] * w["C"] / FS


def useful_xflops(w, n_subbands=None):
    """8 real flops per complex multiply-accumulate, upper triangle incl. autos,
    4 polarisation products, every (subband, channel, spectrum)."""
    B = w["N"] * (w["N"] + 1) // 2
    return 8.0 * B * 4 * w["C"] * w["S"] * (n_subbands or w["SB"])


def tf32_split_tiles(c):
    """Sum of 128 x 2n over the TF32-split X-stage's items of one channel
    (128-row blocks, diagonal and 64-input off-diagonal column tiles)."""
    ip = c.I_pad
    tiles = 0
    for row0 in range(0, ip, 128):
        tiles += 128 * 2 * min(128, ip - row0)
        for c0 in range(row0 + 128, ip, 64):
            tiles += 128 * 2 * min(64, ip - c0)
    return tiles


def executed_xflops_split(c, w):
    """(TF32, BF16) tensor-core flops the TF32-split X-stage issues: per 16
    spectra and item, 4 TF32 MMAs of 128 x 2n x 8 (hi hi') and 4 BF16 MMAs of
    128 x 2n x 16 (hi lo' + lo hi'), 2 flop per multiply-add."""
    per_sp = tf32_split_tiles(c) * c.S_pad * w["C"] * w["SB"]
    return 4.0 * per_sp, 8.0 * per_sp


def executed_xflops(c, w, precision):
    """Tensor-core flops the X-stage issues: 2 x 128 x N x K per MMA. FP16/BF16:
    4 real products of the I_pad x I_pad tile per spectrum (both triangles);
    split FP16: 12; TF32 split: the TF32 and BF16 flops together."""
    if precision == 4:
        return sum(executed_xflops_split(c, w))
    ip, sp = c.I_pad, c.S_pad
    nch = w["C"] * w["SB"]
    mult = {1: 4, 2: 4, 3: 12}[precision]
    return 2.0 * mult * ip * ip * sp * nch


def split_roofline(xflops, ex, ms, tpk, bpk):
    """Tensor roofline of the TF32-split X-stage, whose work is in two dtypes.
    Algorithmic work per complex MAC of the upper triangle: hi hi' in TF32
    (8 flop) and hi lo' + lo hi' in BF16 (16 flop). The time floor is
    F_tf32 / P_tf32 + F_bf16 / P_bf16; `achieved` is that work in TF32-
    equivalent flops (BF16 flops x P_tf32 / P_bf16) per second, so
    frac = floor / time against the TF32 peak."""
    f_t, f_b = xflops, 2.0 * xflops
    t = ms * 1e-3
    ach = (f_t + f_b * tpk / bpk) / t / 1e12
    ex_t, ex_b = ex
    ex_ach = (ex_t + ex_b * tpk / bpk) / t / 1e12
    return {"achieved": ach, "frac": ach / tpk, "executed_TFLOPs": ex_ach, "executed_frac": ex_ach / tpk,
            "floor_ms": (f_t / tpk + f_b / bpk) / 1e9, "executed_floor_ms": (ex_t / tpk + ex_b / bpk) / 1e9}


def samples(w):
    return 2 * w["N"] * w["S"] * w["C"] * w["SB"]


def fp32_alu_peak_tflops(sm_count, mhz=SM_MAX_MHZ):
    """FP32 FMA peak from the device's SM count and clock: SMs x 128 lanes x 2 flop."""
    return sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu record, or None when the
    kernel's source changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if sha != rec["sha256"] or rec["workload"] != workload:
            return None
        return float(rec["bytes_per_launch"])
    except Exception:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing (host logic, covered by a gloo test)
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, world_size: int, device=None) -> float:
    if world_size == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world_size: int):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_value(per_rank_sky_s: float, world_size: int, max_time_s: float) -> float:
    """Whole-job real-time factor: sky seconds processed by all ranks / slowest rank's time."""
    return per_rank_sky_s * world_size / max_time_s


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, name in enumerate(names):
            if any(r[5 + k].lower().startswith("active") for r in self.rows):
                reasons.append(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def workload_inputs(w, device):
    import numpy as np
    import torch

    import synth
    seed = synth.BASE_SEED + w["seed_index"]
    rng = np.random.default_rng(seed)
    N, C = w["N"], w["C"]
    tau = rng.uniform(-5e-6, 5e-6, N)
    ripple = synth.bandpass_ripple(rng, N, C) if w["ripple"] else None
    tones = []
    for k in range(w["ntones"]):
        d = tau + rng.uniform(-2e-7, 2e-7, N) * k
        tones.append(synth.Tone(amp=50.0 if w["fmt"] == 0 else 10.0,
                                channel=int(rng.integers(1, C)), delays=d, ripple=ripple))
    raw = synth.make_raw_torch(seed, w["fmt"], w["SB"], N, C, w["S"], n_taps=w["T"],
                               sigma=w["sigma"], tones=tones, device=device)
    taps = synth.kaiser_sinc_taps(w["T"], C)
    centres = synth.subband_centres(w["SB"])
    bandpass = None if ripple is None else torch.as_tensor(1.0 / ripple, dtype=torch.float32,
                                                           device=device).contiguous()
    delays = torch.as_tensor(tau, dtype=torch.float64, device=device)
    return raw, taps, centres, delays, bandpass, tau, ripple


# ---------------------------------------------------------------------------
# reference arm / cpu baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_sample(w, budget_s=30.0, max_subbands=32):
    """Time the oracle on whole subbands of the workload (subbands are
    independent, so the per-subband time scales linearly to SB)."""
    import numpy as np

    import oracle
    import synth
    seed = synth.BASE_SEED + w["seed_index"]
    rng = np.random.default_rng(seed)
    N, C, S, T = w["N"], w["C"], w["S"], w["T"]
    tau = rng.uniform(-5e-6, 5e-6, N)
    ripple = synth.bandpass_ripple(rng, N, C) if w["ripple"] else None
    tones = [synth.Tone(amp=50.0, channel=int(rng.integers(1, C)), delays=tau, ripple=ripple)]
    o = oracle.default()
    done, elapsed = 0, 0.0
    while done < max_subbands and (done == 0 or elapsed < budget_s / 2):
        blk = synth.make_block(seed + 7919 * done, w["fmt"], 1, N, C, S, n_taps=T,
                               sigma=w["sigma"], tones=tones)
        bp = None if ripple is None else 1.0 / ripple
        t0 = time.perf_counter()
        o.fx(blk.fmt, blk.raw, T, C, S, blk.taps, FS, blk.centres, tau, tau, bandpass=bp)
        elapsed += time.perf_counter() - t0
        done += 1
    per_sb = elapsed / done
    rtf = sky_seconds(w) / (per_sb * w["SB"])
    return {"value": rtf, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
            "sample": f"{done} of {w['SB']} subbands (whole subbands, FP64 C oracle with OpenMP), "
                      f"{elapsed:.1f} s, scaled linearly to {w['SB']} subbands",
            "seconds_per_subband": per_sb}


def config_of(w, ws):
    """The `config` dict both arms print (same workload, same keys)."""
    return {"workload": w["desc"], "stations": w["N"], "subbands_per_gpu": w["SB"], "channels": w["C"],
            "taps": w["T"], "spectra": w["S"],
            "input": {0: "complex int16", 1: "complex int8", 2: "complex int4"}[w["fmt"]],
            "x_stage": PRECISION_NAMES[w["precision"]],
            "l2": "inputs larger than L2 (raw block %.1f GB)" % (samples(w) * (4 if w["fmt"] == 0 else 2) / 1e9
                                                               * (w["S"] + w["T"] - 1) / w["S"]),
            "parallelism": f"subband blocks x {ws} GPU(s), no collective"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    steps = []
    for _ in range(args.warmup):
        oracle_sample(w, budget_s=2.0, max_subbands=1)
    for _ in range(args.steps):
        steps.append(oracle_sample(w, budget_s=10.0, max_subbands=1))
    per_sb = statistics.mean(s["seconds_per_subband"] for s in steps)
    value = sky_seconds(w) / (per_sb * w["SB"])
    cb = dict(steps[-1])
    cb["value"] = value
    cb["sample"] = (f"each step runs the oracle on 1 whole subband of the {w['SB']}-subband block "
                    f"({per_sb:.2f} s measured; ms_per_step is that time); value scales it linearly to "
                    f"{w['SB']} subbands ({per_sb * w['SB']:.0f} s per block)")
    cb.pop("seconds_per_subband", None)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_sb * 1e3,
            "ms_per_block_scaled": per_sb * w["SB"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args.gpus), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def vis_errors(got, ref, N):
    """Normwise relative error per subband (max over subbands) and the
    per-baseline max |dV_ij| / sqrt(|V_ii| |V_jj|), vis arrays [SB][C][B][4][2]."""
    import numpy as np
    g = got[..., 0] + 1j * got[..., 1]
    r = ref[..., 0] + 1j * ref[..., 1]
    norm = float(np.max(np.linalg.norm((g - r).reshape(g.shape[0], -1), axis=1) /
                        np.linalg.norm(r.reshape(r.shape[0], -1), axis=1)))
    jj, ii = np.meshgrid(np.arange(N), np.arange(N))
    up = ii <= jj
    i, j = ii[up], jj[up]
    b = j * (j + 1) // 2 + i
    auto = np.abs(r[:, :, (np.arange(N) * (np.arange(N) + 3)) // 2])
    worst = 0.0
    for p in range(2):
        for q in range(2):
            den = np.sqrt(auto[:, :, i, 3 * p] * auto[:, :, j, 3 * q])
            worst = max(worst, float(np.max(np.abs(g[:, :, b, 2 * p + q] - r[:, :, b, 2 * p + q]) /
                                            np.maximum(den, 1e-300))))
    return {"normwise": norm, "baseline_max": worst}


def oracle_reference(w, raw, taps, centres, tau, ripple, sbs):
    """FP64 oracle visibilities of the subbands `sbs` of the benchmarked block
    (raw samples copied to the host), to state each result's error."""
    import numpy as np

    import oracle
    r = raw[sbs].cpu().numpy()
    bp = None if ripple is None else 1.0 / ripple
    return oracle.fx(w["fmt"], r, w["T"], w["C"], w["S"], taps, FS, np.asarray(centres)[sbs], tau, tau,
                     bandpass=bp)


def measure_peaks(dev):
    """Burst dense tensor throughput of torch matmuls on this GPU (8192^3,
    best of 10): TF32 (FP32 inputs, allow_tf32), FP16 and BF16."""
    import torch
    n, out = 8192, {}
    stream = torch.cuda.current_stream()
    old = torch.backends.cuda.matmul.allow_tf32
    for name, dt, tf in (("tf32", torch.float32, True), ("fp16", torch.float16, False),
                         ("bf16", torch.bfloat16, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        torch.matmul(a, b)
        best = min(_time(lambda: torch.matmul(a, b), 1, stream) for _ in range(10))
        out[name + "_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = old
    out["how"] = "torch.matmul 8192^3, best of 10, CUDA events, this run"
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_fx(args, w):
    import numpy as np
    import torch

    import paper_1801_04834_gb300 as fxg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    prec = w["precision"]

    raw, taps, centres, delays, bandpass, tau, ripple = workload_inputs(w, dev)
    c = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                       fmt=w["fmt"], precision=prec)
    corr = torch.empty(c.corr_shape(), dtype=c.corr_dtype(), device=dev)
    vis = torch.empty(c.vis_shape(), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # one step = fx_channelize_correct (phase table + fused F-stage/correction)
    # + fx_correlate: 3 kernel launches
    def step(ev=None):
        if ev: ev[0].record(stream)
        c.channelize_correct(raw, delays, delays, bandpass=bandpass, out=corr)
        if ev: ev[1].record(stream)
        c.correlate(corr, vis)
        if ev: ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    vis_ids = os.environ.get("CUDA_VISIBLE_DEVICES")
    sampler = ClockSampler(vis_ids.split(",")[local] if vis_ids else str(local))
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    total_ms = start.elapsed_time(stop)
    ms_fc = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    ms_x = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    max_ms = max_over_ranks(total_ms, ws, dev)
    ms_step = max_ms / args.steps
    value = aggregate_value(sky_seconds(w) * args.steps, ws, max_ms / 1e3)

    # error of the benchmarked visibilities against the FP64 oracle on two
    # sampled subbands of this very block
    sbs = sorted({min(1, w["SB"] - 1), max(0, w["SB"] - 2)})
    ref = None
    parity = {"subbands": sbs, "oracle": "FP64 C oracle on the raw samples of these subbands"}
    if rank == 0 and not args.no_parity:
        ref = oracle_reference(w, raw, taps, centres, tau, ripple, sbs)
        parity[PRECISION_NAMES[prec]] = vis_errors(vis[sbs].double().cpu().numpy(), ref, w["N"])

    # the same step through the three separate calls (the paper's kernel split):
    # the stand-alone channeliser is the PPF's HBM roofline
    chan = torch.empty(c.chan_shape(), dtype=torch.float32, device=dev)

    def step3(ev):
        ev[0].record(stream)
        c.channelize(raw, chan)
        ev[1].record(stream)
        c.correct(chan, delays, delays, bandpass=bandpass, out=corr)
        ev[2].record(stream)
        c.correlate(corr, vis)
        ev[3].record(stream)

    ev3 = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps + 1)]
    for e in ev3:
        step3(e)
    torch.cuda.synchronize()
    ms_f = statistics.mean(e[0].elapsed_time(e[1]) for e in ev3[1:])
    ms_c = statistics.mean(e[1].elapsed_time(e[2]) for e in ev3[1:])
    ms_3 = statistics.mean(e[0].elapsed_time(e[3]) for e in ev3[1:])
    del chan

    peaks_run = measure_peaks(dev)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    xflops = useful_xflops(w)
    sz = c.sizes
    x_ach = xflops / (ms_x * 1e-3) / 1e12
    if prec == 4:
        ex = executed_xflops_split(c, w)
        tpk, bpk = peaks_run["tf32_tflops"], peaks_run["bf16_tflops"]
        sr = split_roofline(xflops, ex, ms_x, tpk, bpk)
        roof = {"kernel": "xcorr_tf32_kernel", "bound": "tensor", "achieved": sr["achieved"], "peak": tpk,
                "unit": "TFLOP/s", "frac": sr["frac"],
                "traffic": recorded_traffic("xcorr_tf32_kernel", args.workload),
                "peak_source": "dense TF32 tensor throughput measured in this run (torch TF32 matmul 8192^3, "
                               "burst); MEASURED_PEAKS.json holds no TF32 figure; BF16 peak of the same run "
                               f"({bpk:.0f} TFLOP/s) for the BF16 part",
                "algorithmic": f"{xflops:.4e} TF32 flop (hi hi') + {2 * xflops:.4e} BF16 flop (hi lo' + lo hi') "
                               f"per launch, 8 flop per complex MAC and product, upper triangle incl. autos; "
                               f"achieved in TF32-equivalent flops (BF16 x P_tf32/P_bf16), frac = "
                               f"floor {sr['floor_ms']:.2f} ms / measured {ms_x:.2f} ms",
                "useful_fp32_equiv_TFLOPs": x_ach, "useful_frac": x_ach / tpk,
                "executed_TFLOPs": sr["executed_TFLOPs"], "executed_frac": sr["executed_frac"],
                "executed_note": "whole 128-input tiles (both triangles) are issued: %.2fx the algorithmic work"
                                 % (sr["executed_floor_ms"] / sr["floor_ms"])}
    elif prec == 0:
        fpk = fp32_alu_peak_tflops(sm_count)
        roof = {"kernel": "xcorr_f32_kernel", "bound": "alu", "achieved": x_ach, "peak": fpk,
                "unit": "TFLOP/s", "frac": x_ach / fpk,
                "traffic": recorded_traffic("xcorr_f32_kernel", args.workload),
                "peak_source": f"derived: {sm_count} SMs (device property) x 128 FP32 lanes x 2 flop x 2070 MHz",
                "algorithmic": f"{xflops:.4e} useful flop per launch (8 per complex MAC)"}
    else:
        x_bytes = sz.corr_bytes + sz.vis_bytes
        xb = x_bytes / (ms_x * 1e-3) / 1e9
        roof = {"kernel": "xcorr_tc_kernel", "bound": "hbm", "achieved": xb, "peak": hbm,
                "unit": "GB/s", "frac": xb / hbm, "traffic": recorded_traffic("xcorr_tc_kernel", args.workload),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "algorithmic": f"{x_bytes:.4e} B per launch (operands + visibilities)"}
    f_bytes = sz.raw_bytes + sz.chan_bytes
    c_bytes = sz.chan_bytes + sz.corr_bytes
    fc_bytes = sz.raw_bytes + sz.corr_bytes
    kernels = {
        "channelize_correct_ms": ms_fc, "channelize_correct_GBps": fc_bytes / (ms_fc * 1e-3) / 1e9,
        "channelize_correct_hbm_frac": fc_bytes / (ms_fc * 1e-3) / 1e9 / hbm,
        "correlate_ms": ms_x, "correlate_useful_TFLOPs": x_ach,
        "three_call_path": {
            "step_ms": ms_3, "rtf": sky_seconds(w) / (ms_3 * 1e-3),
            "channelize_ms": ms_f, "channelize_GBps": f_bytes / (ms_f * 1e-3) / 1e9,
            "channelize_hbm_frac": f_bytes / (ms_f * 1e-3) / 1e9 / hbm,
            "correct_ms": ms_c, "correct_GBps": c_bytes / (ms_c * 1e-3) / 1e9,
            "correct_hbm_frac": c_bytes / (ms_c * 1e-3) / 1e9 / hbm},
        "fp32_alu_peak_TFLOPs": fp32_alu_peak_tflops(sm_count),
    }
    # measured FP32 FMA throughput (registers only) beside the derived ALU peak
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    nblk, iters = 8 * sm_count, 4096
    probe = lambda: c.lib.fx_ffma_probe(iters, nblk, ctypes.c_void_p(sink.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
    probe()
    ms_probe = _time(probe, 3, stream)
    kernels["fp32_fma_probe_tflops"] = nblk * 256.0 * iters * 512 / (ms_probe * 1e-3) / 1e12

    # ---- the other X-stage forms on the same block, each with the fused
    # F-stage writing its own operand layout; errors against the same oracle ----
    variants = {}
    if not args.no_variants:
        for vp in (0, 4, 1, 2, 3):
            if vp == prec:
                continue
            name = PRECISION_NAMES[vp]
            try:
                variants[name] = precision_variant(args, w, vp, raw, taps, centres, delays, bandpass, stream,
                                                   sbs, ref)
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)[:200]}
        head = {"step_ms": ms_step, "correlate_ms": ms_x}
        for name, v in variants.items():
            if "step_ms" in v:
                v["step_speedup_vs_" + PRECISION_NAMES[prec]] = head["step_ms"] / v["step_ms"]
                v["xstage_speedup_vs_" + PRECISION_NAMES[prec]] = head["correlate_ms"] / v["correlate_ms"]
        ff = variants.get("fp32_ffma")
        if ff and "step_ms" in ff:
            for name, v in variants.items():
                if "step_ms" in v and name != "fp32_ffma":
                    v["step_speedup_vs_fp32_ffma"] = ff["step_ms"] / v["step_ms"]
                    v["xstage_speedup_vs_fp32_ffma"] = ff["correlate_ms"] / v["correlate_ms"]
            kernels["step_speedup_vs_fp32_ffma"] = ff["step_ms"] / ms_step
            kernels["xstage_speedup_vs_fp32_ffma"] = ff["correlate_ms"] / ms_x

    # ---- end to end: pinned host raw in, visibilities out, copies timed ----
    # fx_process_host: host raw in, host visibilities out, subband chunks with
    # the H2D / compute / D2H of consecutive chunks overlapped (library streams)
    e2e = None
    if not args.no_e2e:
        h_raw = torch.empty(raw.shape, dtype=raw.dtype, pin_memory=True)
        h_raw.copy_(raw)
        h_vis = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
        h_tau = torch.as_tensor(tau, dtype=torch.float64)
        h_bp = None if bandpass is None else bandpass.cpu()
        del corr
        torch.cuda.empty_cache()
        chunk = max(1, min(w["SB"], args.host_chunk))
        ch = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                            fmt=w["fmt"], precision=prec, host_chunk_subbands=chunk)

        def e2e_step():
            ch.process_host(h_raw, h_tau, h_tau, bandpass=h_bp, out=h_vis)

        e2e_step()
        barrier(ws)
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t0) * 1e3
        e_ms = max_over_ranks(max(e0.elapsed_time(e1), wall_ms), ws, dev)
        e2e_err = float(torch.linalg.vector_norm(h_vis.double() - vis.cpu().double()) /
                        torch.linalg.vector_norm(vis.cpu().double()))
        e2e = {"value": aggregate_value(sky_seconds(w) * args.steps, ws, e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sz.raw_bytes + 16 * w["N"]
                                         + (0 if h_bp is None else 4 * w["N"] * w["C"])),
               "d2h_bytes_per_step": int(sz.vis_bytes), "ms_per_step": e_ms / args.steps,
               "api": f"fx_process_host, {chunk}-subband chunks, pinned host buffers",
               "h2d_GBps": sz.raw_bytes / (e_ms / args.steps * 1e-3) / 1e9,
               "rel_diff_vs_device_path": e2e_err}
        ch.close()
        del h_raw, h_vis

    del raw
    torch.cuda.empty_cache()
    precision_form = None
    if not args.no_precision_form and w["SB"] > 8:
        try:
            precision_form = measure_precision_form(args, dev)
        except Exception as ex:
            precision_form = {"error": str(ex)[:300]}
        torch.cuda.empty_cache()
    extras = {}
    if not args.no_extras:
        for key, fn in (("batching", measure_batching), ("differentiation", measure_adjoint),
                        ("beamformer", measure_beamformer)):
            torch.cuda.empty_cache()
            try:
                extras[key] = fn(args, dev)
            except Exception as ex:
                extras[key] = {"error": str(ex)[:300]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w)
        cpu.pop("seconds_per_subband", None)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAMES[prec], "data": "synthetic",
        "config": config_of(w, ws),
        "roofline": roof,
        "kernels": kernels,
        "parity_vs_oracle": parity,
        "samples_per_s": samples(w) * ws / (ms_step * 1e-3),
        "x_stage_useful_TFLOPs": x_ach,
        "peaks_measured_here": peaks_run,
        "variants": variants,
        "precision_form": precision_form,
        **extras,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    c.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def precision_variant(args, w, vp, raw, taps, centres, delays, bandpass, stream, sbs, ref):
    """One X-stage precision on a resident raw block: the fused F-stage in that
    precision's operand layout + the X-stage, timed as a step and alone, with
    the error of the result against the oracle visibilities `ref` of `sbs`."""
    import torch

    import paper_1801_04834_gb300 as fxg
    dev = raw.device
    cv = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                        fmt=w["fmt"], precision=vp)
    corr_v = torch.empty(cv.corr_shape(), dtype=cv.corr_dtype(), device=dev)
    vis_v = torch.empty(cv.vis_shape(), dtype=torch.float32, device=dev)

    def fstage():
        cv.channelize_correct(raw, delays, delays, bandpass=bandpass, out=corr_v)

    def xstage():
        cv.correlate(corr_v, vis_v)

    for _ in range(2):
        fstage()
        xstage()
    step_ms = _time(lambda: (fstage(), xstage()), args.steps, stream)
    f_ms = _time(fstage, args.steps, stream)
    x_ms = _time(xstage, args.steps, stream)
    fstage()
    xstage()
    torch.cuda.synchronize()
    xflops = useful_xflops(w)
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    fc_bytes = cv.sizes.raw_bytes + cv.sizes.corr_bytes
    out = {"step_ms": step_ms, "step_rtf": sky_seconds(w) / (step_ms * 1e-3),
           "channelize_correct_ms": f_ms, "channelize_correct_hbm_frac": fc_bytes / (f_ms * 1e-3) / 1e9 / hbm,
           "correlate_ms": x_ms, "correlate_useful_TFLOPs": xflops / (x_ms * 1e-3) / 1e12}
    if vp != 0:
        ex = executed_xflops(cv, w, vp)
        out["correlate_executed_TFLOPs"] = ex / (x_ms * 1e-3) / 1e12
    if vp in (1, 2, 3):
        xb = cv.sizes.corr_bytes + cv.sizes.vis_bytes
        out["correlate_hbm_frac"] = xb / (x_ms * 1e-3) / 1e9 / hbm
    if ref is not None:
        out["error_vs_oracle"] = vis_errors(vis_v[sbs].double().cpu().numpy(), ref, w["N"])
    del corr_v, vis_v
    cv.close()
    return out


def measure_precision_form(args, dev):
    """The precision workload at its own shape (LOFAR 8-bit mode): 64 stations
    x 2 pols, 488 subbands of complex int8 samples (sigma 20, clipped) + one
    point source, 16-tap PPF to 256 channels in FP32, 768 spectra per block.
    The X-stage in FP16, BF16 and split FP16 (FP32 accumulation), against the
    two FP32 paths (TF32 split on the tensor cores, FFMA on the CUDA cores) at
    the same shape; each result's error against the FP64 oracle on two
    sampled subbands of this block."""
    import torch
    w = WORKLOADS["lofar8_fp16"]
    raw, taps, centres, delays, bandpass, tau, ripple = workload_inputs(w, dev)
    stream = torch.cuda.current_stream()
    sbs = [1, w["SB"] - 2]
    ref = None if args.no_parity else oracle_reference(w, raw, taps, centres, tau, ripple, sbs)
    res = {"workload": w["desc"], "subbands_checked": sbs}
    for vp in (4, 0, 1, 2, 3):
        name = PRECISION_NAMES[vp]
        try:
            res[name] = precision_variant(args, w, vp, raw, taps, centres, delays, bandpass, stream, sbs, ref)
        except Exception as ex:
            res[name] = {"error": str(ex)[:200]}
        torch.cuda.empty_cache()
    for base in ("tf32_split", "fp32_ffma"):
        b = res.get(base, {})
        if "step_ms" not in b:
            continue
        for vp in (1, 2, 3):
            v = res.get(PRECISION_NAMES[vp], {})
            if "step_ms" in v:
                v["step_speedup_vs_" + base] = b["step_ms"] / v["step_ms"]
                v["xstage_speedup_vs_" + base] = b["correlate_ms"] / v["correlate_ms"]
    del raw
    return res


def _time(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_batching(args, dev):
    """Batching workload: 48 uneven correlation jobs (stations U{24..96},
    channels {16, 64, 256}, spectra U{256..3072}, int16 noise + one point
    source, FP16 operands). One autotuned persistent launch, replayed from a
    CUDA graph, against 48 fx_correlate launches (one per job)."""
    import ctypes

    import numpy as np
    import torch

    import paper_1801_04834_gb300 as fxg
    import synth
    from paper_1801_04834_gb300 import _abi
    lib = _abi.load()
    rng = np.random.default_rng(synth.BASE_SEED + 3)
    n_jobs = 48
    Ns, Cs, Ss = rng.integers(24, 97, n_jobs), rng.choice([16, 64, 256], n_jobs), rng.integers(256, 3073, n_jobs)
    jobs, flops, op_bytes, vis_bytes = [], 0.0, 0, 0
    for k in range(n_jobs):
        N, C, S = int(Ns[k]), int(Cs[k]), int(Ss[k])
        jr = np.random.default_rng(synth.BASE_SEED + 3000 + k)
        tau = jr.uniform(-5e-6, 5e-6, N)
        tone = synth.Tone(amp=50.0, channel=int(jr.integers(1, C)), delays=tau)
        c = fxg.Correlator(N, 1, C, S, taps=synth.kaiser_sinc_taps(16, C),
                           centres=synth.subband_centres(1, 120e6 + 0.2e6 * k), precision=1)
        raw = synth.make_raw_torch(synth.BASE_SEED + 3000 + k, 0, 1, N, C, S, tones=[tone],
                                   centre_hz=120e6 + 0.2e6 * k, device=dev)
        d = torch.as_tensor(tau, device=dev)
        corr = c.correct(c.channelize(raw), d, d)
        del raw
        jobs.append(dict(c=c, corr=corr, vis1=torch.empty(c.vis_shape(), dtype=torch.float32, device=dev),
                         visb=torch.empty(c.vis_shape(), dtype=torch.float32, device=dev), N=N, C=C, S=S))
        flops += 8.0 * (N * (N + 1) // 2) * 4 * C * S
        op_bytes += c.sizes.corr_bytes
        vis_bytes += c.sizes.vis_bytes
    stream = torch.cuda.current_stream()

    def singles():
        for j in jobs:
            j["c"].correlate(j["corr"], j["vis1"])

    singles()
    single_ms = _time(singles, args.steps, stream)
    arr = (_abi.fx_job * n_jobs)()
    for k, j in enumerate(jobs):
        arr[k].n_stations, arr[k].n_subbands, arr[k].n_channels, arr[k].n_spectra = j["N"], 1, j["C"], j["S"]
        arr[k].d_corr, arr[k].d_vis = j["corr"].data_ptr(), j["visb"].data_ptr()
    b = ctypes.c_void_p()
    _abi.check(lib.fx_batch_create(arr, n_jobs, 1, 0.0, ctypes.byref(b)), "fx_batch_create")
    sp = ctypes.c_void_p(stream.cuda_stream)
    default_plan = lib.fx_batch_describe(b).decode()
    default_ms = _time(lambda: lib.fx_correlate_batched(b, sp), args.steps, stream)
    _abi.check(lib.fx_batch_autotune(b, 3, sp), "fx_batch_autotune")
    plan = lib.fx_batch_describe(b).decode()
    gs = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=gs):
        _abi.check(lib.fx_correlate_batched(b, ctypes.c_void_p(gs.cuda_stream)), "capture")
    g.replay()
    torch.cuda.synchronize()
    graph_ms = _time(g.replay, args.steps, stream)
    diff = max(float((j["visb"] - j["vis1"]).abs().max() / j["vis1"].abs().max()) for j in jobs)
    lib.fx_batch_destroy(b)
    peaks, _ = measured_peaks()
    by = op_bytes + vis_bytes
    return {"jobs": n_jobs, "single_launches_ms": single_ms, "batched_default_ms": default_ms,
            "batched_graph_ms": graph_ms, "speedup_vs_single_launches": single_ms / graph_ms,
            "useful_TFLOPs": flops / (graph_ms * 1e-3) / 1e12,
            "hbm_GBps": by / (graph_ms * 1e-3) / 1e9, "hbm_frac": by / (graph_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "default_plan": default_plan, "autotuned_plan": plan,
            "max_rel_diff_vs_single": diff, "operand_GB": op_bytes / 1e9}


def measure_adjoint(args, dev):
    """Differentiation workload: 76 stations x 2 pols, 32 subbands, 64
    channels, 768 spectra, channelised FP32 (0.96 GB), gains |g| 0.8..1.2,
    delays +-50 ns. Forward (hot path with gains), raw visibilities
    (recomputed from the channelised block), adjoint, forward from R."""
    import numpy as np
    import torch

    import paper_1801_04834_gb300 as fxg
    import synth
    N, SB, C, S = 76, 32, 64, 768
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    # FP32 accuracy on the tensor cores (the headline's X-stage: hi hi' in TF32,
    # the cross terms in BF16) for the forward pass, R and the backward passes
    c = fxg.Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB),
                       precision=4)
    chan = torch.empty(c.chan_shape(), dtype=torch.float32, device=dev)
    chan.normal_(generator=torch.Generator(device=dev).manual_seed(synth.BASE_SEED + 4))
    g = torch.as_tensor(synth.random_gains(rng, N), dtype=torch.float32, device=dev)
    t = torch.as_tensor(rng.uniform(-50e-9, 50e-9, N), device=dev)
    corr = torch.empty(c.corr_shape(), dtype=torch.float32, device=dev)
    vis = torch.empty(c.vis_shape(), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def fwd():
        c.correct(chan, t, t, gains=g, out=corr)
        c.correlate(corr, vis)

    fwd()
    fwd_ms = _time(fwd, args.steps, stream)
    R = c.raw_vis(chan)
    raw_ms = _time(lambda: c.raw_vis(chan), args.steps, stream)
    G = torch.randn_like(vis)
    c.backward(R, g, t, G)
    bwd_ms = _time(lambda: c.backward(R, g, t, G), args.steps, stream)
    app_ms = _time(lambda: c.apply_gains(R, g, t, out=vis), args.steps, stream)
    # delays moving over the block: backward from the channelised block (recomputes
    # the corrected block, K and M1 with the X-stage, then the contraction)
    te = t + torch.as_tensor(rng.uniform(-20e-9, 20e-9, N), device=dev)
    wv = torch.empty((2,) + c.vis_shape(), dtype=torch.float32, device=dev)
    interp = lambda: c.backward_interp(chan, g, t, te, G, work_corr=corr, work_vis=wv)
    interp()
    interp_ms = _time(interp, args.steps, stream)
    peaks, _ = measured_peaks()
    vb = c.sizes.vis_bytes
    c.close()
    return {"workload": "76 stations x 2 pols, 32 subbands, 64 channels, 768 spectra, FP32 accuracy "
                        "(split X-stage on tcgen05: hi hi' TF32, cross terms BF16)",
            "forward_ms": fwd_ms, "raw_vis_recompute_ms": raw_ms, "backward_ms": bwd_ms,
            "apply_gains_ms": app_ms, "backward_moving_delays_ms": interp_ms,
            "backward_hbm_frac": 2 * vb / (bwd_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "train_step_ms_recompute": raw_ms + bwd_ms + fwd_ms}


def measure_beamformer(args, dev):
    """Beamformer workload (the paper's beamformer requirement): 48 stations x
    2 pols, 244 subbands of complex int16 samples, 256 channels, 768 spectra
    (1.00663 s), 127 coherent beams, Stokes I summed over 16 spectra. Step =
    fused F-stage with FP16 operands + beamformer (weight table + tcgen05
    kernel). Inputs (18.8 GB raw, 18.4 GB operands) are far larger than L2."""
    import numpy as np
    import torch

    import paper_1801_04834_gb300 as fxg
    import synth
    N, SB, C, S, NB, tint = 48, args.beam_subbands, 256, 768, 127, 16
    seed = synth.BASE_SEED + 5
    rng = np.random.default_rng(seed)
    tau = rng.uniform(-5e-6, 5e-6, N)
    tones = [synth.Tone(amp=50.0, channel=int(rng.integers(1, C)), delays=tau)]
    raw = synth.make_raw_torch(seed, 0, SB, N, C, S, n_taps=16, sigma=100.0, tones=tones, device=dev)
    c = fxg.Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB),
                       fmt=0, precision=1, operand_scale=2.0 ** -6, max_beams=NB)
    delays = torch.as_tensor(tau, device=dev)
    corr = torch.empty(c.corr_shape(), dtype=c.corr_dtype(), device=dev)
    bd = torch.as_tensor(rng.uniform(-2e-6, 2e-6, (NB, N)), device=dev)
    out = torch.empty(c.beam_shape(NB, 1, tint), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def fstage():
        c.channelize_correct(raw, delays, delays, out=corr)

    def beams():
        c.beamform(corr, bd, output=1, tint=tint, out=out)

    for _ in range(max(args.warmup, 3)):
        fstage()
        beams()
    step_ms = _time(lambda: (fstage(), beams()), args.steps, stream)
    f_ms = _time(fstage, args.steps, stream)
    b_ms = _time(beams, args.steps, stream)
    # incoherent beam (Stokes I per station, summed) on the same corrected block
    inc = torch.empty((SB, C, S // tint), dtype=torch.float32, device=dev)
    c.beamform_incoherent(corr, output=1, tint=tint, out=inc)
    i_ms = _time(lambda: c.beamform_incoherent(corr, output=1, tint=tint, out=inc), args.steps, stream)
    i_bytes = c.sizes.corr_bytes + inc.numel() * 4
    peaks, _ = measured_peaks()
    nb_pad = (NB + 63) // 64 * 64
    wbytes = SB * C * 3 * nb_pad * 64 * 2                             # planes (im, re, -im) per beam quarter
    bf_bytes = c.sizes.corr_bytes + 2 * wbytes + out.numel() * 4     # operands + weight table (write, read) + Stokes I
    useful = 8.0 * NB * N * 2 * S * C * SB
    sky_s = S * C / synth.SAMPLE_RATE_HZ
    res = {"workload": f"48 stations x 2 pols, {SB} subbands, complex int16, 256 channels, 768 spectra, "
                       "127 beams, coherent Stokes I / 16 spectra, FP16 operands",
           "step_ms": step_ms, "rtf": sky_s / (step_ms * 1e-3),
           "channelize_correct_ms": f_ms, "beamform_ms": b_ms,
           "beamform_useful_TFLOPs": useful / (b_ms * 1e-3) / 1e12,
           "beamform_hbm_GBps": bf_bytes / (b_ms * 1e-3) / 1e9,
           "beamform_hbm_frac": bf_bytes / (b_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
           "beamform_algorithmic_bytes": bf_bytes,
           "incoherent_ms": i_ms, "incoherent_hbm_frac": i_bytes / (i_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    c.close()
    del raw, corr, out, inc
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fx", choices=["fx", "reference"])
    ap.add_argument("--workload", default="lofar16_fp32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-chunk", type=int, default=4,
                    help="subbands per chunk of the host pipeline (e2e)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batching, differentiation and beamformer measurements")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle error checks")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip the 8-bit precision workload at its own shape")
    ap.add_argument("--beam-subbands", type=int, default=244,
                    help="subbands of the beamformer measurement (244 = the paper's requirement)")
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_fx(args, w)


if __name__ == "__main__":
    sys.exit(main())
