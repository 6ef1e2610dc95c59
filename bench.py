#!/usr/bin/env python3
"""Benchmark of the FX correlator hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole hot path over one block of synthetic
LOFAR-shaped input already resident in HBM: fx_channelize (FIR + FFT),
fx_correct (FP64 phase table + FP32 delay/bandpass rotation, transposing
write) and fx_correlate (X-stage), all through the C ABI.

Default workload: 64 stations x 2 pols, 244 subbands, complex int16 noise
(sigma 100) + 3 point sources with seeded delays (+-5 us) and per-station
bandpass ripple, 16-tap PPF to 64 channels, 3072 spectra per block
(1.00663 s of sky), FP32 path. Inputs (24.7 GB raw) are far larger than L2.

value  = real-time factor = seconds of sky processed by all ranks / wall second
e2e    = the same, with the raw block copied host->device from pinned memory and
         the visibilities copied back inside the timed region
Multi-GPU (torchrun): every rank processes its own 244-subband block (subbands
are independent; weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the only other place this file runs oracle/ code besides the
cpu_baseline leg).
"""
from __future__ import annotations

import argparse
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
    "lofar16_fp32": dict(N=64, SB=244, C=64, S=3072, T=16, fmt=0, precision=0, sigma=100.0,
                         ntones=3, ripple=True, seed_index=1,
                         desc="LOFAR 16-bit, FP32 path: 64 stations x 2 pols, 244 subbands, "
                              "16-tap PPF to 64 channels, 3072 spectra (1.00663 s) per block"),
    "lofar8_fp16": dict(N=64, SB=488, C=256, S=768, T=16, fmt=1, precision=1, sigma=20.0,
                        ntones=1, ripple=False, seed_index=2,
                        desc="LOFAR 8-bit, FP16 X-stage: 64 stations x 2 pols, 488 subbands, "
                             "16-tap PPF to 256 channels, 768 spectra (1.00663 s) per block"),
    "lofar16_fp32_small": dict(N=64, SB=8, C=64, S=3072, T=16, fmt=0, precision=0, sigma=100.0,
                               ntones=3, ripple=True, seed_index=1,
                               desc="LOFAR 16-bit FP32 path on 8 subbands (profiling size, ~4 GB)"),
    "tiny_fp32": dict(N=8, SB=1, C=64, S=768, T=16, fmt=0, precision=0, sigma=100.0,
                      ntones=1, ripple=False, seed_index=0,
                      desc="8 stations x 2 pols, 1 subband, 64 channels, 768 spectra"),
}

FP32_LANES_PER_SM = 128
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def sky_seconds(w):
    return w["S"] * w["C"] / FS


def useful_xflops(w, n_subbands=None):
    """8 real flops per complex multiply-accumulate, upper triangle incl. autos,
    4 polarisation products, every (subband, channel, spectrum)."""
    B = w["N"] * (w["N"] + 1) // 2
    return 8.0 * B * 4 * w["C"] * w["S"] * (n_subbands or w["SB"])


def samples(w):
    return 2 * w["N"] * w["S"] * w["C"] * w["SB"]


def fp32_alu_peak_tflops(mhz=SM_MAX_MHZ):
    """FP32 FMA peak from unit counts and clock: 152 SMs x 128 lanes x 2 flop."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


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
    cb["sample"] = f"1 of {w['SB']} subbands per step, {args.steps} steps, scaled linearly"
    cb.pop("seconds_per_subband", None)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_sb * w["SB"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["desc"]}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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

    raw, taps, centres, delays, bandpass, tau, ripple = workload_inputs(w, dev)
    c = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                       fmt=w["fmt"], precision=w["precision"])
    chan = torch.empty(c.chan_shape(), dtype=torch.float32, device=dev)
    corr = torch.empty(c.corr_shape(), dtype=c.corr_dtype(), device=dev)
    vis = torch.empty(c.vis_shape(), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev: ev[0].record(stream)
        c.channelize(raw, chan)
        if ev: ev[1].record(stream)
        c.correct(chan, delays, delays, bandpass=bandpass, out=corr)
        if ev: ev[2].record(stream)
        c.correlate(corr, vis)
        if ev: ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
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
    ms_f = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    ms_c = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    ms_x = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    max_ms = max_over_ranks(total_ms, ws, dev)
    ms_step = max_ms / args.steps
    value = aggregate_value(sky_seconds(w) * args.steps, ws, max_ms / 1e3)

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    xflops = useful_xflops(w)
    sz = c.sizes
    if w["precision"] == 0:
        x_ach = xflops / (ms_x * 1e-3) / 1e12
        roof = {"kernel": "xcorr_f32_kernel", "bound": "alu", "achieved": x_ach,
                "peak": fp32_alu_peak_tflops(), "unit": "TFLOP/s",
                "frac": x_ach / fp32_alu_peak_tflops(),
                "traffic": recorded_traffic("xcorr_f32_kernel", args.workload),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "algorithmic": f"{xflops:.4e} useful flop per launch (8 per complex MAC)"}
    else:
        x_bytes = sz.corr_bytes + sz.vis_bytes
        x_ach = x_bytes / (ms_x * 1e-3) / 1e9
        roof = {"kernel": "xcorr_tc_kernel", "bound": "hbm", "achieved": x_ach, "peak": hbm,
                "unit": "GB/s", "frac": x_ach / hbm,
                "traffic": recorded_traffic("xcorr_tc_kernel", args.workload),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "algorithmic": f"{x_bytes:.4e} B per launch (operands + visibilities)"}
    f_bytes = sz.raw_bytes + sz.chan_bytes
    c_bytes = sz.chan_bytes + sz.corr_bytes
    kernels = {
        "channelize_ms": ms_f, "channelize_GBps": f_bytes / (ms_f * 1e-3) / 1e9,
        "channelize_hbm_frac": f_bytes / (ms_f * 1e-3) / 1e9 / hbm,
        "correct_ms": ms_c, "correct_GBps": c_bytes / (ms_c * 1e-3) / 1e9,
        "correct_hbm_frac": c_bytes / (ms_c * 1e-3) / 1e9 / hbm,
        "correlate_ms": ms_x, "correlate_useful_TFLOPs": xflops / (ms_x * 1e-3) / 1e12,
    }

    # ---- end to end: pinned host raw in, visibilities out, copies timed ----
    e2e = None
    if not args.no_e2e:
        h_raw = torch.empty(raw.shape, dtype=raw.dtype, pin_memory=True)
        h_raw.copy_(raw)
        h_vis = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
        h_tau = torch.as_tensor(tau, dtype=torch.float64).pin_memory()

        def e2e_step():
            raw.copy_(h_raw, non_blocking=True)
            delays.copy_(h_tau, non_blocking=True)
            step()
            h_vis.copy_(vis, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        e2e = {"value": aggregate_value(sky_seconds(w) * args.steps, ws, e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sz.raw_bytes + 8 * w["N"]),
               "d2h_bytes_per_step": int(sz.vis_bytes), "ms_per_step": e_ms / args.steps}
        del h_raw, h_vis

    # ---- tensor-core variants of the X-stage on the same block ----
    variants = {}
    if not args.no_variants and w["precision"] == 0:
        ref_vis = vis.double()
        del corr
        for name, prec in (("fp16", 1), ("split_fp16", 3), ("bf16", 2)):
            try:
                cv = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres,
                                    n_taps=w["T"], fmt=w["fmt"], precision=prec)
                corr_v = torch.empty(cv.corr_shape(), dtype=cv.corr_dtype(), device=dev)
                vis_v = torch.empty_like(vis)
                cv.correct(chan, delays, delays, bandpass=bandpass, out=corr_v)
                cv.correlate(corr_v, vis_v)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(args.steps):
                    cv.correlate(corr_v, vis_v)
                b.record(stream)
                torch.cuda.synchronize()
                vx = a.elapsed_time(b) / args.steps
                err = float(torch.linalg.vector_norm(vis_v.double() - ref_vis) /
                            torch.linalg.vector_norm(ref_vis))
                xb = cv.sizes.corr_bytes + cv.sizes.vis_bytes
                variants[name] = {"correlate_ms": vx, "useful_TFLOPs": xflops / (vx * 1e-3) / 1e12,
                                  "speedup_vs_fp32_xstage": ms_x / vx,
                                  "hbm_GBps": xb / (vx * 1e-3) / 1e9, "hbm_frac": xb / (vx * 1e-3) / 1e9 / hbm,
                                  "rel_err_vs_fp32_path": err}
                del corr_v, vis_v
                cv.close()
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)[:200]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w)
        cpu.pop("seconds_per_subband", None)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if w["precision"] == 0 else "f16",
        "data": "synthetic",
        "config": {"workload": w["desc"], "stations": w["N"], "subbands_per_gpu": w["SB"],
                   "channels": w["C"], "taps": w["T"], "spectra": w["S"],
                   "input": "complex int16" if w["fmt"] == 0 else "complex int8",
                   "l2": "inputs larger than L2 (raw block %.1f GB)" % (sz.raw_bytes / 1e9),
                   "parallelism": f"subband blocks x {ws} GPU(s), no collective"},
        "roofline": roof,
        "kernels": kernels,
        "samples_per_s": samples(w) * ws / (ms_step * 1e-3),
        "x_stage_useful_TFLOPs": xflops / (ms_x * 1e-3) / 1e12,
        "variants": variants,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    c.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


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
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_fx(args, w)


if __name__ == "__main__":
    sys.exit(main())
