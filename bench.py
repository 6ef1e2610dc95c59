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
    "lofar8_fp16_small": dict(N=64, SB=16, C=256, S=768, T=16, fmt=1, precision=1, sigma=20.0,
                              ntones=1, ripple=False, seed_index=2,
                              desc="LOFAR 8-bit FP16 X-stage on 16 subbands (profiling size, ~2.5 GB)"),
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

    # the same step through the three separate calls (paper's kernel split)
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
    # FP32 X-stage in its other forms, same operands
    ms_x_forms = {}
    if w["precision"] == 0:
        for form in ("2x4", "3mult"):
            c2 = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                                fmt=w["fmt"], precision=0, xf32_form=form)
            vis2 = torch.empty_like(vis)
            c2.correlate(corr, vis2)
            ms_x_forms[form] = _time(lambda: c2.correlate(corr, vis2), args.steps, stream)
            ms_x_forms[form + "_rel_diff"] = float(torch.linalg.vector_norm((vis2 - vis).double()) /
                                                   torch.linalg.vector_norm(vis.double()))
            c2.close()
            del vis2
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
    fc_bytes = sz.raw_bytes + sz.corr_bytes
    kernels = {
        "channelize_correct_ms": ms_fc, "channelize_correct_GBps": fc_bytes / (ms_fc * 1e-3) / 1e9,
        "channelize_correct_hbm_frac": fc_bytes / (ms_fc * 1e-3) / 1e9 / hbm,
        "correlate_ms": ms_x, "correlate_useful_TFLOPs": xflops / (ms_x * 1e-3) / 1e12,
        "three_call_path": {
            "step_ms": ms_3, "rtf": sky_seconds(w) / (ms_3 * 1e-3),
            "channelize_ms": ms_f, "channelize_GBps": f_bytes / (ms_f * 1e-3) / 1e9,
            "channelize_hbm_frac": f_bytes / (ms_f * 1e-3) / 1e9 / hbm,
            "correct_ms": ms_c, "correct_GBps": c_bytes / (ms_c * 1e-3) / 1e9,
            "correct_hbm_frac": c_bytes / (ms_c * 1e-3) / 1e9 / hbm},
    }
    if ms_x_forms:
        kernels["correlate_form"] = "4x4-station tiles" if w["N"] >= 16 else "2x4-station tiles"
        kernels["correlate_other_forms_ms"] = ms_x_forms
    # measured FP32 FMA throughput (registers only) beside the derived ALU peak
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    nblk, iters = 8 * torch.cuda.get_device_properties(dev).multi_processor_count, 4096
    probe = lambda: c.lib.fx_ffma_probe(iters, nblk, ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    probe()
    ms_probe = _time(probe, 3, stream)
    kernels["fp32_fma_probe_tflops"] = nblk * 256.0 * iters * 512 / (ms_probe * 1e-3) / 1e12

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
        chunk = max(1, min(w["SB"], args.host_chunk))
        ch = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, n_taps=w["T"],
                            fmt=w["fmt"], precision=w["precision"], host_chunk_subbands=chunk)

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

    # ---- tensor-core variants of the X-stage on the same block ----
    variants = {}
    if not args.no_variants and w["precision"] == 0:
        ref_vis = vis.double()
        del corr
        for name, prec in (("fp16", 1), ("split_fp16", 3), ("bf16", 2), ("tf32_split", 4)):
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
                # the whole step in this precision: phase table + fused F-stage + X-stage
                a.record(stream)
                for _ in range(args.steps):
                    cv.channelize_correct(raw, delays, delays, bandpass=bandpass, out=corr_v)
                    cv.correlate(corr_v, vis_v)
                b.record(stream)
                torch.cuda.synchronize()
                vs = a.elapsed_time(b) / args.steps
                xb = cv.sizes.corr_bytes + cv.sizes.vis_bytes
                # executed tensor work: full I_pad x I_pad (both triangles) per spectrum and channel,
                # 4 real products (x3 for the split forms); TF32 peak = half the BF16 peak
                ip, sp = cv.I_pad, cv.S_pad
                mult = {1: 4, 2: 4, 3: 12, 4: 12}[prec]
                exec_fl = 2.0 * mult * ip * ip * sp * w["C"] * w["SB"]
                tpeak = float(peaks.get("bf16_tflops", 1890.0)) * (0.5 if prec == 4 else 1.0)
                variants[name] = {"correlate_ms": vx, "useful_TFLOPs": xflops / (vx * 1e-3) / 1e12,
                                  "executed_TFLOPs": exec_fl / (vx * 1e-3) / 1e12,
                                  "tensor_frac_executed": exec_fl / (vx * 1e-3) / 1e12 / tpeak,
                                  "tensor_frac_useful": xflops / (vx * 1e-3) / 1e12 / tpeak,
                                  "speedup_vs_fp32_xstage": ms_x / vx,
                                  "hbm_GBps": xb / (vx * 1e-3) / 1e9, "hbm_frac": xb / (vx * 1e-3) / 1e9 / hbm,
                                  "rel_err_vs_fp32_path": err,
                                  "step_ms": vs, "step_rtf": sky_seconds(w) / (vs * 1e-3)}
                del corr_v, vis_v
                cv.close()
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)[:200]}
        # F-stage and X-stage piece by piece through two L2-sized operand buffers
        # (fx_channelize_correlate); pieces of 48 MB or less
        for name, prec, G, TC in (("chunked_fp16", 1, 4, 384), ("chunked_fp32", 0, 4, 192)):
            try:
                if w["S"] % TC or w["SB"] < G:
                    continue
                cv = fxg.Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres,
                                    n_taps=w["T"], fmt=w["fmt"], precision=prec, chunk_subbands=G,
                                    chunk_spectra=TC)
                vis_v = torch.empty_like(vis)
                cv.channelize_correlate(raw, delays, delays, bandpass=bandpass, out=vis_v)
                torch.cuda.synchronize()
                vs = _time(lambda: cv.channelize_correlate(raw, delays, delays, bandpass=bandpass, out=vis_v),
                           args.steps, stream)
                err = float(torch.linalg.vector_norm(vis_v.double() - ref_vis) / torch.linalg.vector_norm(ref_vis))
                variants[name] = {"piece": f"{G} subbands x {TC} spectra", "step_ms": vs,
                                  "step_rtf": sky_seconds(w) / (vs * 1e-3), "rel_err_vs_fp32_path": err}
                del vis_v
                cv.close()
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)[:200]}

    del raw, chan
    extras = {}
    if not args.no_extras:
        torch.cuda.empty_cache()
        try:
            extras["batching"] = measure_batching(args, dev)
        except Exception as ex:
            extras["batching"] = {"error": str(ex)[:300]}
        torch.cuda.empty_cache()
        try:
            extras["differentiation"] = measure_adjoint(args, dev)
        except Exception as ex:
            extras["differentiation"] = {"error": str(ex)[:300]}
        torch.cuda.empty_cache()
        try:
            extras["beamformer"] = measure_beamformer(args, dev)
        except Exception as ex:
            extras["beamformer"] = {"error": str(ex)[:300]}

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
    c = fxg.Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB))
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
    peaks, _ = measured_peaks()
    vb = c.sizes.vis_bytes
    c.close()
    return {"workload": "76 stations x 2 pols, 32 subbands, 64 channels, 768 spectra, FP32",
            "forward_ms": fwd_ms, "raw_vis_recompute_ms": raw_ms, "backward_ms": bwd_ms,
            "apply_gains_ms": app_ms,
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
    ap.add_argument("--host-chunk", type=int, default=16,
                    help="subbands per chunk of the host pipeline (e2e)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batching, differentiation and beamformer measurements")
    ap.add_argument("--beam-subbands", type=int, default=244,
                    help="subbands of the beamformer measurement (244 = the paper's requirement)")
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_fx(args, w)


if __name__ == "__main__":
    sys.exit(main())
