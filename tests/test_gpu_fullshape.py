"""X-stages at the LOFAR 16-bit shape in the launch configuration bench.py
times (64 stations, 64 channels, 3072 spectra; 10 subbands are enough for
the production grid: 256-thread CTAs, 32-spectrum chunks for the FFMA form;
all SMs busy for the persistent tensor-core form), against the FP64 oracle on
sampled channels with the kernels' exact operands.

Bounds: FP32 X-stage 1e-5 normwise per channel (3072-term FP32 sums, about
sqrt(S) * 2^-24 relative); FP16 operands accumulated in FP32 on the tensor
cores 1e-4 (the operands are exact, so this is accumulation only)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import fx

pytestmark = pytest.mark.gpu
N, C, S, SB = 64, 64, 3072, 10
SAMPLES = [(0, 0), (4, 31), (9, 63)]          # (subband, channel)


def _correlator(precision):
    return fx().Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB),
                           precision=precision)


def _rel(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_xstage_fp32_full_shape_sampled():
    fxg = fx()
    c = _correlator(0)
    g = torch.Generator(device="cuda").manual_seed(180104834)
    y = torch.randn((SB, C, S, N, 2, 2), generator=g, device="cuda") * 30.0      # [SB][C][S][N][P][2]
    vis = c.correlate(fxg.f32_block(y))
    torch.cuda.synchronize()
    for sb, k in SAMPLES:
        ref = oracle.correlate(y[sb:sb + 1, k:k + 1].double().cpu().numpy())[0, 0]
        e = _rel(vis[sb, k].double().cpu().numpy(), ref)
        assert e < 1e-5, (sb, k, e)
    c.close()


def test_xstage_fp16_full_shape_sampled():
    c = _correlator(1)
    I = 2 * N
    g = torch.Generator(device="cuda").manual_seed(180104835)
    ops = torch.zeros(c.corr_shape(), dtype=torch.float16, device="cuda")          # [SB][C][2][I_pad][S_pad]
    ops[:, :, :, :I, :S] = (torch.randn((SB, C, 2, I, S), generator=g, device="cuda") * 30.0).half()
    vis = c.correlate(ops)
    torch.cuda.synchronize()
    for sb, k in SAMPLES:
        pl = ops[sb, k, :, :I, :S].double().cpu().numpy()                          # [2][I][S]
        held = np.ascontiguousarray(pl.transpose(2, 1, 0)).reshape(1, 1, S, N, 2, 2)
        ref = oracle.correlate(held)[0, 0]
        e = _rel(vis[sb, k].double().cpu().numpy(), ref)
        assert e < 1e-4, (sb, k, e)
    c.close()


def test_xstage_tf32_split_full_shape_sampled():
    """The FP32-accurate tensor-core X-stage (hi hi' in TF32, hi lo' + lo hi'
    in BF16) on FP32 planar operands: 48 accumulator chains of 64 spectra
    summed in IEEE FP32 per channel; held to the FP32 path's bound (1e-5)."""
    c = _correlator(4)
    I = 2 * N
    g = torch.Generator(device="cuda").manual_seed(180104836)
    ops = torch.zeros(c.corr_shape(), dtype=torch.float32, device="cuda")          # [SB][C][2][I_pad][S_pad]
    ops[:, :, :, :I, :S] = torch.randn((SB, C, 2, I, S), generator=g, device="cuda") * 30.0
    vis = c.correlate(ops)
    torch.cuda.synchronize()
    for sb, k in SAMPLES:
        pl = ops[sb, k, :, :I, :S].double().cpu().numpy()
        held = np.ascontiguousarray(pl.transpose(2, 1, 0)).reshape(1, 1, S, N, 2, 2)
        ref = oracle.correlate(held)[0, 0]
        e = _rel(vis[sb, k].double().cpu().numpy(), ref)
        assert e < 1e-5, (sb, k, e)
    c.close()


def test_xstage_split_fp16_full_shape_sampled():
    """Split FP16 operands (hi, lo planes) at the full shape: the represented
    values hi + lo are exact inputs to the oracle; hi hi' + hi lo' + lo hi'
    leaves out lo lo' (below 2^-22 relative), accumulation in FP32: 1e-4."""
    c = _correlator(3)
    I = 2 * N
    g = torch.Generator(device="cuda").manual_seed(180104837)
    x = torch.randn((SB, C, 2, I, S), generator=g, device="cuda") * 30.0
    hi = x.half()
    lo = (x - hi.float()).half()
    ops = torch.zeros(c.corr_shape(), dtype=torch.float16, device="cuda")          # [SB][C][4][I_pad][S_pad]
    ops[:, :, 0:2, :I, :S] = hi
    ops[:, :, 2:4, :I, :S] = lo
    vis = c.correlate(ops)
    torch.cuda.synchronize()
    for sb, k in SAMPLES:
        pl = (ops[sb, k, 0:2, :I, :S].double() + ops[sb, k, 2:4, :I, :S].double()).cpu().numpy()
        held = np.ascontiguousarray(pl.transpose(2, 1, 0)).reshape(1, 1, S, N, 2, 2)
        ref = oracle.correlate(held)[0, 0]
        e = _rel(vis[sb, k].double().cpu().numpy(), ref)
        assert e < 1e-4, (sb, k, e)
    c.close()


def test_xstage_tf32_split_76_stations_sampled():
    """The FP32-accurate tensor-core X-stage at the differentiation workload's
    shape (76 stations = 152 inputs: a 128-column diagonal tile, a 32-column
    off-diagonal tile and a ragged 32-row diagonal tile per channel; 32
    subbands, 64 channels, 768 spectra) against the oracle on sampled channels
    with the kernel's exact operands: 1e-5 normwise, and per baseline
    max |dV_ij| / sqrt(|V_ii| |V_jj|) below 2e-5."""
    from test_gpu_parity import baseline_max_rel
    N76, SB76, S76 = 76, 32, 768
    c = fx().Correlator(N76, SB76, C, S76, taps=synth.kaiser_sinc_taps(16, C),
                        centres=synth.subband_centres(SB76), precision=4)
    I = 2 * N76
    g = torch.Generator(device="cuda").manual_seed(180104838)
    ops = torch.zeros(c.corr_shape(), dtype=torch.float32, device="cuda")
    ops[:, :, :, :I, :S76] = torch.randn((SB76, C, 2, I, S76), generator=g, device="cuda") * 30.0
    vis = c.correlate(ops)
    torch.cuda.synchronize()
    for sb, k in [(0, 0), (17, 40), (31, 63)]:
        pl = ops[sb, k, :, :I, :S76].double().cpu().numpy()
        held = np.ascontiguousarray(pl.transpose(2, 1, 0)).reshape(1, 1, S76, N76, 2, 2)
        ref = oracle.correlate(held)[0, 0]
        got = vis[sb, k].double().cpu().numpy()
        assert _rel(got, ref) < 1e-5, (sb, k)
        assert baseline_max_rel(got[None, None], ref[None, None], N76) < 2e-5, (sb, k)
    c.close()


def test_fp32_accurate_path_lofar_block_vs_oracle():
    """The headline step (fused F-stage writing FP32 planar operands + TF32
    split X-stage) on a LOFAR 16-bit block drawn with the benchmark's recipe
    (64 stations, 64 channels, 3072 spectra, int16 noise + 3 tones + bandpass
    ripple; 13 subbands keep the benchmark's 64-round CTAs) against the FP64
    oracle end to end on two subbands: 1e-5 normwise, per-baseline max below
    1e-4."""
    from test_gpu_parity import baseline_max_rel
    import bench
    w = dict(bench.WORKLOADS["lofar16_fp32"], SB=13)
    raw, taps, centres, delays, bandpass, tau, ripple = bench.workload_inputs(w, torch.device("cuda"))
    c = fx().Correlator(w["N"], w["SB"], w["C"], w["S"], taps=taps, centres=centres, precision=4)
    vis = c.correlate(c.channelize_correct(raw, delays, delays, bandpass=bandpass))
    torch.cuda.synchronize()
    sbs = [1, 11]
    ref = oracle.fx(0, raw[sbs].cpu().numpy(), 16, w["C"], w["S"], taps, synth.SAMPLE_RATE_HZ,
                    np.asarray(centres)[sbs], tau, tau, bandpass=1.0 / ripple)
    got = vis[sbs].double().cpu().numpy()
    for k in range(2):
        assert _rel(got[k], ref[k]) < 1e-5, k
    assert baseline_max_rel(got, ref, w["N"]) < 1e-4
    c.close()
