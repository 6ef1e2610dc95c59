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
    """The FP32-accurate tensor-core X-stage (hi/lo TF32 split) on FP32 planar
    operands: 48 accumulator chains of 64 spectra summed in IEEE FP32 per
    channel; held to the FP32 path's bound (1e-5)."""
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
