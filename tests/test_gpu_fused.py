"""fx_channelize_correct (F-stage + correction in one pass) against the
two-call path (fx_channelize, fx_correct) and against the FP64 oracle.

The fused kernel evaluates the per-sample phasor with a fast sin/cos after an
FP32 reduction (absolute error ~4e-7), so FP32 outputs agree with the
two-call path to ~1e-6 normwise (bound 2e-6); FP16/BF16 outputs may differ by
one unit in the last place where that difference crosses a rounding
boundary. End to end against the oracle the stated bounds apply.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import make_corr, per_subband_rel, tone_block

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def d(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


CASES = [  # (fmt, SB, N, C, T, S)
    (synth.CI16, 2, 3, 64, 16, 37),
    (synth.CI16, 1, 9, 16, 16, 40),
    (synth.CI8, 2, 2, 256, 16, 19),
    (synth.CI16, 1, 5, 16, 4, 33),
    (synth.CI8, 1, 64, 64, 8, 130),
    (synth.CI16, 1, 1, 64, 16, 1),
]


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
@pytest.mark.parametrize("fmt,SB,N,C,T,S", CASES)
def test_fused_matches_two_calls(precision, fmt, SB, N, C, T, S):
    blk, tau, rip = tone_block(300 + S + N, fmt, SB, N, C, S, T=T, ripple=True,
                               sigma=20.0 if fmt == synth.CI8 else 100.0)
    rng = np.random.default_rng(4)
    te = tau + rng.uniform(-2e-8, 2e-8, N)
    g = synth.random_gains(rng, N)
    c = make_corr(blk, precision=precision, operand_scale=0.5 if precision else 0.0)
    raw = torch.from_numpy(blk.raw).cuda()
    tb_d, te_d, bp_d, g_d = d(tau, torch.float64), d(te, torch.float64), d(1.0 / rip), d(g)
    two = c.correct(c.channelize(raw), tb_d, te_d, bandpass=bp_d, gains=g_d)
    out = torch.full_like(two, float("nan")) if precision == 0 else torch.full_like(two, 7.0)
    fused = c.channelize_correct(raw, tb_d, te_d, bandpass=bp_d, gains=g_d, out=out)
    torch.cuda.synchronize()
    a, b = fused.double(), two.double()
    if precision == 3:   # compare the represented value hi + lo
        a, b = a[:, :, 0:2] + a[:, :, 2:4], b[:, :, 0:2] + b[:, :, 2:4]
    rel = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
    if precision in (0, 3):
        assert rel < 2e-6, rel
        if precision == 3 and (c.I_pad > c.I or c.S_pad > S):
            assert torch.all(fused[:, :, :, c.I:, :] == 0) and torch.all(fused[:, :, :, :, S:] == 0)
    else:
        # at most one unit of the operand type per element, plus the FP32-level
        # absolute difference (~1e-7 of the block's largest value) that shows on
        # elements near cancellation
        ulp = {1: 2.0 ** -10, 2: 2.0 ** -7}[precision]
        assert torch.all((a - b).abs() <= ulp * b.abs() + 1e-6 * b.abs().max()), rel
        assert rel < {1: 1e-4, 2: 1e-3}[precision], rel
        if c.I_pad > c.I or c.S_pad > S:
            assert torch.all(fused[:, :, :, c.I:, :] == 0) and torch.all(fused[:, :, :, :, S:] == 0)


@pytest.mark.parametrize("precision,bound", [(0, 1e-5), (1, 5e-3), (3, 1e-4), (4, 1e-5)])
def test_fused_end_to_end_vs_oracle(precision, bound):
    """8 stations x 2 pols, 1 subband, 64 channels, 768 spectra (the tiny
    workload) and a ragged 5-station int8 case, through the fused path."""
    for (fmt, SB, N, C, S) in [(synth.CI16, 1, 8, 64, 768), (synth.CI8, 2, 5, 256, 33)]:
        blk, tau, _ = tone_block(synth.BASE_SEED + N, fmt, SB, N, C, S,
                                 sigma=20.0 if fmt == synth.CI8 else 100.0)
        ref = oracle.fx(blk.fmt, blk.raw, 16, C, S, blk.taps, FS, blk.centres, tau, tau)
        c = make_corr(blk, precision=precision)
        t = d(tau, torch.float64)
        vis = c.correlate(c.channelize_correct(torch.from_numpy(blk.raw).cuda(), t, t))
        e = per_subband_rel(vis.cpu().numpy().astype(np.float64), ref)
        assert np.all(e < bound), (precision, N, e)


@pytest.mark.parametrize("precision,bound", [(0, 1e-5), (1, 5e-3), (4, 1e-5)])
@pytest.mark.parametrize("C,S", [(16, 40), (64, 33), (256, 17)])
def test_ci4_end_to_end(precision, bound, C, S):
    """4-bit mode: packed int4 samples through the two-call and fused paths
    against the FP64 oracle (which decodes the nibbles itself)."""
    N, SB = 6, 2
    rng = np.random.default_rng(C + S)
    tau = rng.uniform(-5e-6, 5e-6, N)
    tone = synth.Tone(amp=3.0, channel=int(rng.integers(1, C)), delays=tau)
    blk = synth.make_block(77 + C, synth.CI4, SB, N, C, S, sigma=2.5, tones=[tone])
    ref = oracle.fx(blk.fmt, blk.raw, 16, C, S, blk.taps, FS, blk.centres, tau, tau)
    c = make_corr(blk, precision=precision)
    raw = torch.from_numpy(blk.raw).cuda()
    t = d(tau, torch.float64)
    chan_ref = oracle.channelize(blk.fmt, blk.raw, 16, C, S, blk.taps)
    chan = c.channelize(raw).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(chan - chan_ref) / np.linalg.norm(chan_ref) < 2e-6
    for vis in (c.correlate(c.correct(c.channelize(raw), t, t)), c.correlate(c.channelize_correct(raw, t, t))):
        e = per_subband_rel(vis.cpu().numpy().astype(np.float64), ref)
        assert np.all(e < bound), e


@pytest.mark.parametrize("precision,fmt,SB,N,C,T,S,stations", [
    # grids that keep 4 rounds per CTA (ragged last round): the FIR/FFT buffer
    # and phase-table ping-pong of the warp-specialised kernel runs past its first reuse
    (0, synth.CI16, 2, 64, 64, 16, 1210, [0, 33, 63]),
    (1, synth.CI16, 2, 64, 64, 16, 1210, [1, 62]),
    (3, synth.CI16, 2, 64, 64, 16, 1210, [5, 60]),
    (4, synth.CI8, 2, 64, 64, 16, 1210, [0, 63]),
    (2, synth.CI16, 4, 64, 16, 4, 2430, [6, 58]),
    (0, synth.CI8, 4, 64, 16, 8, 2430, [2, 3, 61]),
    (0, synth.CI4, 2, 64, 64, 16, 1210, [9, 44]),
    # 256 channels, planar outputs (one CTA per station and pol, all 48 rounds of
    # the 8-bit workload's 768 spectra in one CTA)
    (1, synth.CI8, 5, 64, 256, 16, 768, [3, 50]),
    (3, synth.CI16, 5, 48, 256, 16, 768, [0, 47]),
    (4, synth.CI8, 5, 64, 256, 16, 768, [63]),
    (2, synth.CI16, 1, 3, 256, 8, 40, [0, 2]),          # 8 and 4 taps at 256 channels, ragged
    (1, synth.CI8, 2, 2, 256, 4, 33, [1]),
    # the LOFAR 16-bit shape on 13 subbands: 64 rounds per CTA as in the benchmark
    (0, synth.CI16, 13, 64, 64, 16, 3072, [7, 40]),
])
def test_fused_multiround_vs_oracle(precision, fmt, SB, N, C, T, S, stations):
    """Long CTA runs of the fused F-stage against the oracle's channelize +
    correct on a few stations (both treat stations independently). FP32
    outputs (plain and the TF32-split planes) to 2e-6 normwise; FP16 operands
    to 1e-3 (2^-11 relative rounding per value), split FP16 (hi + lo) to 2e-6,
    BF16 to 1e-2 (2^-8)."""
    import paper_1801_04834_gb300 as fxg
    rng = np.random.default_rng(S + C + precision + 10 * fmt)
    if fmt == synth.CI4:
        raw = rng.integers(0, 256, size=(SB, N, (S + T - 1) * C, 2, 1), dtype=np.uint8)
    else:
        amp = 60 if fmt == synth.CI8 else 300
        raw = rng.integers(-amp, amp + 1, size=(SB, N, (S + T - 1) * C, 2, 2),
                           dtype=np.int8 if fmt == synth.CI8 else np.int16)
    taps = synth.kaiser_sinc_taps(T, C)
    centres = synth.subband_centres(SB)
    tb = rng.uniform(-5e-6, 5e-6, N)
    te = tb + rng.uniform(-2e-8, 2e-8, N)
    bp = rng.uniform(0.7, 1.3, (N, C))
    g = synth.random_gains(rng, N)
    scaled = precision in (1, 2, 3)
    c = fxg.Correlator(N, SB, C, S, taps=taps, centres=centres, n_taps=T, fmt=fmt, precision=precision,
                       operand_scale=2.0 ** -8 if scaled else 0.0)
    corr = c.channelize_correct(torch.from_numpy(raw).cuda(), d(tb, torch.float64), d(te, torch.float64),
                                bandpass=d(bp), gains=d(g))
    sbs = [0, SB - 1]
    if precision == 0:
        y = fxg.f32_unblock(corr, S)[sbs].cpu().numpy().astype(np.float64)      # [2][C][S][N][P][2]
    else:
        a = corr[sbs].float().cpu().numpy().astype(np.float64)[:, :, :, :c.I, :S]
        if precision == 3:
            a = a[:, :, 0:2] + a[:, :, 2:4]                                      # hi + lo
        if scaled:
            a = a / c.operand_scale
        y = a.reshape(2, C, 2, N, 2, S).transpose(0, 1, 5, 3, 4, 2)             # [2][C][S][N][P][2]
    y = y[:, :, :, stations]
    chan = oracle.channelize(fmt, raw[sbs][:, stations], T, C, S, taps)
    ref = oracle.correct(chan, FS, centres[sbs], tb[stations], te[stations], bandpass=bp[stations],
                         gains=g[stations])
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    bound = {0: 2e-6, 1: 1e-3, 2: 1e-2, 3: 2e-6, 4: 2e-6}[precision]
    assert rel < bound, rel
    c.close()
