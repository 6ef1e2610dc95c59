"""Coherent beamformer (fx_beamform, tcgen05) against the FP64 oracle.

Two comparisons per case:
  kernel  the beamformer on the GPU's own FP16/BF16 corrected block against
          the oracle's beamformer on the same block decoded to FP64: the only
          differences are the FP16/BF16 weights (relative 2^-11 / 2^-8 per
          weight) and FP32 accumulation, so normwise per subband the bound is
          2e-3 (FP16) and 1e-2 (BF16);
  end to end  raw samples -> fused F-stage -> beamformer against the oracle's
          channelize -> correct -> beamform in FP64: the operand rounding adds
          the same again (bounds 5e-3 and 2e-2).
Stokes values are compared the same way (they are squares, so the relative
error doubles; bounds are twice the voltage bounds).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import make_corr, per_subband_rel

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def decode_planar(c, corr):
    """FP16/BF16 planar corr [SB][C][2][I_pad][S_pad] -> oracle layout [SB][C][S][N][P][2]."""
    a = corr.float().cpu().numpy().astype(np.float64)[:, :, :, :c.I, :c.S] / c.operand_scale
    a = a.reshape(c.SB, c.C, 2, c.N, 2, c.S)                 # [SB][C][re/im][n][p][s]
    return np.ascontiguousarray(a.transpose(0, 1, 5, 3, 4, 2))


CASES = [  # (fmt, SB, N, C, S, NB, precision)
    (synth.CI16, 2, 7, 16, 200, 5, 1),
    (synth.CI8, 1, 48, 256, 96, 130, 1),
    (synth.CI16, 1, 64, 64, 128, 64, 2),
    (synth.CI16, 2, 1, 16, 64, 3, 1),
    (synth.CI8, 1, 20, 64, 256, 200, 1),
]


@pytest.mark.parametrize("fmt,SB,N,C,S,NB,precision", CASES)
@pytest.mark.parametrize("output,tint", [(0, 1), (1, 8), (2, 4), (2, 1)])
def test_beamform_vs_oracle(fmt, SB, N, C, S, NB, precision, output, tint):
    rng = np.random.default_rng(N * 1000 + C + S + NB)
    tau = rng.uniform(-5e-6, 5e-6, N)
    tone = synth.Tone(amp=30.0 if fmt == synth.CI16 else 8.0, channel=int(rng.integers(1, C)), delays=tau)
    blk = synth.make_block(500 + N + C, fmt, SB, N, C, S, sigma=100.0 if fmt == synth.CI16 else 20.0, tones=[tone])
    c = make_corr(blk, precision=precision, operand_scale=2.0 ** -6, max_beams=NB + 7)
    dl = rng.uniform(-2e-6, 2e-6, (NB, N))
    dl[0] = 0.0                                              # a phase-centre beam
    wts = rng.uniform(0.5, 1.5, N).astype(np.float32)
    t = torch.from_numpy(tau).cuda()
    corr = c.channelize_correct(torch.from_numpy(blk.raw).cuda(), t, t)
    got = c.beamform(corr, torch.from_numpy(dl).cuda(), torch.from_numpy(wts).cuda(), output=output, tint=tint)
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.float64)
    vb = {1: 2e-3, 2: 1e-2}[precision] * (2 if output else 1)
    # kernel: same operands on both sides
    ref_k = oracle.beamform(decode_planar(c, corr), FS, blk.centres, dl, wts, mode=output, tint=tint)
    e = per_subband_rel(got, ref_k)
    assert np.all(e < vb), ("kernel", e)
    # end to end from the raw samples
    chan = oracle.channelize(fmt, blk.raw, 16, C, S, blk.taps)
    ref = oracle.beamform(oracle.correct(chan, FS, blk.centres, tau, tau), FS, blk.centres, dl, wts,
                          mode=output, tint=tint)
    e2 = per_subband_rel(got, ref)
    assert np.all(e2 < 2.5 * vb), ("end to end", e2)
    c.close()


def test_beamform_point_source_gain():
    """Without delay compensation, a beam steered at the tone's delays adds
    all stations in phase: in the tone's channel its power is far above that
    of the phase-centre beam, where the stations add with scattered phases."""
    fmt, SB, N, C, S = synth.CI16, 1, 16, 64, 128
    rng = np.random.default_rng(3)
    tau = rng.uniform(-5e-6, 5e-6, N)
    ch = 20
    tone = synth.Tone(amp=200.0, channel=ch, delays=tau)
    blk = synth.make_block(9, fmt, SB, N, C, S, sigma=1.0, tones=[tone])
    c = make_corr(blk, precision=1, operand_scale=2.0 ** -8, max_beams=2)
    zero = torch.zeros(N, dtype=torch.float64, device="cuda")
    corr = c.channelize_correct(torch.from_numpy(blk.raw).cuda(), zero, zero)   # no delay compensation
    dl = np.stack([tau, np.zeros(N)])
    st = c.beamform(corr, torch.from_numpy(dl).cuda(), output=1, tint=32)[0, :, ch].cpu().numpy()
    on, off = st[0].sum(), st[1].sum()
    assert on > 10 * off, (on, off)
    c.close()


def test_beamform_rejects_bad_arguments():
    fmt, SB, N, C, S = synth.CI16, 1, 4, 16, 64
    blk = synth.make_block(1, fmt, SB, N, C, S)
    c = make_corr(blk, precision=1, max_beams=4)
    corr = torch.zeros(c.corr_shape(), dtype=c.corr_dtype(), device="cuda")
    with pytest.raises(RuntimeError):
        c.beamform(corr, torch.zeros((5, N), dtype=torch.float64, device="cuda"))   # more than max_beams
    with pytest.raises(RuntimeError):
        c.beamform(corr, torch.zeros((2, N), dtype=torch.float64, device="cuda"), output=1, tint=3)
    with pytest.raises(RuntimeError):
        c.beamform(corr, torch.zeros((2, N), dtype=torch.float64, device="cuda"), output=0, tint=2)
    c.close()
    with pytest.raises(RuntimeError):
        make_corr(blk, precision=0, max_beams=4)                                      # FP32 handle


@pytest.mark.parametrize("precision,bound", [(0, 2e-6), (1, 4e-3), (2, 2e-2), (4, 2e-6)])
@pytest.mark.parametrize("output,tint", [(1, 1), (1, 16), (2, 4)])
@pytest.mark.parametrize("fmt,SB,N,C,S", [(synth.CI16, 2, 7, 64, 96), (synth.CI8, 1, 24, 256, 64),
                                          (synth.CI16, 1, 1, 16, 160)])
def test_incoherent_vs_oracle(precision, bound, output, tint, fmt, SB, N, C, S):
    """Incoherent beam against the oracle on the GPU's own corrected block
    decoded to FP64 (the kernel alone; FP32 accumulation over stations and
    spectra, so FP32 operands are held to 2e-6), and end to end from the raw
    samples at the operand precision's bound."""
    rng = np.random.default_rng(N + C + S)
    tau = rng.uniform(-5e-6, 5e-6, N)
    blk = synth.make_block(800 + N, fmt, SB, N, C, S, sigma=100.0 if fmt == synth.CI16 else 20.0,
                           tones=[synth.Tone(amp=20.0, channel=3, delays=tau)])
    c = make_corr(blk, precision=precision, operand_scale=2.0 ** -6 if precision in (1, 2) else 0.0)
    wts = rng.uniform(0.5, 1.5, N).astype(np.float32)
    t = torch.from_numpy(tau).cuda()
    corr = c.channelize_correct(torch.from_numpy(blk.raw).cuda(), t, t)
    got = c.beamform_incoherent(corr, torch.from_numpy(wts).cuda(), output=output, tint=tint)
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.float64)
    # the same operands as the kernel read, in FP64 and unscaled
    if precision == 0:
        import paper_1801_04834_gb300 as fxg
        y = fxg.f32_unblock(corr, c.S).cpu().numpy().astype(np.float64)
    else:
        y = decode_planar(c, corr)
    ref_k = oracle.beamform_incoherent(y, wts, mode=output, tint=tint)
    ek = per_subband_rel(got, ref_k)
    assert np.all(ek < 2e-6), ("kernel", ek)
    chan = oracle.channelize(fmt, blk.raw, 16, C, S, blk.taps)
    ref = oracle.beamform_incoherent(oracle.correct(chan, FS, blk.centres, tau, tau), wts, mode=output, tint=tint)
    e = per_subband_rel(got, ref)
    assert np.all(e < bound), e
    c.close()
