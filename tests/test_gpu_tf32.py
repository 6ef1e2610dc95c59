"""FP32-accurate tensor-core X-stage (FX_TF32_SPLIT) against the FP64 oracle.

Each FP32 corrected sample x is split in the kernel into hi = x with the 13
low mantissa bits cleared (exactly a TF32 value) and lo = x - hi (exact in
FP32, |lo| < 2^-10 |x|); the MMAs form hi hi' in TF32 and the cross terms
hi lo' + lo hi' in BF16, all with FP32 accumulation. The BF16 rounding of
the cross terms' operands moves each product by at most 2^-18 of itself
(about 2^-21 RMS, zero mean) and the dropped lo lo' term is below 2^-20, so
the visibilities must meet the FP32 path's bound: normwise relative error
per subband below 1e-5 against the oracle, and agreement with the FFMA
X-stage on the same corrected block to the same level.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import baseline_max_rel, make_corr, per_subband_rel, tone_block

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def d(a, dt=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


CASES = [  # (fmt, SB, N, C, S)
    (synth.CI16, 1, 8, 64, 768),
    (synth.CI16, 2, 5, 16, 33),
    (synth.CI8, 2, 64, 64, 100),
    (synth.CI8, 1, 48, 256, 64),
    (synth.CI16, 2, 1, 16, 20),
    (synth.CI4, 1, 17, 64, 96),
    # beyond one 128-input row block: off-diagonal column tiles and a ragged
    # last row block (76 stations = 152 inputs, 80 = the paper's design target,
    # 130 = two full 64-column off-diagonal tiles plus a ragged one)
    (synth.CI16, 1, 76, 16, 70),
    (synth.CI8, 1, 80, 16, 64),
    (synth.CI16, 1, 130, 16, 40),
]


@pytest.mark.parametrize("fmt,SB,N,C,S", CASES)
def test_tf32_split_vs_oracle(fmt, SB, N, C, S):
    sigma = {synth.CI16: 100.0, synth.CI8: 20.0, synth.CI4: 2.5}[fmt]
    if fmt == synth.CI4:
        rng = np.random.default_rng(S)
        tau = rng.uniform(-5e-6, 5e-6, N)
        blk = synth.make_block(40 + N, fmt, SB, N, C, S, sigma=sigma,
                               tones=[synth.Tone(amp=3.0, channel=5, delays=tau)])
    else:
        blk, tau, _ = tone_block(70 + N + C, fmt, SB, N, C, S, sigma=sigma)
    ref = oracle.fx(blk.fmt, blk.raw, 16, C, S, blk.taps, FS, blk.centres, tau, tau)
    c = make_corr(blk, precision=4)
    c32 = make_corr(blk, precision=0)
    raw = torch.from_numpy(blk.raw).cuda()
    t = d(tau, torch.float64)
    fused = c.correlate(c.channelize_correct(raw, t, t))
    two = c.correlate(c.correct(c.channelize(raw), t, t))
    ffma = c32.correlate(c32.channelize_correct(raw, t, t))
    torch.cuda.synchronize()
    for vis in (fused, two):
        e = per_subband_rel(vis.cpu().numpy().astype(np.float64), ref)
        assert np.all(e < 1e-5), e
    e = per_subband_rel(fused.cpu().numpy().astype(np.float64), ffma.cpu().numpy().astype(np.float64))
    assert np.all(e < 1e-5), e
    c.close()
    c32.close()


def test_tf32_split_planar_operands_match_fp32_path():
    """The FP32 planar operands equal the FP32 interleaved corrected block
    (same fused kernel, same arithmetic, only the layout differs), and the
    padding is zero."""
    blk, tau, _ = tone_block(5, synth.CI16, 2, 7, 64, 50)
    c = make_corr(blk, precision=4)
    c32 = make_corr(blk, precision=0)
    raw = torch.from_numpy(blk.raw).cuda()
    t = d(tau, torch.float64)
    p = torch.full(c.corr_shape(), float("nan"), dtype=torch.float32, device="cuda")
    c.channelize_correct(raw, t, t, out=p)
    import paper_1801_04834_gb300 as fxg
    f = fxg.f32_unblock(c32.channelize_correct(raw, t, t), c.S)   # [SB][C][S][N][2][2]
    torch.cuda.synchronize()
    I, S = c.I, c.S
    re = p[:, :, 0, :I, :S].permute(0, 1, 3, 2)               # [SB][C][S][I]
    im = p[:, :, 1, :I, :S].permute(0, 1, 3, 2)
    f = f.reshape(c.SB, c.C, S, I, 2)
    assert torch.equal(re, f[..., 0]) and torch.equal(im, f[..., 1])
    assert torch.all(p[:, :, :, I:, :] == 0) and torch.all(p[:, :, :, :, S:] == 0)
    c.close()
    c32.close()


def test_tf32_split_limits():
    blk = synth.make_block(1, synth.CI16, 1, 513, 16, 8)
    with pytest.raises(RuntimeError):
        make_corr(blk, precision=4)                             # more than 512 stations
    blk = synth.make_block(1, synth.CI16, 1, 4, 16, 8)
    with pytest.raises(RuntimeError):
        make_corr(blk, precision=4, operand_scale=0.5)          # no operand scaling in FP32


def _einsum_vis(y):
    """y [SB][C][S][N][2] complex128 -> vis [SB][C][B][4][2] (b = j(j+1)/2 + i, pq = 2p + q)."""
    SB, C, S, N, _ = y.shape
    v = np.einsum("bcsip,bcsjq->bcijpq", y, np.conj(y))
    out = np.zeros((SB, C, N * (N + 1) // 2, 4, 2))
    for j in range(N):
        for i in range(j + 1):
            b = j * (j + 1) // 2 + i
            blk = v[:, :, i, j].reshape(SB, C, 4)
            out[:, :, b, :, 0] = blk.real
            out[:, :, b, :, 1] = blk.imag
    return out


@pytest.mark.parametrize("exact,N", [(True, 24), (False, 24), (False, 64), (False, 76), (True, 100),
                                     (False, 200)])
def test_tf32_split_kernel_on_given_operands(exact, N):
    """fx_correlate alone on planar FP32 operands written here: values with
    13 zero low mantissa bits (hi only, lo = 0) and arbitrary FP32 values
    (lo carries the low bits) against an FP64 einsum. The second kind also
    checks that the TF32 MMAs read a raw FP32 operand as its hi part (the
    kernel leaves the low bits in place): a TF32 MMA that used the low bits
    or rounded them would be off by up to 2^-11 per product. Bound: each TMEM
    accumulator chain spans 64 spectra = 32 MMAs (4 TF32 + 4 BF16 per 16
    spectra), and the tensor core's accumulation may lose up to 2^-24 of the
    running sum per MMA (32 x 2^-24 = 1.9e-6), plus the BF16 rounding of the
    cross terms (zero mean) and the dropped lo lo' term (below 2^-20); chains
    are summed in IEEE FP32. So 4e-6 normwise, against 1e-5 for the FP32 path
    end to end.
    Station counts above 64 exercise off-diagonal column tiles (A and B from
    different inputs) and ragged diagonal tiles of the last row block.
    Per baseline, max |dV_ij| / sqrt(|V_ii| |V_jj|) (so cross terms are not
    hidden by the autocorrelations in the norm) stays below 2e-5."""
    SB, C, S = 2, 16, 96
    blk = synth.make_block(1, synth.CI16, SB, N, C, S)
    c = make_corr(blk, precision=4)
    rng = np.random.default_rng(11 + exact)
    y = (rng.normal(size=(SB, C, S, N, 2)) + 1j * rng.normal(size=(SB, C, S, N, 2))) * 100.0
    y = y.astype(np.complex64)
    if exact:
        bits = y.view(np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
        y = bits.view(np.float32).view(np.complex64)
    planar = np.zeros(c.corr_shape(), dtype=np.float32)          # [SB][C][2][I_pad][S_pad]
    yi = y.reshape(SB, C, S, 2 * N).transpose(0, 1, 3, 2)         # [SB][C][I][S]
    planar[:, :, 0, :2 * N, :S] = yi.real
    planar[:, :, 1, :2 * N, :S] = yi.imag
    vis = c.correlate(torch.from_numpy(planar).cuda())
    torch.cuda.synchronize()
    ref = _einsum_vis(y.astype(np.complex128))
    got = vis.cpu().numpy().astype(np.float64)
    e = per_subband_rel(got, ref)
    assert np.all(e < 4e-6), e
    assert baseline_max_rel(got, ref, N) < 2e-5
    c.close()
