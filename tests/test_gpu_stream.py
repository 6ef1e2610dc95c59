"""Streaming form (fx_stream_block) against the FP64 oracle.

A continuous stream of K blocks per (subband, station, pol) is generated on
the host. For block k the oracle gets, per station n, the window of stream
samples [k*S*C - (T-1)*C - d_n, (k+1)*S*C - d_n) (zeros before the stream
starts), i.e. the FIR history carried from the previous block and the
integer coarse delay d_n applied by whole samples (paper, Sec. "Signal
processing with GPU kernels" and Sec. "Software architecture"). The GPU gets
only the S*C new samples of each call and keeps the history itself.

Checks: (1) without flags the streamed corrected block is bit-identical to
fx_channelize_correct on the host-assembled window (the assembly and the
history move bytes only); (2) corrected samples and visibilities against the
oracle at the FP32 bounds of the non-streaming path; (3) per-baseline counts
of valid spectra exact (sums of 0/1 products); (4) fx_stream_reset restarts
the stream; (5) an out-of-range coarse shift is clamped, reported through
fx_poll_status and the call's buffers stay in bounds.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import baseline_max_rel, per_subband_rel

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ
SIGMA = {synth.CI16: 100.0, synth.CI8: 20.0, synth.CI4: 2.5}


def fxg():
    import paper_1801_04834_gb300 as m
    return m


def make_stream(seed, fmt, SB, N, n_samples):
    rng = np.random.default_rng(seed)
    z = rng.normal(0, SIGMA[fmt], (SB, N, n_samples, 2)) + 1j * rng.normal(0, SIGMA[fmt], (SB, N, n_samples, 2))
    return synth.quantise(z, fmt)          # [SB][N][L][P][2 or 1]


def window(stream, k, S, C, T, shifts):
    """Raw block of block k: station n reads its stream d_n samples late."""
    SB, N, L, P, W = stream.shape
    out = np.zeros((SB, N, (S + T - 1) * C, P, W), dtype=stream.dtype)
    for n in range(N):
        start = k * S * C - (T - 1) * C - int(shifts[n])
        lo = max(start, 0)
        hi = start + (S + T - 1) * C
        out[:, n, lo - start:] = stream[:, n, lo:hi]
    return out


def dev(a, dt):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


CASES = [  # (fmt, SB, N, C, S, max_shift, precision)
    (synth.CI16, 2, 5, 64, 24, 40, 0),
    (synth.CI8, 1, 7, 256, 9, 300, 0),
    (synth.CI4, 2, 4, 16, 33, 17, 0),
    (synth.CI16, 1, 9, 64, 20, 64, 1),
    (synth.CI8, 1, 3, 16, 17, 0, 0),
    (synth.CI16, 2, 6, 64, 40, 30, 4),          # the FP32-accurate tensor-core path (TF32 split)
]


@pytest.mark.parametrize("fmt,SB,N,C,S,M,precision", CASES)
def test_stream_blocks_vs_oracle(fmt, SB, N, C, S, M, precision):
    T, K = 16, 4
    rng = np.random.default_rng(1000 + N * C + S)
    taps = synth.kaiser_sinc_taps(T, C)
    centres = synth.subband_centres(SB)
    stream = make_stream(synth.BASE_SEED + C + N, fmt, SB, N, K * S * C)
    bp = (1.0 / synth.bandpass_ripple(rng, N, C)).astype(np.float32)
    g = synth.random_gains(rng, N)
    c = fxg().Correlator(N, SB, C, S, taps=taps, centres=centres, n_taps=T, fmt=fmt, precision=precision,
                         streaming=True, max_coarse_shift=M)
    rdt = c.raw_dtype()
    for k in range(K):
        shifts = rng.integers(0, M + 1, N).astype(np.int32)
        tb = rng.uniform(-2e-6, 2e-6, N)
        te = tb + rng.uniform(-2e-8, 2e-8, N)
        flags = None
        if k % 2 == 1:
            flags = (rng.random((N, S)) > 0.2).astype(np.float32)
            flags[0, :] = 0.0 if k == 3 else flags[0, :]      # one station lost for a whole block
        new = torch.from_numpy(np.ascontiguousarray(stream[:, :, k * S * C:(k + 1) * S * C])).cuda()
        args = dict(bandpass=dev(bp, torch.float32), gains=dev(g, torch.float32))
        tb_d, te_d = dev(tb, torch.float64), dev(te, torch.float64)
        corr, vis, counts = c.stream_block(new, tb_d, te_d, coarse_shift=dev(shifts, torch.int32),
                                           flags=dev(flags, torch.float32), **args)
        torch.cuda.synchronize()
        win = window(stream, k, S, C, T, shifts)
        if flags is None:
            direct = c.channelize_correct(torch.from_numpy(win).cuda(), tb_d, te_d, **args)
            torch.cuda.synchronize()
            assert torch.equal(corr, direct), k
            assert counts is None
        chan_ref = oracle.channelize(fmt, win, T, C, S, taps)
        corr_ref = oracle.correct(chan_ref, FS, centres, tb, te, bp, g, flags)
        vis_ref = oracle.correlate(corr_ref)
        if precision == 0:
            got = fxg().f32_unblock(corr, S).cpu().numpy().astype(np.float64)
            e = np.linalg.norm(got - corr_ref) / np.linalg.norm(corr_ref)
            assert e < 2e-6, (k, e)
        got_vis = vis.cpu().numpy().astype(np.float64)
        e = per_subband_rel(got_vis, vis_ref)
        fp32 = precision in (0, 4)                      # FFMA or TF32 split: FP32 accuracy
        assert np.all(e < (1e-5 if fp32 else 5e-3)), (k, e)
        # per baseline, max |dV_ij| / sqrt(|V_ii| |V_jj|): 5e-5 for FP32 accuracy, 1e-3 for FP16 operands
        assert baseline_max_rel(got_vis, vis_ref, N) < (5e-5 if fp32 else 1e-3), k
        if flags is not None:
            cnt_ref = oracle.baseline_counts(flags, N, S)
            assert np.array_equal(counts.cpu().numpy().astype(np.float64), cnt_ref), k
    c.close()


def test_stream_reset_and_bad_shift():
    fmt, SB, N, C, S, M, T = synth.CI16, 1, 4, 64, 12, 10, 16
    taps = synth.kaiser_sinc_taps(T, C)
    centres = synth.subband_centres(SB)
    stream = make_stream(7, fmt, SB, N, 3 * S * C)
    c = fxg().Correlator(N, SB, C, S, taps=taps, centres=centres, fmt=fmt, streaming=True, max_coarse_shift=M)
    zero = torch.zeros(N, dtype=torch.float64, device="cuda")
    shifts = torch.tensor([0, 3, 10, 7], dtype=torch.int32, device="cuda")

    def blk(k):
        return torch.from_numpy(np.ascontiguousarray(stream[:, :, k * S * C:(k + 1) * S * C])).cuda()

    first = [c.stream_block(blk(k), zero, zero, coarse_shift=shifts)[1].clone() for k in range(3)]
    c.stream_reset()
    again = [c.stream_block(blk(k), zero, zero, coarse_shift=shifts)[1].clone() for k in range(3)]
    torch.cuda.synchronize()
    for a, b in zip(first, again):
        assert torch.equal(a, b)
    # the first block after a reset sees zeros before the stream, the later ones do not
    assert not torch.equal(first[0], first[1])

    lib = c.lib
    code = ctypes.c_int(0)
    assert lib.fx_poll_status(c.handle, ctypes.byref(code)) == 0 and code.value == 0
    bad = torch.tensor([0, M + 5, -2, 1], dtype=torch.int32, device="cuda")
    c.stream_block(blk(0), zero, zero, coarse_shift=bad)
    torch.cuda.synchronize()
    rc = lib.fx_poll_status(c.handle, ctypes.byref(code))
    assert rc == fxg()._abi.FX_ERR_INVALID and code.value == 5
    assert lib.fx_poll_status(c.handle, ctypes.byref(code)) == 0     # cleared
    c.close()


def test_stream_requires_flag():
    fmt, SB, N, C, S = synth.CI16, 1, 2, 16, 4
    c = fxg().Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB))
    zero = torch.zeros(N, dtype=torch.float64, device="cuda")
    new = torch.zeros(c.new_shape(), dtype=torch.int16, device="cuda")
    with pytest.raises(RuntimeError):
        c.stream_block(new, zero, zero)
    c.close()
