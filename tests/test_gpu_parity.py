"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic): the FIR+FFT and the correction run
in FP32 with O(T + log2 C) rounding steps of 2^-24 each, so the channelised
and corrected samples agree with FP64 to a few 1e-7 relative; the FP32
X-stage sums S products, adding about sqrt(S) * 2^-24. The FP32 path is held
to the end-to-end bound of 1e-5 normwise relative visibility error per
subband (||dV||_F / ||V||_F), and each step to 2e-6.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle_pins import cplx

pytestmark = pytest.mark.gpu

FS = synth.SAMPLE_RATE_HZ


def fx():
    import paper_1801_04834_gb300 as fxg
    return fxg


def rel_err(got, ref, axis=None):
    d = np.linalg.norm((got - ref).reshape(got.shape[0], -1) if axis == 0 else (got - ref).ravel())
    r = np.linalg.norm(ref.reshape(ref.shape[0], -1) if axis == 0 else ref.ravel())
    return d / r


def per_subband_rel(got, ref):
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)


def baseline_max_rel(got, ref, N):
    """max over (subband, channel, i <= j, p, q) of |dV_ij^pq| / sqrt(|V_ii^pp| |V_jj^qq|)
    on vis arrays [SB][C][B][4][2] (the second error metric of the error
    reading: each cross term is judged against its own stations' powers, not
    against the autocorrelation-dominated norm)."""
    g = got[..., 0] + 1j * got[..., 1]
    r = ref[..., 0] + 1j * ref[..., 1]
    jj, ii = np.meshgrid(np.arange(N), np.arange(N))
    up = ii <= jj
    i, j = ii[up], jj[up]
    b = j * (j + 1) // 2 + i
    auto = np.abs(r[:, :, (np.arange(N) * (np.arange(N) + 3)) // 2])      # [SB][C][N][4]
    worst = 0.0
    for p in range(2):
        for q in range(2):
            den = np.sqrt(auto[:, :, i, 3 * p] * auto[:, :, j, 3 * q])
            num = np.abs(g[:, :, b, 2 * p + q] - r[:, :, b, 2 * p + q])
            # stations whose data were all flagged have zero autos: judged against the largest power
            worst = max(worst, float(np.max(num / np.maximum(den, 1e-9 * auto.max() + 1e-300))))
    return worst


def make_corr(blk, precision=0, **kw):
    fxg = fx()
    return fxg.Correlator(blk.n_stations, blk.n_subbands, blk.n_channels, blk.n_spectra,
                          taps=blk.taps, centres=blk.centres, n_taps=blk.n_taps, fmt=blk.fmt,
                          precision=precision, **kw)


def tone_block(seed, fmt, SB, N, C, S, T=16, sigma=100.0, amp=50.0, ripple=False):
    rng = np.random.default_rng(seed)
    tau = rng.uniform(-5e-6, 5e-6, N)
    rip = synth.bandpass_ripple(rng, N, C) if ripple else None
    tones = [synth.Tone(amp=amp, channel=int(rng.integers(1, C)), delays=tau, ripple=rip)]
    blk = synth.make_block(seed, fmt, SB, N, C, S, n_taps=T, sigma=sigma, tones=tones)
    return blk, tau, rip


CHANNELIZE_CASES = [
    # (fmt, SB, N, C, T, S)  -- S values span several 16-spectrum rounds plus a ragged tail
    (synth.CI16, 2, 3, 64, 16, 37),
    (synth.CI16, 1, 5, 16, 16, 40),
    (synth.CI8, 2, 2, 256, 16, 19),
    (synth.CI16, 1, 9, 16, 4, 33),
    (synth.CI8, 1, 3, 64, 8, 130),
    (synth.CI16, 1, 1, 64, 16, 1),
]


@pytest.mark.parametrize("fmt,SB,N,C,T,S", CHANNELIZE_CASES)
def test_channelize_parity(fmt, SB, N, C, T, S):
    blk, _, _ = tone_block(100 + S, fmt, SB, N, C, S, T=T, sigma=20.0 if fmt == synth.CI8 else 100.0)
    ref = oracle.channelize(fmt, blk.raw, T, C, S, blk.taps)
    c = make_corr(blk)
    raw = torch.from_numpy(blk.raw).cuda()
    got = c.channelize(raw).cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert rel_err(got, ref) < 2e-6
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) < 2e-5 * scale * np.sqrt(C)


@pytest.mark.parametrize("fmt,SB,N,C,T,S,stations", [
    # sizes whose grid keeps 4 rounds per CTA (ragged last round): the FIR/FFT
    # buffer ping-pong of the warp-specialised PPF runs past its first reuse
    (synth.CI16, 2, 64, 64, 16, 1210, [0, 31, 63]),
    (synth.CI8, 4, 64, 16, 8, 2430, [2, 3, 60]),
    # the LOFAR 16-bit shape on 13 subbands: 64 rounds per CTA as in the benchmark
    (synth.CI16, 13, 64, 64, 16, 3072, [5, 62]),
])
def test_channelize_multiround(fmt, SB, N, C, T, S, stations):
    """Long CTA runs of the PPF against the oracle on a few stations (the
    channeliser treats stations independently, so the oracle runs on those
    stations' samples alone)."""
    rng = np.random.default_rng(S + C)
    amp = 60 if fmt == synth.CI8 else 300
    dt = np.int8 if fmt == synth.CI8 else np.int16
    raw = rng.integers(-amp, amp + 1, size=(SB, N, (S + T - 1) * C, 2, 2), dtype=dt)
    taps = synth.kaiser_sinc_taps(T, C)
    fxg = fx()
    c = fxg.Correlator(N, SB, C, S, taps=taps, centres=synth.subband_centres(SB), n_taps=T, fmt=fmt, precision=0)
    sbs, st = torch.tensor([0, SB - 1]), torch.tensor(stations)
    got = c.channelize(torch.from_numpy(raw).cuda())[sbs.cuda()][:, st.cuda()].cpu().numpy().astype(np.float64)
    ref = oracle.channelize(fmt, raw[[0, SB - 1]][:, stations], T, C, S, taps)
    assert got.shape == ref.shape
    assert rel_err(got, ref) < 2e-6
    assert np.max(np.abs(got - ref)) < 2e-5 * np.sqrt(np.mean(ref ** 2)) * np.sqrt(C)
    c.close()


@pytest.mark.parametrize("N,C,S,ramp", [(8, 64, 48, False), (5, 16, 70, True), (3, 256, 9, True)])
def test_correct_f32_parity(N, C, S, ramp):
    rng = np.random.default_rng(7 + N)
    SB = 2
    chan = synth.channelised_noise(11 + N, SB, N, 2, C, S, sigma=300.0)
    centres = synth.subband_centres(SB)
    tb = rng.uniform(-5e-6, 5e-6, N)
    te = tb + (rng.uniform(-3e-8, 3e-8, N) if ramp else 0.0)
    bp = rng.uniform(0.7, 1.3, (N, C))
    g = synth.random_gains(rng, N)
    ref = oracle.correct(chan, FS, centres, tb, te, bandpass=bp, gains=g)
    blk = synth.Block(0, SB, N, 2, C, 16, S, None, synth.kaiser_sinc_taps(16, C), centres)
    c = make_corr(blk)
    dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    unblock = fx().f32_unblock
    got = unblock(c.correct(dev(chan), dev(tb, torch.float64), dev(te, torch.float64), bandpass=dev(bp),
                            gains=dev(g)), S).cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert rel_err(got, ref) < 2e-6
    # without bandpass / gains (NULL pointers mean ones)
    ref0 = oracle.correct(chan, FS, centres, tb, te)
    got0 = unblock(c.correct(dev(chan), dev(tb, torch.float64), dev(te, torch.float64)), S).cpu().numpy()
    assert rel_err(got0.astype(np.float64), ref0) < 2e-6


@pytest.mark.parametrize("form", ["auto", "2x4", "3mult"])
@pytest.mark.parametrize("N,C,S,SB", [(8, 64, 100, 2), (64, 4 * 4, 33, 1), (1, 16, 20, 3),
                                      (13, 16, 65, 1), (76, 16, 40, 1), (96, 16, 17, 1),
                                      (150, 16, 45, 1), (64, 64, 70, 3), (17, 16, 9, 2), (18, 64, 31, 1)])
def test_correlate_f32_parity(N, C, S, SB, form):
    """FFMA X-stage in each form (4 x 4 tiles by default from 16 stations,
    2 x 4 tiles, 2 x 4 tiles with the three-multiplication product), ragged
    station counts."""
    if C not in (16, 64, 256):
        pytest.skip("channel count not built")
    corr = synth.noise(21 + N, (SB, C, S, N, 2, 2))
    ref = oracle.correlate(corr)
    blk = synth.Block(0, SB, N, 2, C, 16, S, None, synth.kaiser_sinc_taps(16, C),
                      synth.subband_centres(SB))
    c = make_corr(blk, xf32_form=form)
    blocked = fx().f32_block(torch.from_numpy(corr).to("cuda", torch.float32))
    got = c.correlate(blocked).cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert np.all(per_subband_rel(got, ref) < 2e-6)


def run_chain(c, blk, tb, te, bandpass=None, gains=None):
    raw = torch.from_numpy(blk.raw).cuda()
    d = lambda a, dt=torch.float32: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    chan = c.channelize(raw)
    corr = c.correct(chan, d(tb, torch.float64), d(te, torch.float64), bandpass=d(bandpass), gains=d(gains))
    return c.correlate(corr)


def test_end_to_end_tiny_fp32():
    """8 stations x 2 pols, 1 subband at 150 MHz, 64 channels, 16 taps, 768
    spectra, int16 noise sigma=100 plus a tone delayed +-5 us per station."""
    blk, tau, _ = tone_block(synth.BASE_SEED + 0, synth.CI16, 1, 8, 64, 768)
    ref = oracle.fx(blk.fmt, blk.raw, 16, 64, 768, blk.taps, FS, blk.centres, tau, tau)
    c = make_corr(blk)
    got = run_chain(c, blk, tau, tau).cpu().numpy().astype(np.float64)
    e = per_subband_rel(got, ref)
    assert np.all(e < 1e-5), e
    # max |dV_ij| / sqrt(|V_ii| |V_jj|) over all baselines
    V = cplx(ref)
    G = cplx(got)
    auto = np.abs(V[:, :, [j * (j + 1) // 2 + j for j in range(8)], 0])
    worst = 0.0
    for j in range(8):
        for i in range(j + 1):
            b = j * (j + 1) // 2 + i
            den = np.sqrt(auto[:, :, i] * auto[:, :, j])
            worst = max(worst, float(np.max(np.abs(G[:, :, b] - V[:, :, b]) / den[..., None])))
    assert worst < 1e-5


@pytest.mark.parametrize("fmt,SB,N,C,S", [(synth.CI8, 2, 5, 256, 33), (synth.CI16, 3, 11, 16, 50)])
def test_end_to_end_ragged_fp32(fmt, SB, N, C, S):
    blk, tau, rip = tone_block(31 + N, fmt, SB, N, C, S, ripple=True,
                               sigma=20.0 if fmt == synth.CI8 else 100.0)
    te = tau + 1e-8
    rng = np.random.default_rng(5)
    g = synth.random_gains(rng, N)
    ref = oracle.fx(blk.fmt, blk.raw, 16, C, S, blk.taps, FS, blk.centres, tau, te,
                    bandpass=1.0 / rip, gains=g)
    c = make_corr(blk)
    got = run_chain(c, blk, tau, te, bandpass=1.0 / rip, gains=g).cpu().numpy().astype(np.float64)
    assert np.all(per_subband_rel(got, ref) < 1e-5)


def test_deterministic():
    blk, tau, _ = tone_block(3, synth.CI16, 1, 6, 64, 64)
    c = make_corr(blk)
    a = run_chain(c, blk, tau, tau).cpu()
    b = run_chain(c, blk, tau, tau).cpu()
    assert torch.equal(a, b)


def test_shape_and_dtype_checks():
    fxg = fx()
    blk, tau, _ = tone_block(3, synth.CI16, 1, 4, 16, 20)
    c = make_corr(blk)
    with pytest.raises(ValueError):
        c.channelize(torch.zeros(10, dtype=torch.int16, device="cuda"))
    with pytest.raises(TypeError):
        c.channelize(torch.zeros(c.raw_shape(), dtype=torch.int8, device="cuda"))
    with pytest.raises(fxg.FxError):
        # misaligned output pointer is rejected by the library
        buf = torch.zeros(int(np.prod(c.chan_shape())) + 1, dtype=torch.float32, device="cuda")
        raw = torch.zeros(c.raw_shape(), dtype=torch.int16, device="cuda")
        from paper_1801_04834_gb300 import _abi
        import ctypes
        _abi.check(c.lib.fx_channelize(c.handle, ctypes.c_void_p(raw.data_ptr()),
                                       ctypes.c_void_p(buf.data_ptr() + 4), None), "fx_channelize")
